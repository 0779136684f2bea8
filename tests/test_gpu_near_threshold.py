"""SNR decisions at the threshold (App. D: a candidate is resolved when rho > rho_th), through
the C ABI, against the FP64 oracle.

Sources are placed at rho = rho_th (1 + delta) for delta in +-{1e-10, 1e-8, 1e-6, 1e-5, 1e-4}
on top of a dense faint background, with one-bin, three-bin, ten-bin and forty-bin (a
whole warp walks them, and recomputes them in FP64 across its lanes) and downward sweeps.  The sources sit 400 bins apart and the estimators are the median
and the median then the mean over 101 bins: a resolvable source is among the brightest
bins of every window it touches, so S_gal at its bins does not depend on its exact
amplitude, and the amplitude that gives the wanted rho can be solved for against the
oracle's own S_gal of the first iteration.

Asserted:
  - FP64 (FP32 screen with the FP64 recomputation inside its margin) and strict FP64 take
    the oracle's decision on every source with |delta| >= 1e-9; the |delta| = 1e-10 ones
    are counted by sub_stats.n_near, and any disagreement is among them;
  - the screened run recomputes some decisions in FP64 (n_exact > 0);
  - mixed precision disagrees with the oracle only on decisions its FP32 value could not
    settle (n_uncertain), and counts every source within 1e-6 of rho_th among those;
  - the FP32 screen's measured error over every kept candidate of a large run stays below
    the bound the screen's margin is built on.
"""
import numpy as np
import pytest

import oracle
from paper_2602_18560_gb300 import gbsub, synth

pytestmark = pytest.mark.gpu

T = synth.YEAR
F_MAX = 3e-3
W = 101
DELTAS = [s * d for d in (1e-10, 1e-8, 1e-6, 1e-5, 1e-4) for s in (1.0, -1.0)]
# (u0 - k, du) in bin units: the sweep [u0, u0 + du] of a source centred on bin k
KINDS = {"single": (-0.3, 0.5), "three": (-0.3, 2.6), "ten": (-0.3, 9.4),
         "forty": (-0.3, 39.6), "down": (0.2, -3.3)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    gbsub.lib()


def background(k_lo, n, S, R, frac=0.04):
    """Three faint single-bin sources per bin, each of power frac * S_instr (rho_0 = 0.4)."""
    j = np.repeat(np.arange(n), 3)
    off = np.tile([-0.3, 0.0, 0.3], n)
    f = (k_lo + j + off) / T
    A = np.sqrt(5.0 * frac * S[j] / (T * R[j]))
    return A, f, np.zeros_like(f)


def source_rows(k_lo):
    rows = []
    for i, (delta, kind) in enumerate((d, k) for d in DELTAS for k in KINDS):
        k = k_lo + 1500 + 400 * i
        a, du = KINDS[kind]
        rows.append((delta, kind, (k + a) / T, du / T**2))
    return rows


def build_placed():
    """The catalog (background, then the test sources at their solved amplitudes) and the
    delta of every test source, per estimator (oracle only)."""
    k_lo, n = oracle.grid(T, 1e-4, F_MAX)
    S, R = oracle.tables(T, k_lo, n, True)
    Ab, fb, fdb = background(k_lo, n, S, R)
    rows = source_rows(k_lo)
    ft = np.array([r[2] for r in rows])
    fdt = np.array([r[3] for r in rows])
    delta = np.array([r[0] for r in rows])
    # nominal amplitudes (rho about rho_th against S_instr alone), then the first
    # iteration's S_gal of the oracle with them in place
    c0 = oracle.snr2(T, k_lo, n, S, R, None, np.ones_like(ft), ft, fdt)
    A0 = 7.0 / np.sqrt(c0)
    out = {}
    for est in (gbsub.MEDIAN, gbsub.MEDIAN_MEAN):
        prm = oracle.make_params(T_obs=T, f_max=F_MAX, window=W, estimator=est, max_iter=1)
        cat = [np.concatenate([Ab, A0]), np.concatenate([fb, ft]), np.concatenate([fdb, fdt])]
        Sg1 = oracle.run(prm, *cat, trace_iters=1)["trace"][0]
        c = oracle.snr2(T, k_lo, n, S, R, Sg1, np.ones_like(ft), ft, fdt)
        At = 7.0 * (1.0 + delta) / np.sqrt(c)
        cat[0] = np.concatenate([Ab, At])
        chk = oracle.run(prm, *cat, trace_iters=1)["trace"][0]
        # the first S_gal does not depend on the test amplitudes (they only move the top of
        # the windows' order)
        assert np.array_equal(chk.view(np.uint64), Sg1.view(np.uint64))
        rho = np.sqrt(oracle.snr2(T, k_lo, n, S, R, Sg1, At, ft, fdt))
        assert np.all(np.abs(rho / 7.0 - 1.0 - delta) < 1e-14)
        out[est] = (cat, len(Ab), delta)
    return out


@pytest.fixture(scope="module")
def placed():
    return build_placed()


@pytest.mark.parametrize("est", [gbsub.MEDIAN, gbsub.MEDIAN_MEAN])
def test_decisions_at_the_threshold_match_the_oracle(placed, est):
    cat, nb_bg, delta = placed[est]
    ref = oracle.run(oracle.make_params(T_obs=T, f_max=F_MAX, window=W, estimator=est), *cat)
    ref_t = ref["resolved"][nb_bg:]
    # the oracle itself resolves exactly the sources placed above the threshold
    assert np.array_equal(ref_t, delta > 0)
    assert not ref["resolved"][:nb_bg].any()
    tiny = np.abs(delta) < 1e-9
    for prec in (gbsub.FP64, gbsub.FP64_STRICT):
        with gbsub.Subtraction(T_obs=T, f_max=F_MAX, window=W, estimator=est,
                               precision=prec) as s:
            s.load(*cat)
            st = s.run()
            res = s.resolved().astype(bool)
            sg = s.spectrum()
        got = res[nb_bg:]
        assert np.array_equal(got[~tiny], ref_t[~tiny]), np.nonzero(got != ref_t)
        assert np.array_equal(res[:nb_bg], ref["resolved"][:nb_bg])
        assert st.n_near >= int(tiny.sum())
        assert int(np.sum(got != ref_t)) <= st.n_near
        assert st.n_uncertain == 0
        nz = ref["S_gal"] != 0
        assert np.all(sg[~nz] == 0)
        assert np.max(np.abs(sg[nz] / ref["S_gal"][nz] - 1.0)) <= 1e-10
        if prec == gbsub.FP64:
            assert st.n_exact > 0   # the screen handed the near ones to FP64
    with gbsub.Subtraction(T_obs=T, f_max=F_MAX, window=W, estimator=est,
                           precision=gbsub.MIXED) as s:
        s.load(*cat)
        st = s.run()
        res = s.resolved().astype(bool)
    assert st.n_near == 0
    assert st.n_uncertain >= int(np.sum(np.abs(delta) <= 1e-6))
    assert int(np.sum(res != ref["resolved"])) <= st.n_uncertain


def test_fp32_screen_error_stays_inside_its_bound():
    # every kept candidate of a realistic run (1e6 sources, 4 yr, W = 1000, median then
    # mean): the FP32 screen against the FP64 value in the oracle's order of summation, and
    # that value against the oracle's own rho^2 on the run's S_gal
    w = synth.workload("nb1e6_4yr")
    A, f, fdot = synth.catalog(w.n_sources, w.seed, w.pop)
    with gbsub.Subtraction(T_obs=w.T_obs, window=1000, estimator=gbsub.MEDIAN_MEAN) as s:
        s.load(A, f, fdot)
        s.run()
        chk = s.snr_check()
        sg = s.spectrum()
        nb, k_lo = s.grid
    assert chk["src"].size > 100
    ex = chk["exact"]
    ok = ex > 0
    err = np.abs(chk["screen"][ok].astype(np.float64) / ex[ok] - 1.0)
    bound = 2.2e-6 + 2e-7 * chk["nbins"][ok]   # the screen's bound (its margin is twice it)
    assert np.all(err < bound), float(np.max(err / bound))
    S, R = oracle.tables(w.T_obs, k_lo, nb, True)
    src = chk["src"]
    orc = oracle.snr2(w.T_obs, k_lo, nb, S, R, sg, A[src], f[src], fdot[src])
    assert np.max(np.abs(ex / orc - 1.0)) < 1e-12
