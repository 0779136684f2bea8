"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance (stated for the FP64 path): S_gal relative error <= 1e-10 in every bin where
the oracle's S_gal is non-zero, exact zeros where it is zero; the resolved set identical
except for sources whose rho is within 1e-9 of rho_th (counted); iteration counts equal.
"""
import numpy as np
import pytest

import oracle
from paper_2602_18560_gb300 import gbsub, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    gbsub.lib()


def rel_err(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    zero = ref == 0
    assert np.all(got[zero] == 0), "non-zero where the oracle is zero"
    if np.all(zero):
        return 0.0
    return float(np.max(np.abs(got[~zero] - ref[~zero]) / ref[~zero]))


def near_threshold(A, f, fdot, T, f_max, S_gal, rho_th=7.0, f_min=1e-4):
    k_lo, n = oracle.grid(T, f_min, f_max)
    S, R = oracle.tables(T, k_lo, n, True)
    r = np.sqrt(oracle.snr2(T, k_lo, n, S, R, S_gal, A, f, fdot))
    return np.abs(r - rho_th) / rho_th < 1e-9


def compare_run(A, f, fdot, T, est, W, f_max=1e-2, f_min=1e-4, **kw):
    prm = oracle.make_params(T_obs=T, estimator=est, window=W, f_max=f_max, f_min=f_min, **kw)
    ref = oracle.run(prm, A, f, fdot)
    with gbsub.Subtraction(T_obs=T, window=W, estimator=est, f_max=f_max, f_min=f_min,
                           **{k: v for k, v in kw.items()}) as s:
        s.load(A, f, fdot)
        st = s.run()
        sg = s.spectrum()
        res = s.resolved().astype(bool)
        hist = s.history()
    assert st.n_bins == ref["n_bins"] and st.k_lo == ref["k_lo"]
    err = rel_err(sg, ref["S_gal"])
    assert err <= RTOL, err
    diff = res != ref["resolved"]
    if diff.any():
        amb = near_threshold(A[diff], f[diff], fdot[diff], T, f_max, ref["S_gal"], f_min=f_min)
        assert amb.all(), "resolved sets differ at %d sources" % diff.sum()
    assert st.iterations == ref["iterations"]
    assert st.converged == ref["converged"]
    assert st.n_resolved == ref["n_resolved"]
    assert st.n_candidates >= ref["n_candidates"]
    assert hist.sum() == st.n_resolved and len(hist) == st.iterations
    return st, sg, res, ref


def test_grid_and_tables_match_oracle():
    for T in (synth.YEAR, 4 * synth.YEAR):
        for tdi2 in (0, 1):
            with gbsub.Subtraction(T_obs=T, window=100, tdi2=tdi2) as s:
                nb, k_lo = s.grid
                S, R = s.tables()
            k2, n2 = oracle.grid(T)
            assert (nb, k_lo) == (n2, k2)
            So, Ro = oracle.tables(T, k2, n2, bool(tdi2))
            assert rel_err(S, So) < 1e-13
            assert rel_err(R, Ro) < 1e-13


def _band_for(n, T=synth.YEAR, f_min=1e-4):
    k_lo, _ = oracle.grid(T, f_min, 1e-2)
    return (k_lo + n - 1 + 0.25) / T


def _spectrum(n, seed):
    rng = np.random.default_rng(seed)
    P = rng.exponential(1.0, n) * 10 ** rng.uniform(-50, -38, n)
    P[rng.random(n) < 0.15] = 0.0
    P[rng.random(n) < 0.05] = P[min(1, n - 1)]  # exact ties
    return P


@pytest.mark.parametrize("W", [1, 2, 3, 4, 31, 32, 33, 64, 100, 999, 1000, 1001, 2000, 3000, 4096])
@pytest.mark.parametrize("n", [1, 5, 777, 5000, 20011])
def test_estimators_match_oracle(W, n):
    T = synth.YEAR
    f_max = _band_for(n, T)
    P = _spectrum(n, W * 7 + n)
    for est in (gbsub.MEAN, gbsub.MEDIAN, gbsub.MEDIAN_MEAN):
        with gbsub.Subtraction(T_obs=T, window=W, estimator=est, f_max=f_max) as s:
            assert s.grid[0] == n
            got = s.estimate(P)
        ref = oracle.smooth(est, W, P)
        if est == gbsub.MEDIAN:
            np.testing.assert_array_equal(got, ref)  # selection: the same doubles
        else:
            assert rel_err(got, ref) <= 1e-12


def test_estimator_extreme_dynamic_range():
    # 70 decades: windows whose sum is far below the largest value use the direct sum
    T = synth.YEAR
    n = 6000
    f_max = _band_for(n, T)
    rng = np.random.default_rng(2)
    P = 10 ** rng.uniform(-100, -30, n)
    P[2000:2600] = 10 ** rng.uniform(-300, -280, 600)
    for est in (gbsub.MEAN, gbsub.MEDIAN_MEAN):
        with gbsub.Subtraction(T_obs=T, window=100, estimator=est, f_max=f_max) as s:
            got = s.estimate(P)
        assert rel_err(got, oracle.smooth(est, 100, P)) <= 1e-12


def test_estimator_all_zero_and_constant():
    T = synth.YEAR
    n = 3000
    f_max = _band_for(n, T)
    for est in (gbsub.MEAN, gbsub.MEDIAN, gbsub.MEDIAN_MEAN):
        with gbsub.Subtraction(T_obs=T, window=500, estimator=est, f_max=f_max) as s:
            assert np.all(s.estimate(np.zeros(n)) == 0.0)
            c = np.full(n, 3.25e-45)
            got = s.estimate(c)
        assert rel_err(got, oracle.smooth(est, 500, c)) <= 1e-12


@pytest.mark.parametrize("est", [gbsub.MEAN, gbsub.MEDIAN, gbsub.MEDIAN_MEAN])
def test_small_workload_1e4_sources(est):
    w = synth.workload("nb1e4_1yr")
    A, f, fdot = synth.catalog(w.n_sources, w.seed, w.pop)
    st, *_ = compare_run(A, f, fdot, w.T_obs, est, 1000)
    assert st.n_candidates > 0


@pytest.fixture(scope="module")
def dense():
    A, f, fdot = synth.catalog(300000, 31, synth.Population(2.0, 2.0))
    keep = f < 2e-3
    return A[keep] * 2.5, f[keep], fdot[keep]


@pytest.mark.parametrize("est", [gbsub.MEAN, gbsub.MEDIAN, gbsub.MEDIAN_MEAN])
@pytest.mark.parametrize("W", [30, 257])
def test_dense_catalog_many_iterations(dense, est, W):
    A, f, fdot = dense
    st, *_ = compare_run(A, f, fdot, synth.YEAR, est, W, f_max=2e-3)
    if W == 30:
        assert st.iterations >= 3


def test_widest_window_run(dense):
    # W = 8192: the widest chunks (eight elements per sorting thread) through a whole run,
    # the re-sorts of chunks with few changed bins included
    A, f, fdot = dense
    keep = f < 1e-3
    compare_run(A[keep], f[keep], fdot[keep], synth.YEAR, gbsub.MEDIAN_MEAN, 8192, f_max=1e-3)


def test_chirping_sources_span_many_bins():
    A, f, fdot = synth.catalog(20000, 5, synth.Population(2.0, 2.0))
    fdot = fdot * 3e3   # sweeps of up to hundreds of bins, some leaving the band
    A = A * 4.0
    for est in (gbsub.MEAN, gbsub.MEDIAN_MEAN):
        compare_run(A, f, fdot, synth.YEAR, est, 200)


def test_workload_1e6_sources_4yr():
    w = synth.workload("nb1e6_4yr")
    A, f, fdot = synth.catalog(w.n_sources, w.seed, w.pop)
    st, *_ = compare_run(A, f, fdot, w.T_obs, gbsub.MEDIAN_MEAN, 1000)
    assert st.n_resolved > 100


def test_kappa_and_max_iter_and_rtol(dense):
    A, f, fdot = dense
    T = synth.YEAR
    for kappa in (0.0, 1.0):
        compare_run(A, f, fdot, T, gbsub.MEDIAN_MEAN, 30, f_max=2e-3, kappa=kappa)
    # max_iter exhaustion: S_gal re-estimated from the final resolved set
    prm = oracle.make_params(T_obs=T, estimator=gbsub.MEAN, window=30, f_max=2e-3, max_iter=2)
    ref = oracle.run(prm, A, f, fdot)
    assert not ref["converged"]
    with gbsub.Subtraction(T_obs=T, window=30, estimator=gbsub.MEAN, f_max=2e-3, max_iter=2) as s:
        s.load(A, f, fdot)
        st = s.run()
        assert st.status == gbsub.ENOTCONVERGED and not st.converged and st.iterations == 2
        assert rel_err(s.spectrum(), ref["S_gal"]) <= RTOL
        np.testing.assert_array_equal(s.resolved().astype(bool), ref["resolved"])
    # an S_n tolerance stops the loop early, at the same iteration as the oracle
    compare_run(A, f, fdot, T, gbsub.MEAN, 30, f_max=2e-3, conv_rtol=1e-3)


def test_screened_fp64_equals_strict_fp64(dense):
    # the FP32 screen with an FP64 recomputation inside its error margin must give the
    # same bits as computing every rho^2 in FP64
    A, f, fdot = dense
    outs = []
    for prec in (gbsub.FP64, gbsub.FP64_STRICT):
        for est in (gbsub.MEAN, gbsub.MEDIAN_MEAN):
            with gbsub.Subtraction(T_obs=synth.YEAR, window=30, estimator=est, f_max=2e-3,
                                   precision=prec) as s:
                s.load(A, f, fdot)
                st = s.run()
                outs.append((prec, est, s.spectrum(), s.resolved(), st))
    for i in range(2):
        a, b = outs[i], outs[i + 2]
        assert np.array_equal(a[2].view(np.uint64), b[2].view(np.uint64))
        assert np.array_equal(a[3], b[3])
        assert a[4].iterations == b[4].iterations
        assert a[4].n_exact < 0.01 * max(1, a[4].n_live * a[4].iterations)
        assert b[4].n_exact > 0


def test_live_candidates_and_paper_candidate_count(dense):
    # n_candidates counts rho_0 >= kappa rho_th as the paper does; only rho_0 > rho_th can
    # ever be resolved and only those are kept
    A, f, fdot = dense
    T = synth.YEAR
    k_lo, n = oracle.grid(T, 1e-4, 2e-3)
    S, R = oracle.tables(T, k_lo, n, True)
    r0 = oracle.snr2(T, k_lo, n, S, R, None, A, f, fdot)
    with gbsub.Subtraction(T_obs=T, window=30, estimator=gbsub.MEAN, f_max=2e-3) as s:
        s.load(A, f, fdot)
        st = s.run()
    assert st.n_candidates == int(np.sum(r0 >= 1.0))
    assert st.n_live == int(np.sum(r0 > 49.0))


def test_edge_catalogs():
    T = synth.YEAR
    with gbsub.Subtraction(T_obs=T, window=100, estimator=gbsub.MEDIAN_MEAN) as s:
        # empty catalog
        s.load(np.zeros(0), np.zeros(0), np.zeros(0))
        st = s.run()
        assert st.iterations == 1 and st.converged and st.n_resolved == 0
        assert np.all(s.spectrum() == 0.0)
        # every source outside the band
        A = np.full(10, 1e-21)
        f = np.concatenate([np.full(5, 5e-5), np.full(5, 2e-2)])
        s.load(A, f, np.zeros(10))
        st = s.run()
        assert st.n_candidates == 0 and st.n_resolved == 0 and np.all(s.spectrum() == 0.0)
    # one bright monochromatic source: resolved in the first pass, S_gal = 0 after
    k_lo, n = oracle.grid(T)
    f0 = (k_lo + n // 2) / T
    compare_run(np.array([1e-21]), np.array([f0]), np.array([0.0]), T, gbsub.MEAN, 1000)
    compare_run(np.array([1e-21]), np.array([f0]), np.array([0.0]), T, gbsub.MEDIAN, 1000)


def test_runs_are_bitwise_deterministic(dense):
    A, f, fdot = dense
    outs = []
    for _ in range(3):
        with gbsub.Subtraction(T_obs=synth.YEAR, window=30, estimator=gbsub.MEDIAN_MEAN,
                               f_max=2e-3) as s:
            s.load(A, f, fdot)
            s.run()
            outs.append((s.spectrum(), s.resolved()))
    for sg, r in outs[1:]:
        assert np.array_equal(sg.view(np.uint64), outs[0][0].view(np.uint64))
        assert np.array_equal(r, outs[0][1])


def test_device_buffers_and_reuse():
    import torch
    A, f, fdot = synth.catalog(5000, 9, synth.Population(3.0, 2.0))
    A = A * 3
    ref = oracle.run(oracle.make_params(T_obs=synth.YEAR, window=300, estimator=gbsub.MEDIAN,
                                        f_max=3e-3), A, f, fdot)
    dev = [torch.from_numpy(x).cuda() for x in (A, f, fdot)]
    with gbsub.Subtraction(T_obs=synth.YEAR, window=300, estimator=gbsub.MEDIAN, f_max=3e-3) as s:
        for _ in range(2):  # the same context runs twice with a reloaded catalog
            s.load(*dev)
            s.run()
            out = torch.empty(s.grid[0], dtype=torch.float64, device="cuda")
            s.spectrum(out)
            m = torch.empty(A.size, dtype=torch.uint8, device="cuda")
            s.resolved(m)
            assert rel_err(out.cpu().numpy(), ref["S_gal"]) <= RTOL
            np.testing.assert_array_equal(m.cpu().numpy().astype(bool), ref["resolved"])


def test_errors_are_reported():
    T = synth.YEAR
    with gbsub.Subtraction(T_obs=T, window=100) as s:
        with pytest.raises(gbsub.SubError) as ei:
            gbsub.sub_run(s.ctx)
        assert ei.value.code == gbsub.ESTATE
        # a power beyond the fixed-point range
        s.load(np.array([1e-12]), np.array([3e-3]), np.array([0.0]))
        with pytest.raises(gbsub.SubError) as ei:
            s.run()
        assert ei.value.code == gbsub.ERANGE
    # a device memory budget too small for the catalog buffers
    with gbsub.Subtraction(T_obs=T, window=100, hbm_budget=64 << 20) as s:
        with pytest.raises(gbsub.SubError) as ei:
            s.load(np.zeros(10_000_000), np.zeros(10_000_000), np.zeros(10_000_000))
        assert ei.value.code == gbsub.EBUDGET


def mixed_vs_oracle(A, f, fdot, T, est, W, f_max=1e-2):
    """Mixed precision (FP32 SNR decisions, FP32 median selection, exact fixed-point sums)
    against the FP64 oracle: every source decided differently lies within the FP32 screen's
    error of rho_th, and S_gal is within 1e-5 away from the bins of those sources."""
    prm = oracle.make_params(T_obs=T, estimator=est, window=W, f_max=f_max)
    ref = oracle.run(prm, A, f, fdot)
    with gbsub.Subtraction(T_obs=T, window=W, estimator=est, f_max=f_max,
                           precision=gbsub.MIXED) as s:
        s.load(A, f, fdot)
        st = s.run()
        sg = s.spectrum()
        res = s.resolved().astype(bool)
    diff = np.nonzero(res != ref["resolved"])[0]
    if len(diff):
        k_lo, n = oracle.grid(T, 1e-4, f_max)
        S, R = oracle.tables(T, k_lo, n, True)
        r2 = oracle.snr2(T, k_lo, n, S, R, ref["S_gal"], A[diff], f[diff], fdot[diff])
        assert np.all(np.abs(r2 / 49.0 - 1.0) < 1e-4), r2
    keep = np.ones(len(sg), dtype=bool)
    k_lo = ref["k_lo"]
    for s_ in diff:
        k = int(np.floor(f[s_] * T + 0.5)) - k_lo
        keep[max(0, k - 2 * W):k + 2 * W + 1] = False
    err = rel_err(sg[keep], ref["S_gal"][keep])
    assert err <= 1e-5, err
    return st, ref, len(diff), err


@pytest.mark.parametrize("est", [gbsub.MEAN, gbsub.MEDIAN, gbsub.MEDIAN_MEAN])
def test_mixed_precision_dense_catalog(dense, est):
    A, f, fdot = dense
    st, ref, ndiff, err = mixed_vs_oracle(A, f, fdot, synth.YEAR, est, 30, f_max=2e-3)
    assert ndiff <= max(1, 1e-4 * ref["n_resolved"])


def test_mixed_precision_1e6_workload():
    w = synth.workload("nb1e6_4yr")
    A, f, fdot = synth.catalog(w.n_sources, w.seed, w.pop)
    st, ref, ndiff, err = mixed_vs_oracle(A, f, fdot, w.T_obs, gbsub.MEDIAN_MEAN, 1000)
    assert ndiff == 0
    assert st.iterations == ref["iterations"]


def test_non_finite_catalog_values_are_reported():
    A, f, fdot = synth.catalog(5000, 61, synth.Population(3.5, 2.0))
    for field, bad in ((0, np.inf), (1, np.nan), (2, -np.inf), (1, np.inf)):
        cat = [A.copy(), f.copy(), fdot.copy()]
        cat[field][1234] = bad
        with gbsub.Subtraction(T_obs=synth.YEAR, window=100) as s:
            s.load(*cat)
            with pytest.raises(gbsub.SubError) as ei:
                s.run()
            assert ei.value.code == gbsub.EINVAL
            s.load(A, f, fdot)   # a clean catalog runs normally afterwards
            assert s.run().n_sources == len(A)
