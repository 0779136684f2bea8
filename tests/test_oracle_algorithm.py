"""Pins for the oracle's subtraction loop (App. D, Algorithm).

  * closed forms: one bright single-bin source with the mean and the median;
  * identity: when no source exceeds the threshold the run takes one iteration
    and S_gal is the estimator of the full deposited power;
  * invariants: S_gal shrinks pointwise from one iteration to the next, the
    resolved set only grows, and the pre-filter factor kappa cannot change the
    result (S_n >= S_instr makes rho <= rho_0);
  * brute force: tiny catalogs against a naive re-implementation written here
    from the definitions (explicit loops, math.fsum, sorted medians).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_18560_gb300 import synth

C = 729.0 / 512.0
BRIGHT_FMAX = 2e-3
BRIGHT_W = 30


def _single_source_case(est, W, A, T=oracle.YEAR):
    k_lo, n = oracle.grid(T)
    j0 = n // 2
    f = (k_lo + j0) / T
    prm = oracle.make_params(T_obs=T, estimator=est, window=W)
    return prm, k_lo, n, j0, f


@pytest.mark.parametrize("A", [1e-21, 3e-23])
def test_single_bright_source_mean_closed_form(A):
    W = 1000
    prm, k_lo, n, j0, f = _single_source_case(oracle.MEAN, W, A)
    S, R = oracle.tables(prm.T_obs, k_lo, n, True)
    T = prm.T_obs
    P = T * R[j0] * A * A / 5.0
    rho2_first = 4 * P / (S[j0] + P / W)
    out = oracle.run(prm, [A], [f], [0.0], trace_iters=3)
    first = out["trace"][0]
    # first estimate: P/W on the W bins whose window holds j0, zero elsewhere
    nz = np.nonzero(first)[0]
    assert nz.min() == j0 - (W - 1 - W // 2) and nz.max() == j0 + W // 2
    np.testing.assert_allclose(first[nz], P / W, rtol=1e-13)
    if rho2_first > 49:
        assert out["resolved"][0] and out["iterations"] == 2
        assert np.all(out["S_gal"] == 0.0)
    else:
        assert not out["resolved"][0] and out["iterations"] == 1
        np.testing.assert_array_equal(out["S_gal"], first)


@pytest.mark.parametrize("W", [3, 1000])
def test_single_source_median_is_zero_foreground(W):
    for A, resolved in ((1e-21, True), (1e-24, False)):
        prm, k_lo, n, j0, f = _single_source_case(oracle.MEDIAN, W, A)
        S, R = oracle.tables(prm.T_obs, k_lo, n, True)
        rho2 = 4 * prm.T_obs * R[j0] * A * A / 5.0 / S[j0]
        assert (rho2 > 49) == resolved
        out = oracle.run(prm, [A], [f], [0.0])
        assert np.all(out["S_gal"] == 0.0)
        assert out["resolved"][0] == resolved
        assert out["iterations"] == (2 if resolved else 1)


def test_identity_when_nothing_exceeds_threshold():
    T = oracle.YEAR
    A, f, fdot = synth.catalog(3000, 21)
    A = A * 1e-3  # far below threshold
    for est in (oracle.MEAN, oracle.MEDIAN, oracle.MEDIAN_MEAN):
        prm = oracle.make_params(T_obs=T, estimator=est, window=200)
        out = oracle.run(prm, A, f, fdot)
        assert out["iterations"] == 1 and out["converged"] and out["n_resolved"] == 0
        k_lo, n = oracle.grid(T)
        S, R = oracle.tables(T, k_lo, n, True)
        P = oracle.power(T, R, oracle.deposit(T, k_lo, n, A, f, fdot))
        np.testing.assert_array_equal(out["S_gal"], oracle.smooth(est, 200, P))


@pytest.fixture(scope="module")
def bright_catalog():
    # a dense, bright catalog on a narrow band so that every estimator needs
    # several iterations (the median ignores isolated bright bins)
    A, f, fdot = synth.catalog(300000, 31, synth.Population(2.0, 2.0))
    keep = f < BRIGHT_FMAX
    return A[keep] * 2.5, f[keep], fdot[keep]


@pytest.mark.parametrize("est", [oracle.MEAN, oracle.MEDIAN, oracle.MEDIAN_MEAN])
def test_monotone_iterations_and_growing_resolved_set(bright_catalog, est):
    A, f, fdot = bright_catalog
    T = oracle.YEAR
    prm = oracle.make_params(T_obs=T, estimator=est, window=BRIGHT_W, f_max=BRIGHT_FMAX)
    out = oracle.run(prm, A, f, fdot, trace_iters=100)
    tr = out["trace"]
    assert out["converged"] and out["iterations"] >= 3
    for i in range(1, tr.shape[0]):
        assert np.all(tr[i] <= tr[i - 1])
    np.testing.assert_array_equal(out["S_gal"], tr[-1])
    # every resolved source is a candidate, every unresolved candidate is now below threshold
    k_lo, n = oracle.grid(T, f_max=BRIGHT_FMAX)
    S, R = oracle.tables(T, k_lo, n, True)
    r2 = oracle.snr2(T, k_lo, n, S, R, out["S_gal"], A, f, fdot)
    assert np.all(r2[~out["resolved"]] <= 49.0)
    r20 = oracle.snr2(T, k_lo, n, S, R, None, A, f, fdot)
    assert np.all(r20[out["resolved"]] > 49.0)
    assert np.all(r2 <= r20 * (1 + 1e-15))
    # the resolved set grows: re-running with max_iter = i gives nested sets
    prev = None
    for i in range(1, out["iterations"] + 1):
        p = oracle.make_params(T_obs=T, estimator=est, window=BRIGHT_W, f_max=BRIGHT_FMAX,
                               max_iter=i)
        o = oracle.run(p, A, f, fdot)
        if prev is not None:
            assert np.all(o["resolved"] >= prev)
        prev = o["resolved"]
    np.testing.assert_array_equal(prev, out["resolved"])


def test_prefilter_invariance(bright_catalog):
    A, f, fdot = bright_catalog
    T = oracle.YEAR
    outs = [oracle.run(oracle.make_params(T_obs=T, estimator=oracle.MEDIAN_MEAN, window=BRIGHT_W,
                                          f_max=BRIGHT_FMAX, kappa=k), A, f, fdot)
            for k in (0.0, 1 / 7.0, 1.0)]
    assert outs[0]["n_candidates"] == A.size
    assert outs[0]["n_candidates"] > outs[1]["n_candidates"] > outs[2]["n_candidates"]
    for o in outs[1:]:
        np.testing.assert_array_equal(o["resolved"], outs[0]["resolved"])
        np.testing.assert_array_equal(o["S_gal"], outs[0]["S_gal"])
        assert o["iterations"] == outs[0]["iterations"]


def test_max_iter_exhaustion_reports_not_converged(bright_catalog):
    A, f, fdot = bright_catalog
    T = oracle.YEAR
    kw = dict(T_obs=T, estimator=oracle.MEAN, window=BRIGHT_W, f_max=BRIGHT_FMAX)
    full = oracle.run(oracle.make_params(**kw), A, f, fdot)
    assert full["iterations"] >= 3
    o = oracle.run(oracle.make_params(max_iter=1, **kw), A, f, fdot)
    assert not o["converged"] and o["iterations"] == 1 and o["n_resolved"] > 0
    # S_gal is re-estimated from the final resolved set
    k_lo, n = oracle.grid(T, f_max=BRIGHT_FMAX)
    S, R = oracle.tables(T, k_lo, n, True)
    P = oracle.power(T, R, oracle.deposit(T, k_lo, n, A, f, fdot, o["resolved"].astype(np.uint8)))
    np.testing.assert_array_equal(o["S_gal"], oracle.smooth(oracle.MEAN, BRIGHT_W, P))


# ---------------------------------------------------------------- brute force


def _naive_run(T, f_lo, f_hi, W, est, A, f, fdot, rho_th=7.0, kappa=1 / 7.0, max_iter=100):
    k_lo = math.ceil(f_lo * T)
    k_hi = math.floor(f_hi * T)
    n = k_hi - k_lo + 1
    Sins = [oracle.s_instr((k_lo + j) / T, True) for j in range(n)]
    Rr = [oracle.response((k_lo + j) / T, True) for j in range(n)]

    def pieces(fs, fd):
        u0 = fs * T
        u1 = u0 + fd * (T * T)
        lo, hi = min(u0, u1), max(u0, u1)
        if hi == lo:
            k = math.floor(lo + 0.5)
            return [(k - k_lo, 1.0)] if k_lo <= k <= k_hi else []
        out = []
        for k in range(math.floor(lo + 0.5), math.floor(hi + 0.5) + 1):
            a, b = max(lo, k - 0.5), min(hi, k + 0.5)
            if b > a and k_lo <= k <= k_hi:
                out.append((k - k_lo, (b - a) / (hi - lo)))
        return out

    pcs = [pieces(fs, fd) for fs, fd in zip(f, fdot)]

    def rho2(s, Sg):
        return 4 * math.fsum(T / 5 * Rr[j] * A[s] ** 2 * w / (Sins[j] + Sg[j]) for j, w in pcs[s])

    def est_w(P):
        def bounds(j):
            s = j - W // 2
            return max(0, s), min(n - 1, s + W - 1)

        def med(v):
            v = sorted(v)
            c = len(v)
            return v[c // 2] if c % 2 else 0.5 * (v[c // 2 - 1] + v[c // 2])

        mean = [math.fsum(P[a:b + 1]) / (b - a + 1) for a, b in map(bounds, range(n))]
        if est == oracle.MEAN:
            return mean
        m = [C * med(P[a:b + 1]) for a, b in map(bounds, range(n))]
        if est == oracle.MEDIAN:
            return m
        return [math.fsum(m[a:b + 1]) / (b - a + 1) for a, b in map(bounds, range(n))]

    zero = [0.0] * n
    cand = [s for s in range(len(A)) if rho2(s, zero) >= (kappa * rho_th) ** 2]
    res = set()
    for it in range(1, max_iter + 1):
        D = [[] for _ in range(n)]
        for s in range(len(A)):
            if s not in res:
                for j, w in pcs[s]:
                    D[j].append(A[s] ** 2 * w)
        P = [T / 5 * Rr[j] * math.fsum(D[j]) for j in range(n)]
        Sg = est_w(P)
        new = [s for s in cand if s not in res and rho2(s, Sg) > rho_th**2]
        if not new:
            return Sg, res, it
        res.update(new)
    raise AssertionError("naive run did not converge")


N_TINY = 8


def _tiny_case(seed):
    """5-20 sources packed into 80 of ~280 bins, amplitudes from just above the
    instrument noise to far above it, a mix of monochromatic and chirping sources."""
    rng = np.random.default_rng(100 + seed)
    T = 2.0e5
    f_lo, f_hi = 1e-4, 1.5e-3          # bins 20 .. 300
    N = int(rng.integers(5, 21))
    f = (100 + rng.uniform(0, 80, N)) / T
    fdot = rng.choice([0.0, 1.0], N) * rng.uniform(0, 8, N) / T**2
    S_mid = oracle.s_instr(5e-4, True) / oracle.response(5e-4, True)
    A = np.sqrt(S_mid / T) * 10 ** rng.uniform(0.5, 2.5, N)
    W = int(rng.choice([13, 16, 20, 25]))
    return T, f_lo, f_hi, W, A, f, fdot


@pytest.mark.parametrize("seed", range(N_TINY))
@pytest.mark.parametrize("est", [oracle.MEAN, oracle.MEDIAN, oracle.MEDIAN_MEAN])
def test_brute_force_tiny_catalogs(seed, est):
    T, f_lo, f_hi, W, A, f, fdot = _tiny_case(seed)
    Sg, res, it = _naive_run(T, f_lo, f_hi, W, est, A.tolist(), f.tolist(), fdot.tolist())
    prm = oracle.make_params(T_obs=T, f_min=f_lo, f_max=f_hi, window=W, estimator=est)
    out = oracle.run(prm, A, f, fdot)
    assert out["iterations"] == it
    assert set(np.nonzero(out["resolved"])[0].tolist()) == res
    np.testing.assert_allclose(out["S_gal"], Sg, rtol=1e-13, atol=0)


def test_brute_force_exercises_several_iterations():
    # guard that the tiny cases above are not trivial for any estimator
    for est in (oracle.MEAN, oracle.MEDIAN, oracle.MEDIAN_MEAN):
        iters = []
        for seed in range(N_TINY):
            T, f_lo, f_hi, W, A, f, fdot = _tiny_case(seed)
            prm = oracle.make_params(T_obs=T, f_min=f_lo, f_max=f_hi, window=W, estimator=est)
            iters.append(oracle.run(prm, A, f, fdot)["iterations"])
        assert max(iters) >= 3 and min(iters) >= 2
