"""Coarse graining through the C ABI (Sec. "Coarse-graining of the data") against the
oracle: identical bin counts, bin-averaged spectrum and frequencies to rounding."""
import numpy as np
import pytest

import oracle
from paper_2602_18560_gb300 import gbsub, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    gbsub.lib()


def same(got, ref, rtol):
    (S, f, c), (S0, f0, c0) = got, ref
    np.testing.assert_array_equal(c, c0)
    np.testing.assert_array_equal(np.isnan(S), np.isnan(S0))
    np.testing.assert_array_equal(np.isnan(f), np.isnan(f0))
    ok = ~np.isnan(S0)
    np.testing.assert_allclose(S[ok], S0[ok], rtol=rtol, atol=0)
    np.testing.assert_allclose(f[ok], f0[ok], rtol=1e-14, atol=0)


@pytest.mark.parametrize("T,nbins", [(synth.YEAR, 100), (4 * synth.YEAR, 100),
                                     (2 * synth.YEAR, 1), (synth.YEAR, 5000), (1.0e5, 100)])
def test_random_series_matches_oracle(T, nbins):
    k_lo, n = oracle.grid(T)
    x = np.random.default_rng(nbins).exponential(1.0, n) * 10 ** np.random.default_rng(7).uniform(-44, -38, n)
    with gbsub.Subtraction(T_obs=T) as s:
        assert s.grid == (n, k_lo)
        got = s.coarse_grain(x, nbins)
    same(got, oracle.coarse_grain(T, 1e-4, 1e-2, k_lo, x, nbins), 1e-13)


def test_noise_psd_and_device_series():
    import torch
    T = 2 * synth.YEAR
    k_lo, n = oracle.grid(T)
    S_instr, _ = oracle.tables(T, k_lo, n, True)
    x = np.random.default_rng(3).random(n) * 1e-41
    with gbsub.Subtraction(T_obs=T) as s:
        got = s.coarse_grain(x, 100, add_instr=True)
        dev = s.coarse_grain(torch.from_numpy(x).cuda(), 100, add_instr=True)
    same(got, oracle.coarse_grain(T, 1e-4, 1e-2, k_lo, S_instr + x, 100), 1e-12)
    for a, b in zip(got, dev):
        np.testing.assert_array_equal(a, b.cpu().numpy())


def test_coarse_grained_foreground_of_a_run():
    w = synth.workload("nb1e4_1yr")
    A, f, fdot = synth.catalog(w.n_sources, w.seed, w.pop)
    A = A * 30.0  # a visible foreground
    prm = oracle.make_params(T_obs=w.T_obs, estimator=gbsub.MEDIAN_MEAN, window=1000)
    ref = oracle.run(prm, A, f, fdot)
    with gbsub.Subtraction(T_obs=w.T_obs, window=1000, estimator=gbsub.MEDIAN_MEAN) as s:
        with pytest.raises(gbsub.SubError):
            s.coarse_grain()  # no run yet
        s.load(A, f, fdot)
        s.run()
        got = s.coarse_grain()
        again = s.coarse_grain(s.spectrum())
    for a, b in zip(got, again):
        np.testing.assert_array_equal(a, b)
    k_lo, n = oracle.grid(w.T_obs)
    assert np.any(got[0] > 0)
    same(got, oracle.coarse_grain(w.T_obs, 1e-4, 1e-2, k_lo, ref["S_gal"], 100), 1e-10)
