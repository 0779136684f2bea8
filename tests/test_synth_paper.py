"""The paper's population model (Sec. II.B, Table I; App. A, Gaussian copula) as the
single-precision recipe the device generator implements: its special functions against
library evaluations, and its catalogs against the distributions the paper states.

Pinned:
  - the inverse normal CDF, the normal tail, log Gamma and the regularized incomplete gamma
    function against scipy, at single-precision accuracy;
  - the marginals: f follows p(f) ~ f^alpha_pl on [0.1, 10] mHz, log10(fdot) - mu_g a Gamma
    distribution (concentration alpha_g, rate beta_g), log10(f^(-2/3) A) - mu a log-normal of
    width sigma (Kolmogorov-Smirnov);
  - the copula: the rank correlation of f and fdot is that of a Gaussian copula of
    correlation rho, Spearman's rho_S = (6/pi) asin(rho/2) and Kendall's tau = (2/pi) asin(rho),
    whatever the marginals;
  - determinism: every source is a function of (seed, index), slices agree;
  - the prior draws stay inside the Table I ranges.
"""
import math

import numpy as np
import pytest

from paper_2602_18560_gb300 import synth

sp = pytest.importorskip("scipy.special")
st = pytest.importorskip("scipy.stats")


def test_inverse_normal_cdf():
    p = np.concatenate([np.geomspace(1e-30, 0.4999, 3000),
                        np.linspace(0.001, 0.999, 3000)]).astype(np.float32)
    got = synth.norm_ppf32(p).astype(np.float64)
    ref = sp.ndtri(p.astype(np.float64))
    assert np.all(np.abs(got - ref) <= 2e-6 * np.maximum(np.abs(ref), 0.5))
    # symmetry of the two halves (u on a grid where 1 - u is exact)
    u = (np.arange(10, 500, 7) / 1024.0).astype(np.float32)
    assert np.array_equal(synth.norm_ppf32(u), -synth.norm_ppf32(np.float32(1) - u))


def test_normal_tail_and_erfc():
    z = np.linspace(-8.0, 9.0, 4001).astype(np.float32)
    got = synth.norm_sf32(z).astype(np.float64)
    ref = sp.ndtr(-z.astype(np.float64))
    assert np.max(np.abs(got - ref) / ref) < 2e-5
    x = np.linspace(0.0, 9.0, 901).astype(np.float32)
    assert np.max(np.abs(synth.erfc32(x) / sp.erfc(x.astype(np.float64)) - 1)) < 2e-5


@pytest.mark.parametrize("a", [1.0, 1.37, 1.96, 2.5, 3.0])
def test_incomplete_gamma(a):
    gln = synth.lgamma32(a)
    assert abs(float(gln) - sp.gammaln(a)) < 1e-6
    x = np.geomspace(1e-6, 60.0, 4000).astype(np.float32)
    P, Q = synth.gamma_pq32(a, x, gln)
    xd = x.astype(np.float64)
    assert np.max(np.abs(P - sp.gammainc(a, xd))) < 2e-6
    ref_q = sp.gammaincc(a, xd)
    tail = ref_q > 1e-30
    assert np.max(np.abs(Q[tail] - ref_q[tail]) / ref_q[tail]) < 2e-5


POPS = [synth.PaperPopulation(),
        synth.PaperPopulation(alpha_pl=-3.7, alpha_g=2.6, beta_g=1.2, mu_g=-20.5, mu=-22.6,
                              sigma=0.27, rho=0.4),
        synth.PaperPopulation(alpha_pl=-2.1, alpha_g=1.0, beta_g=2.9, mu_g=-21.8, mu=-21.2,
                              sigma=0.11, rho=0.0)]


@pytest.fixture(scope="module", params=range(len(POPS)))
def sample(request):
    pop = POPS[request.param]
    A, f, fdot, lat = synth.catalog_paper(200_000, 1000 + request.param, pop, with_latent=True)
    return pop, A, f, fdot, lat


def test_marginals(sample):
    pop, A, f, fdot, (xi, am, z1, z2) = sample
    assert np.all((f >= 1e-4 * (1 - 1e-6)) & (f <= 1e-2 * (1 + 1e-6)))
    e = pop.alpha_pl + 1.0
    lo, hi = 1e-4 ** e, 1e-2 ** e

    def cdf_f(x):
        return (np.asarray(x) ** e - lo) / (hi - lo)

    assert st.kstest(f, cdf_f).pvalue > 1e-3
    assert st.kstest(xi, st.gamma(pop.alpha_g, scale=1.0 / pop.beta_g).cdf).pvalue > 1e-3
    assert st.kstest(am, st.lognorm(s=pop.sigma).cdf).pvalue > 1e-3
    # the catalog is built from them: fdot = 10^(mu_g + xi), A = f^(2/3) 10^(mu + am)
    assert np.allclose(np.log10(fdot) - pop.mu_g, xi, rtol=0, atol=2e-5 * (1 + np.abs(xi)))
    assert np.allclose(np.log10(f ** (-2.0 / 3.0) * A) - pop.mu, am, rtol=0, atol=3e-5)


def test_copula_rank_correlation(sample):
    pop, A, f, fdot, (xi, am, z1, z2) = sample
    rs = st.spearmanr(f, fdot).statistic
    expect = 6.0 / math.pi * math.asin(pop.rho / 2.0)
    assert abs(rs - expect) < 0.006, (rs, expect)
    n = 20_000
    tau = st.kendalltau(f[:n], fdot[:n]).statistic
    assert abs(tau - 2.0 / math.pi * math.asin(pop.rho)) < 0.012
    # the latent normals: standard, with correlation rho; the amplitude independent of both
    assert abs(np.mean(z1)) < 0.01 and abs(np.std(z1) - 1) < 0.01
    assert abs(np.mean(z2)) < 0.01 and abs(np.std(z2) - 1) < 0.01
    assert abs(np.corrcoef(z1, z2)[0, 1] - pop.rho) < 0.006
    assert abs(st.spearmanr(am, f).statistic) < 0.01


def test_deterministic_and_sliceable():
    pop = POPS[1]
    a = synth.catalog_paper(5000, 77, pop)
    b = synth.catalog_paper(5000, 77, pop, chunk=777)
    c = synth.catalog_paper(1000, 77, pop, start=3000)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y)
        assert np.array_equal(x[3000:4000], z)
    d = synth.catalog_paper(5000, 78, pop)
    assert not np.array_equal(a[1], d[1])


def test_prior_draws_inside_table_I():
    for i in range(200):
        pop, n_b = synth.paper_population_draw(5, i)
        for name, (lo, hi) in synth.PAPER_PRIOR.items():
            v = n_b if name == "n_b" else getattr(pop, name)
            assert lo <= v <= hi, (name, v)


def test_normal_draws_stay_bounded():
    # the uniforms behind the copula's and the amplitude's normals are never 0 or 1 (a 32-bit
    # word's float can round to 1, whose normal deviate would be unbounded): every normal stays
    # within 5.34 standard deviations, so no amplitude leaves the spectrum's range
    words = np.array([0, 1, 511, 512, 2**31, 2**32 - 513, 2**32 - 1], dtype=np.uint32)
    u = synth.u23f(words)
    assert np.all((u > 0) & (u < 1))
    z = synth.norm_ppf32(u)
    assert np.all(np.isfinite(z)) and np.max(np.abs(z)) < 5.34
