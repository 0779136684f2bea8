"""The paper's population model drawn on the device (through the C ABI, sub_load_population):
the device produces synth.catalog_paper bit for bit, a run on a fused population catalog (the
sources generated inside the catalog pass) equals the run on the same catalog loaded from the
host and matches the FP64 oracle, and a served population job equals the same catalog run
alone."""
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


POPS = [synth.PaperPopulation(),
        synth.PaperPopulation(alpha_pl=-3.7, alpha_g=2.6, beta_g=1.2, mu_g=-20.5, mu=-22.6,
                              sigma=0.27, rho=0.4),
        synth.PaperPopulation(alpha_pl=-2.1, alpha_g=1.0, beta_g=2.9, mu_g=-21.8, mu=-21.2,
                              sigma=0.11, rho=0.0),
        synth.PaperPopulation(alpha_pl=-1.0, alpha_g=3.0, beta_g=1.0, mu_g=-20.0, mu=-23.0,
                              sigma=0.3, rho=0.999)]


@pytest.mark.parametrize("pi", range(len(POPS)))
def test_device_population_equals_host_recipe(pi):
    pop = POPS[pi]
    n = 150_001
    ref = synth.catalog_paper(n, 2000 + pi, pop)
    with gbsub.Subtraction(T_obs=synth.YEAR) as s:
        s.load_population(n, 2000 + pi, pop, fused=False)
        got = s.catalog()
        for a, b in zip(got, ref):
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
        s.load_population(n, 2000 + pi, pop, fused=True)
        part = s.catalog(99_999, 5_000)
    for a, b in zip(part, ref):
        assert np.array_equal(a, b[99_999:104_999])


def test_population_validation():
    with gbsub.Subtraction(T_obs=synth.YEAR) as s:
        for bad in (dict(rho=1.0), dict(alpha_g=0.5), dict(sigma=0.0), dict(beta_g=-1.0)):
            kw = {**synth.PaperPopulation().__dict__, **bad}
            with pytest.raises(gbsub.SubError) as ei:
                s.load_population(10, 1, synth.PaperPopulation(**kw))
            assert ei.value.code == gbsub.EINVAL


# a prior draw and a bright one (several iterations in the cut band)
RUN_POP = synth.PaperPopulation(alpha_pl=-2.4, alpha_g=2.0, beta_g=1.5, mu_g=-21.0, mu=-21.3,
                                sigma=0.25, rho=0.8)


def test_population_run_matches_oracle_and_loaded_run():
    n, seed, T, f_max = 400_000, 31, synth.YEAR, 3e-3
    A, f, fdot = synth.catalog_paper(n, seed, RUN_POP)
    prm = oracle.make_params(T_obs=T, estimator=gbsub.MEDIAN_MEAN, window=1000, f_max=f_max)
    ref = oracle.run(prm, A, f, fdot)
    assert ref["n_resolved"] > 20 and ref["iterations"] >= 2
    kw = dict(T_obs=T, window=1000, estimator=gbsub.MEDIAN_MEAN, f_max=f_max)
    with gbsub.Subtraction(**kw) as s:
        s.load(A, f, fdot)
        st0 = s.run()
        sg0, m0 = s.spectrum(), s.resolved()
        s.load_population(n, seed, RUN_POP, fused=True)
        st = s.run()
        sg, m = s.spectrum(), s.resolved()
    assert np.array_equal(sg.view(np.uint64), sg0.view(np.uint64)) and np.array_equal(m, m0)
    assert st.iterations == st0.iterations == ref["iterations"]
    assert np.array_equal(m.astype(bool), ref["resolved"])
    nz = ref["S_gal"] != 0
    assert np.all(sg[~nz] == 0)
    assert np.max(np.abs(sg[nz] / ref["S_gal"][nz] - 1.0)) <= 1e-10


def test_served_population_job_equals_solo_run():
    T = 2 * synth.YEAR
    nb = int(np.floor(1e-2 * T)) - int(np.ceil(1e-4 * T)) + 1
    jobs = [(300_000, 41, POPS[0]), (120_000, 42, RUN_POP), (1, 43, POPS[1])]
    outs = {}
    with gbsub.Server(max_inflight=3, window=1000, estimator=gbsub.MEDIAN_MEAN) as srv:
        for i, (n, seed, pop) in enumerate(jobs):
            outs[i] = (np.zeros(nb), np.zeros(n, dtype=np.uint8))
            srv.submit_population(i, T, n, seed, pop, *outs[i])
        got = {}
        while len(got) < len(jobs):
            for r in srv.poll(timeout_ms=2000):
                got[r["job_id"]] = r
    assert all(r["status"] in (gbsub.OK, gbsub.ENOTCONVERGED) for r in got.values())
    for i, (n, seed, pop) in enumerate(jobs):
        with gbsub.Subtraction(T_obs=T, window=1000, estimator=gbsub.MEDIAN_MEAN) as s:
            s.load_population(n, seed, pop, fused=True)
            s.run()
            assert np.array_equal(outs[i][0].view(np.uint64), s.spectrum().view(np.uint64))
            assert np.array_equal(outs[i][1], s.resolved())
