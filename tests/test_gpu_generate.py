"""On-device catalog generation (through the C ABI): the device produces synth.catalog_single
bit for bit, and a run on a fused generated catalog (sources generated inside the catalog
pass) equals, bit for bit, the run on the same catalog loaded from the host, which in turn
matches the oracle."""
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


POPS = [synth.Population(11.0 / 3.0, 2.0), synth.Population(3.0, 1.5),
        synth.Population(4.5, 3.0), synth.Population(1.0, 1.0), synth.Population(-2.0, 40.0)]


@pytest.mark.parametrize("pi", range(len(POPS)))
def test_device_catalog_equals_host_recipe(pi):
    pop = POPS[pi]
    n = 120_001
    ref = synth.catalog_single(n, 1000 + pi, pop)
    with gbsub.Subtraction(T_obs=synth.YEAR) as s:
        s.load_generated(n, 1000 + pi, pop, fused=False)
        got = s.catalog()
        for a, b in zip(got, ref):
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
        s.load_generated(n, 1000 + pi, pop, fused=True)
        part = s.catalog(77_777, 4_000)
        dev = s.catalog(5, 3_000, device=True)
    for a, b in zip(part, ref):
        assert np.array_equal(a, b[77_777:81_777])
    for a, b in zip(dev, ref):
        assert np.array_equal(a.cpu().numpy(), b[5:3_005])


def same_run(a, b):
    (st_a, sg_a, m_a), (st_b, sg_b, m_b) = a, b
    assert st_a.iterations == st_b.iterations and st_a.n_resolved == st_b.n_resolved
    assert np.array_equal(sg_a.view(np.uint64), sg_b.view(np.uint64))
    assert np.array_equal(m_a, m_b)


@pytest.mark.parametrize("precision", [gbsub.FP64, gbsub.MIXED])
def test_fused_generation_run_equals_loaded_catalog_run(precision):
    pop = synth.Population(3.3, 2.2)
    n, seed, T = 400_000, 77, 4 * synth.YEAR
    kw = dict(T_obs=T, window=1000, estimator=gbsub.MEDIAN_MEAN, precision=precision)
    out = []
    with gbsub.Subtraction(**kw) as s:
        s.load(*synth.catalog_single(n, seed, pop))
        out.append((s.run(), s.spectrum(), s.resolved()))
        for fused in (True, False, True):
            s.load_generated(n, seed, pop, fused=fused)
            out.append((s.run(), s.spectrum(), s.resolved()))
    for o in out[1:]:
        same_run(out[0], o)
    assert out[0][0].n_resolved > 0


def test_generated_catalog_run_matches_oracle():
    pop = synth.Population(11.0 / 3.0, 2.0)
    n, seed, T = 20_000, 5, synth.YEAR
    A, f, fdot = synth.catalog_single(n, seed, pop)
    prm = oracle.make_params(T_obs=T, estimator=gbsub.MEDIAN_MEAN, window=1000)
    ref = oracle.run(prm, A, f, fdot)
    with gbsub.Subtraction(T_obs=T, window=1000, estimator=gbsub.MEDIAN_MEAN) as s:
        s.load_generated(n, seed, pop, fused=True)
        st = s.run()
        sg = s.spectrum()
        res = s.resolved().astype(bool)
    assert st.iterations == ref["iterations"]
    assert np.array_equal(res, ref["resolved"])
    nz = ref["S_gal"] != 0
    assert np.all(sg[~nz] == 0)
    assert np.max(np.abs(sg[nz] - ref["S_gal"][nz]) / ref["S_gal"][nz]) <= 1e-10


def test_generation_arguments_are_checked():
    with gbsub.Subtraction(T_obs=synth.YEAR) as s:
        for bad in (dict(gamma=11.0), dict(shape=0.5), dict(shape=float("nan"))):
            args = dict(gamma=3.0, shape=2.0)
            args.update(bad)
            with pytest.raises(gbsub.SubError) as ei:
                gbsub.sub_load_generated(s.ctx, 100, 1, **args)
            assert ei.value.code == gbsub.EINVAL
        s.load_generated(1000, 1)
        with pytest.raises(gbsub.SubError):
            s.catalog(990, 20)
