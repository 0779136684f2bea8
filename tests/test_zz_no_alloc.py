"""sub_running_mean_noalloc: the running mean for callers that cannot allocate device memory.

Such a caller owns no allocator (for example a plug-in that is handed device buffers
by a host framework which manages all device memory, or a loop that must never enter
cudaMalloc), so the entry point keeps its scratch in a static device array.  Here it
is called through the C ABI on device buffers, twice in a row with different sizes
and windows (the shared scratch keeps the previous call's contents), on the legacy
default stream and on a stream of the caller's; its output is compared with the FP64
oracle's running mean (App. D, Eq. running mean) and with the context path's
(sub_estimate, SUB_MEAN), and the free device memory must not move across calls.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2602_18560_gb300 import gbsub, synth

pytestmark = pytest.mark.gpu

CASES = [(1249681, 1000), (70001, 257)]  # the 4-yr band first, then a smaller one


def _context_mean(P, W):
    k_lo = int(np.ceil(1e-4 * synth.YEAR))
    f_max = (k_lo + P.size - 1 + 0.25) / synth.YEAR
    with gbsub.Subtraction(T_obs=synth.YEAR, window=W, estimator=gbsub.MEAN, f_max=f_max) as s:
        assert s.grid[0] == P.size
        return s.estimate(P)


def _rel_err(got, ref):
    zero = ref == 0
    assert np.all(got[zero] == 0)
    return float(np.max(np.abs(got[~zero] - ref[~zero]) / ref[~zero])) if (~zero).any() else 0.0


def _spectra():
    rng = np.random.default_rng(11)
    out = []
    for n, W in CASES:
        P = rng.exponential(1.0, n) * 10 ** rng.uniform(-50, -38, n)
        P[rng.random(n) < 0.2] = 0.0
        out.append((P, W))
    return out


def _call(L, x, out, n, W, stream):
    rc = L.sub_running_mean_noalloc(ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), n, W,
                                    ctypes.c_void_p(stream) if stream else None)
    assert rc == gbsub.OK, L.sub_last_error(None).decode()


def test_noalloc_running_mean_matches_the_oracle_twice():
    import torch
    assert torch.cuda.is_available()
    L = gbsub.lib()
    cases = _spectra()
    refs = [oracle.smooth(oracle.MEAN, W, P) for P, W in cases]
    ctx_refs = [_context_mean(P, W) for P, W in cases]
    dev = [(torch.from_numpy(P).cuda(),
            torch.full((P.size,), float("nan"), dtype=torch.float64, device="cuda"))
           for P, _ in cases]
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    # the first call on the device looks up the array's address; after it, calls allocate
    # nothing, so the device's free memory stays where it is
    _call(L, dev[0][0], dev[0][1], cases[0][0].size, cases[0][1], None)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for (P, W), (x, out), ref, cref in zip(cases, dev, refs, ctx_refs):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        _call(L, x, out, P.size, W, None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert _rel_err(got, ref) <= 1e-12
        assert _rel_err(got, cref) <= 1e-12
    # on a stream of the caller's, the larger case again
    (P, W), (x, out), ref = cases[0], dev[0], refs[0]
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    _call(L, x, out, P.size, W, s.cuda_stream)
    s.synchronize()
    assert _rel_err(out.cpu().numpy(), ref) <= 1e-12
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    L = gbsub.lib()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.sub_running_mean_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                    1310721, 100, None)
    assert rc == gbsub.EINVAL
    assert "1310720" in L.sub_last_error(None).decode()
    rc = L.sub_running_mean_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                    8, 8193, None)
    assert rc == gbsub.EINVAL
