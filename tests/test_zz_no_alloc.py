"""sub_running_mean_noalloc: the running mean for callers that cannot allocate device memory.

Such a caller owns no allocator (for example a plug-in that is handed device buffers
by a host framework which manages all device memory, or a loop that must never enter
cudaMalloc), so the entry point keeps its scratch in a static device array.  Here it
is called through the C ABI on device buffers, twice in a row with different sizes
and windows (the shared scratch keeps the previous call's contents), and its output
is compared with the context path's running mean (sub_estimate, SUB_MEAN).
"""
import ctypes

import numpy as np
import pytest

from paper_2602_18560_gb300 import gbsub, synth

pytestmark = pytest.mark.gpu


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


def test_noalloc_running_mean_matches_context_path_twice():
    import torch
    assert torch.cuda.is_available()
    L = gbsub.lib()
    rng = np.random.default_rng(11)
    cases = [(1249681, 1000), (70001, 257)]  # the 4-yr band first, then a smaller one
    for n, W in cases:
        P = rng.exponential(1.0, n) * 10 ** rng.uniform(-50, -38, n)
        P[rng.random(n) < 0.2] = 0.0
        x = torch.from_numpy(P).cuda()
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = L.sub_running_mean_noalloc(ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), n, W, None)
        assert rc == gbsub.OK, L.sub_last_error(None).decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _context_mean(P, W)
        assert _rel_err(got, ref) <= 1e-12


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
