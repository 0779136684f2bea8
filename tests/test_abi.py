"""The C-ABI library builds and exports every function include/gbsub.h declares (no GPU needed:
nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

from paper_2602_18560_gb300 import build, gbsub

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "gbsub.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sub_[a-z_]+)\s*\(", txt,
                       flags=re.M)
    return sorted(set(names))


def test_header_declarations_found():
    names = _declared()
    for must in ("sub_create", "sub_load_catalog", "sub_run", "sub_get_spectrum",
                 "sub_get_resolved_mask", "sub_destroy"):
        assert must in names
    assert set(names) == set(gbsub.EXPORTS)


def test_library_builds_and_exports_all_symbols():
    path = build.build()
    L = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(L, name), name


def test_params_default_and_struct_layout():
    p = gbsub.sub_params_default()
    assert p.window == 2000 and p.rho_th == 7.0 and abs(p.kappa - 1 / 7) < 1e-16
    assert p.T_obs == 4 * gbsub.YEAR and p.tdi2 == 1 and p.estimator == gbsub.MEAN
    assert ctypes.sizeof(gbsub.sub_params) == 80
    assert ctypes.sizeof(gbsub.sub_stats) == 88


def test_invalid_parameters_rejected_before_any_device_call():
    # validation happens before the first CUDA call, so this runs without a GPU
    for bad in (dict(window=0), dict(window=100000), dict(T_obs=-1.0), dict(f_min=0.0),
                dict(f_max=1e-5), dict(estimator=7), dict(max_iter=0), dict(rho_th=0.0),
                dict(kappa=-1.0), dict(precision=5)):
        with pytest.raises(gbsub.SubError) as ei:
            gbsub.sub_create(gbsub.sub_params_default(**bad))
        assert ei.value.code == gbsub.EINVAL


def test_calls_without_a_context_are_rejected():
    # every call checks its context first and touches no device without one
    import ctypes as C
    L = gbsub.lib()
    buf = (C.c_double * 4)()
    n64 = (C.c_int64 * 4)()
    assert L.sub_load_generated(None, 10, 1, 3.0, 2.0, 1) == gbsub.EINVAL
    assert L.sub_get_catalog(None, buf, buf, buf, 0, 1, gbsub.HOST) == gbsub.EINVAL
    assert L.sub_coarse_grain(None, None, 0, 100, buf, buf, n64, gbsub.HOST) == gbsub.EINVAL
    assert L.sub_get_work(None, n64, 4) == gbsub.EINVAL
    assert L.sub_load_catalog(None, buf, buf, buf, 1, gbsub.HOST_MAPPED) == gbsub.EINVAL
    assert L.sub_run(None, None) == gbsub.EINVAL


def test_struct_layouts_match_the_c_header(tmp_path):
    # sizes and field offsets of every public struct as the C compiler lays them out
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "gbsub.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(sub_params), sizeof(sub_stats),
         sizeof(sub_server_params), sizeof(sub_job_result), sizeof(sub_server_stats));
  printf("%zu %zu %zu %zu\n", offsetof(sub_server_params, f_min),
         offsetof(sub_job_result, stats), offsetof(sub_job_result, latency_ms),
         offsetof(sub_server_stats, inflight));
  printf("%d %d %d\n", SUB_HOST, SUB_DEVICE, SUB_HOST_MAPPED);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = [int(x) for x in out[:5]]
    offs = [int(x) for x in out[5:9]]
    assert [int(x) for x in out[9:]] == [gbsub.HOST, gbsub.DEVICE, gbsub.HOST_MAPPED]
    assert sizes == [ctypes.sizeof(t) for t in (gbsub.sub_params, gbsub.sub_stats,
                                                gbsub.sub_server_params, gbsub.sub_job_result,
                                                gbsub.sub_server_stats)]
    assert offs == [gbsub.sub_server_params.f_min.offset, gbsub.sub_job_result.stats.offset,
                    gbsub.sub_job_result.latency_ms.offset,
                    gbsub.sub_server_stats.inflight.offset]
