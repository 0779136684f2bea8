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
    assert ctypes.sizeof(gbsub.sub_stats) == 72


def test_invalid_parameters_rejected_before_any_device_call():
    # validation happens before the first CUDA call, so this runs without a GPU
    for bad in (dict(window=0), dict(window=100000), dict(T_obs=-1.0), dict(f_min=0.0),
                dict(f_max=1e-5), dict(estimator=7), dict(max_iter=0), dict(rho_th=0.0),
                dict(kappa=-1.0), dict(precision=5)):
        with pytest.raises(gbsub.SubError) as ei:
            gbsub.sub_create(gbsub.sub_params_default(**bad))
        assert ei.value.code == gbsub.EINVAL
