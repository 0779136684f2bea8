"""FP64 CPU oracle of the iterative galactic-binary subtraction (arXiv 2602.18560, App. D).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may load this package; the library never does.
It shares no code with the CUDA path.  The arithmetic lives in ``oracle.cpp``
(plain loops, FP64, one thread, compiled without fused multiply-add); this
module compiles it with g++ and exposes it through ctypes with numpy arrays.

Parity status per function (what pins it is in the test suite):
  tables, pieces, SNR, deposition, estimators, loop, coarse-graining: pinned
  (closed forms, quadrature of the waveform average, brute force, library special
  cases, invariants).  The paper's Table III counts are not reproducible here
  (parity unpinned for them: different catalog and waveform model).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

MEAN, MEDIAN, MEDIAN_MEAN = 0, 1, 2
YEAR = 365.25 * 86400.0


class Params(ctypes.Structure):
    _fields_ = [
        ("T_obs", ctypes.c_double),
        ("f_min", ctypes.c_double),
        ("f_max", ctypes.c_double),
        ("window", ctypes.c_int32),
        ("estimator", ctypes.c_int32),
        ("rho_th", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("tdi2", ctypes.c_int32),
        ("conv_rtol", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("n_candidates", ctypes.c_int64),
        ("n_resolved", ctypes.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.cpp into a shared library (g++, -O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            P = ctypes.c_void_p
            for name in ("orc_fstar", "orc_median_bias"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = []
            for name in ("orc_p_oms", "orc_p_tm"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d]
            for name in ("orc_s_instr", "orc_response"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, i32]
            L.orc_grid.restype = i32
            L.orc_grid.argtypes = [d, d, d, P, P]
            L.orc_tables.restype = None
            L.orc_tables.argtypes = [d, i64, i64, i32, P, P]
            L.orc_source_pieces.restype = i64
            L.orc_source_pieces.argtypes = [d, i64, i64, d, d, P, P, i64]
            L.orc_smooth.restype = None
            L.orc_smooth.argtypes = [i32, i64, P, i64, P]
            L.orc_smooth_at.restype = None
            L.orc_smooth_at.argtypes = [i32, i64, P, i64, P, i64, P]
            L.orc_deposit.restype = None
            L.orc_deposit.argtypes = [d, i64, i64, P, P, P, i64, P, P]
            L.orc_power.restype = None
            L.orc_power.argtypes = [d, P, P, i64, P]
            L.orc_snr2.restype = None
            L.orc_snr2.argtypes = [d, i64, i64, P, P, P, P, P, P, i64, P]
            L.orc_coarse_grain.restype = None
            L.orc_coarse_grain.argtypes = [d, d, d, i64, i64, P, i32, P, P, P]
            L.orc_run.restype = i32
            L.orc_run.argtypes = [ctypes.POINTER(Params), P, P, P, i64, P, P,
                                  ctypes.POINTER(Stats), P, i64]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def fstar() -> float:
    return lib().orc_fstar()


def median_bias() -> float:
    return lib().orc_median_bias()


def p_oms(f: float) -> float:
    return lib().orc_p_oms(f)


def p_tm(f: float) -> float:
    return lib().orc_p_tm(f)


def s_instr(f: float, tdi2: bool = True) -> float:
    return lib().orc_s_instr(f, int(tdi2))


def response(f: float, tdi2: bool = True) -> float:
    return lib().orc_response(f, int(tdi2))


def grid(T: float, f_min: float = 1e-4, f_max: float = 1e-2):
    k_lo = ctypes.c_int64()
    n = ctypes.c_int64()
    rc = lib().orc_grid(T, f_min, f_max, ctypes.byref(k_lo), ctypes.byref(n))
    if rc != 0:
        raise ValueError("empty or invalid grid")
    return k_lo.value, n.value


def tables(T: float, k_lo: int, n: int, tdi2: bool = True):
    S = np.empty(n)
    R = np.empty(n)
    lib().orc_tables(T, k_lo, n, int(tdi2), _p(S), _p(R))
    return S, R


def source_pieces(T, k_lo, n, f, fdot, cap=100000):
    j = np.empty(cap, dtype=np.int64)
    w = np.empty(cap)
    m = lib().orc_source_pieces(T, k_lo, n, f, fdot, _p(j), _p(w), cap)
    m = min(m, cap)
    return j[:m].copy(), w[:m].copy()


def smooth(est: int, W: int, P):
    P = _f64(P)
    out = np.empty_like(P)
    lib().orc_smooth(est, W, _p(P), P.size, _p(out))
    return out


def smooth_at(est: int, W: int, P, idx):
    P = _f64(P)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.size)
    lib().orc_smooth_at(est, W, _p(P), P.size, _p(idx), idx.size, _p(out))
    return out


def deposit(T, k_lo, n, A, f, fdot, exclude=None):
    A, f, fdot = _f64(A), _f64(f), _f64(fdot)
    ex = None if exclude is None else np.ascontiguousarray(exclude, dtype=np.uint8)
    D = np.empty(n)
    lib().orc_deposit(T, k_lo, n, _p(A), _p(f), _p(fdot), A.size, _p(ex), _p(D))
    return D


def power(T, R, D):
    R, D = _f64(R), _f64(D)
    P = np.empty_like(D)
    lib().orc_power(T, _p(R), _p(D), D.size, _p(P))
    return P


def coarse_grain(T, f_min, f_max, k_lo, x, nbins=100):
    """(S_k, f_k, N_k): bin averages of the per-bin series x over nbins log-spaced bins."""
    x = _f64(x)
    S = np.empty(nbins)
    fk = np.empty(nbins)
    c = np.empty(nbins, dtype=np.int64)
    lib().orc_coarse_grain(T, f_min, f_max, k_lo, x.size, _p(x), nbins, _p(S), _p(fk), _p(c))
    return S, fk, c


def snr2(T, k_lo, n, S_instr, R, S_gal, A, f, fdot):
    A, f, fdot = _f64(A), _f64(f), _f64(fdot)
    S_instr, R = _f64(S_instr), _f64(R)
    Sg = None if S_gal is None else _f64(S_gal)
    out = np.empty(A.size)
    lib().orc_snr2(T, k_lo, n, _p(S_instr), _p(R), _p(Sg), _p(A), _p(f), _p(fdot),
                   A.size, _p(out))
    return out


def make_params(T_obs=YEAR, f_min=1e-4, f_max=1e-2, window=1000, estimator=MEDIAN_MEAN,
                rho_th=7.0, kappa=None, max_iter=100, tdi2=True, conv_rtol=0.0) -> Params:
    if kappa is None:
        kappa = 1.0 / rho_th
    return Params(T_obs, f_min, f_max, window, estimator, rho_th, kappa, max_iter,
                  int(tdi2), conv_rtol)


def run(params: Params, A, f, fdot, trace_iters: int = 0):
    """Run the whole subtraction; returns dict with S_gal, resolved, stats (and trace)."""
    A, f, fdot = _f64(A), _f64(f), _f64(fdot)
    k_lo, n = grid(params.T_obs, params.f_min, params.f_max)
    Sg = np.empty(n)
    res = np.empty(A.size, dtype=np.uint8)
    st = Stats()
    trace = np.empty((trace_iters, n)) if trace_iters > 0 else None
    rc = lib().orc_run(ctypes.byref(params), _p(A), _p(f), _p(fdot), A.size, _p(Sg),
                       _p(res), ctypes.byref(st), _p(trace), trace_iters)
    if rc < 0:
        raise ValueError("invalid parameters")
    out = dict(S_gal=Sg, resolved=res.astype(bool), iterations=st.iterations,
               converged=bool(st.converged), n_candidates=st.n_candidates,
               n_resolved=st.n_resolved, k_lo=k_lo, n_bins=n)
    if trace is not None:
        out["trace"] = trace[: min(trace_iters, st.iterations)]
    return out
