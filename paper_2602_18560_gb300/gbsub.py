"""Python binding of libgbsub.so (C ABI declared in include/gbsub.h).

Argument marshalling only: every step of the subtraction runs in the library's
CUDA kernels.  Functions keep the C names (sub_create, sub_load_catalog, sub_run,
sub_get_spectrum, sub_get_resolved_mask, sub_destroy, ...); ``Subtraction`` wraps
a context for convenience.  Buffers are numpy arrays (host memory) or torch CUDA
tensors (device memory, passed by data_ptr()).  There is no fallback: if the
library is missing or a call fails, an exception is raised.

Typical use::

    from paper_2602_18560_gb300 import gbsub, synth
    with gbsub.Subtraction(T_obs=4 * synth.YEAR, window=1000,
                           estimator=gbsub.MEDIAN_MEAN) as s:
        s.load(A, f, fdot)                   # or s.load(..., mapped=True) for pinned
                                             # host arrays read in place, or
                                             # s.load_generated(n, seed, population)
        stats = s.run()                      # iterations, resolved count, ...
        S_gal = s.spectrum()                 # per bin, from k_lo / T_obs upwards
        resolved = s.resolved()              # one byte per source
        S_k, f_k, N_k = s.coarse_grain()     # 100 log-spaced bin averages

Many catalogs at once: ``Batch`` (one graph launch, ``autotune.tune_batch``);
a request loop: ``Server`` (submit/poll, memory budget, pooled contexts).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ETIMEOUT, EBUDGET, ERANGE, ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
MEAN, MEDIAN, MEDIAN_MEAN = 0, 1, 2
FP64, MIXED, FP64_STRICT = 0, 1, 2
HOST, DEVICE, HOST_MAPPED = 0, 1, 2
YEAR = 365.25 * 86400.0

_ERRNAMES = {OK: "SUB_OK", EINVAL: "SUB_EINVAL", ENOMEM: "SUB_ENOMEM", ECUDA: "SUB_ECUDA",
             ENOTCONVERGED: "SUB_ENOTCONVERGED", ETIMEOUT: "SUB_ETIMEOUT",
             EBUDGET: "SUB_EBUDGET", ERANGE: "SUB_ERANGE", ESTATE: "SUB_ESTATE"}


class SubError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, code), msg))
        self.code = code


class sub_params(ctypes.Structure):
    _fields_ = [
        ("T_obs", ctypes.c_double), ("f_min", ctypes.c_double), ("f_max", ctypes.c_double),
        ("window", ctypes.c_int32), ("estimator", ctypes.c_int32),
        ("rho_th", ctypes.c_double), ("kappa", ctypes.c_double),
        ("max_iter", ctypes.c_int32), ("tdi2", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("reserved0", ctypes.c_int32),
        ("conv_rtol", ctypes.c_double), ("hbm_budget", ctypes.c_uint64),
    ]


class sub_stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
        ("n_sources", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
        ("n_resolved", ctypes.c_int64), ("n_bins", ctypes.c_int64), ("k_lo", ctypes.c_int64),
        ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("n_live", ctypes.c_int64), ("n_exact", ctypes.c_int64),
        ("n_near", ctypes.c_int64), ("n_uncertain", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class sub_population(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("alpha_pl", "alpha_g", "beta_g", "mu_g", "mu", "sigma", "rho")]


def _population_struct(pop):
    return sub_population(*(float(getattr(pop, k)) for k, _ in sub_population._fields_))


class sub_server_params(ctypes.Structure):
    _fields_ = [
        ("hbm_budget", ctypes.c_uint64), ("max_inflight", ctypes.c_int32),
        ("window", ctypes.c_int32), ("estimator", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("tdi2", ctypes.c_int32),
        ("grid_div", ctypes.c_int32), ("max_contexts", ctypes.c_int32),
        ("f_min", ctypes.c_double), ("f_max", ctypes.c_double),
        ("rho_th", ctypes.c_double), ("kappa", ctypes.c_double),
    ]


class sub_job_result(ctypes.Structure):
    _fields_ = [
        ("job_id", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("stats", sub_stats), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
        ("gpu_ms", ctypes.c_double),
    ]


class sub_server_stats(ctypes.Structure):
    _fields_ = [
        ("queued", ctypes.c_int64), ("contexts_created", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64), ("peak_device_bytes", ctypes.c_int64),
        ("inflight", ctypes.c_int32), ("contexts", ctypes.c_int32),
    ]


_lib = None
_lock = threading.Lock()
EXPORTS = ("sub_params_default", "sub_create", "sub_load_catalog", "sub_load_generated",
           "sub_load_population", "sub_server_submit_population",
           "sub_get_catalog", "sub_run", "sub_get_stats",
           "sub_get_history", "sub_get_spectrum", "sub_get_resolved_mask", "sub_estimate",
           "sub_get_tables", "sub_get_timing", "sub_get_work", "sub_coarse_grain", "sub_profile",
           "sub_device_bytes", "sub_snr_check", "sub_get_profile_iterations",
           "sub_destroy",
           "sub_last_error", "sub_running_mean_noalloc", "sub_get_power", "sub_batch_create",
           "sub_batch_run", "sub_batch_last_ms", "sub_batch_last_error", "sub_batch_destroy",
           "sub_set_grid_div", "sub_set_tuning", "sub_test_hooks", "sub_server_params_default", "sub_server_create",
           "sub_server_submit", "sub_server_submit_generated", "sub_server_poll",
           "sub_server_info", "sub_server_last_error",
           "sub_server_prewarm",
           "sub_server_destroy")
KERNELS = ("prepass", "sort", "median", "prefix", "mean", "snr", "control")


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libgbsub.so (building it first if it is missing and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError("libgbsub.so is not built: run paper_2602_18560_gb300.build")
            _build.build()
        L = ctypes.CDLL(path)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        sig = {
            "sub_params_default": (i32, [ctypes.POINTER(sub_params)]),
            "sub_create": (i32, [ctypes.POINTER(sub_params), P, ctypes.POINTER(P)]),
            "sub_load_catalog": (i32, [P, P, P, P, i64, i32]),
            "sub_run": (i32, [P, ctypes.POINTER(sub_stats)]),
            "sub_get_stats": (i32, [P, ctypes.POINTER(sub_stats)]),
            "sub_get_history": (i32, [P, P, i32]),
            "sub_get_spectrum": (i32, [P, P, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), i32]),
            "sub_get_resolved_mask": (i32, [P, P, i64, i32]),
            "sub_estimate": (i32, [P, P, P, i64, i32]),
            "sub_get_tables": (i32, [P, P, P, i64, i32]),
            "sub_get_power": (i32, [P, P, i64, i32]),
            "sub_get_timing": (i32, [P, P, P, P]),
            "sub_get_work": (i32, [P, P, i32]),
            "sub_load_generated": (i32, [P, i64, ctypes.c_uint64, ctypes.c_double,
                                         ctypes.c_double, i32]),
            "sub_get_catalog": (i32, [P, P, P, P, i64, i64, i32]),
            "sub_load_population": (i32, [P, i64, ctypes.c_uint64, ctypes.POINTER(sub_population),
                                          i32]),
            "sub_server_submit_population": (i32, [P, i64, ctypes.c_double, i64, ctypes.c_uint64,
                                                   ctypes.POINTER(sub_population), P, i64, P]),
            "sub_coarse_grain": (i32, [P, P, i32, i32, P, P, P, i32]),
            "sub_profile": (i32, [P, P, P, ctypes.POINTER(sub_stats)]),
            "sub_device_bytes": (i64, [P]),
            "sub_snr_check": (i32, [P, P, P, P, P, i64, ctypes.POINTER(i64)]),
            "sub_get_profile_iterations": (i32, [P, P, i32]),
            "sub_destroy": (None, [P]),
            "sub_last_error": (ctypes.c_char_p, [P]),
            "sub_running_mean_noalloc": (i32, [P, P, i64, i32, P]),
            "sub_batch_create": (i32, [P, i32, ctypes.POINTER(P)]),
            "sub_batch_run": (i32, [P, P]),
            "sub_batch_last_ms": (ctypes.c_float, [P]),
            "sub_batch_last_error": (ctypes.c_char_p, [P]),
            "sub_batch_destroy": (None, [P]),
            "sub_set_grid_div": (i32, [P, i32]),
            "sub_set_tuning": (i32, [P, i32, i32]),
            "sub_test_hooks": (i32, [P, i32]),
            "sub_server_params_default": (i32, [ctypes.POINTER(sub_server_params)]),
            "sub_server_create": (i32, [ctypes.POINTER(sub_server_params), ctypes.POINTER(P)]),
            "sub_server_submit": (i32, [P, i64, ctypes.c_double, P, P, P, i64, P, i64, P]),
            "sub_server_submit_generated": (i32, [P, i64, ctypes.c_double, i64, ctypes.c_uint64,
                                                  ctypes.c_double, ctypes.c_double, P, i64, P]),
            "sub_server_poll": (i32, [P, ctypes.POINTER(sub_job_result), i32, i32]),
            "sub_server_info": (i32, [P, ctypes.POINTER(sub_server_stats)]),
            "sub_server_prewarm": (i32, [P, ctypes.c_double, i64, i32]),
            "sub_server_last_error": (ctypes.c_char_p, [P]),
            "sub_server_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib


# ------------------------------------------------------------------ marshalling

def _is_torch(x):
    return hasattr(x, "data_ptr") and hasattr(x, "is_cuda")


def _ptr(x, dtype):
    """(pointer, where, n) of a numpy array (host) or a torch CUDA tensor (device)."""
    if x is None:
        return None, HOST, 0
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError("tensor must be contiguous %s" % want)
        if x.is_cuda:
            # the library's stream waits for nothing torch queued: make it visible first
            torch.cuda.current_stream(x.device).synchronize()
            return ctypes.c_void_p(x.data_ptr()), DEVICE, x.numel()
        return ctypes.c_void_p(x.data_ptr()), HOST, x.numel()
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError("array must be contiguous %s" % np.dtype(dtype))
    return a.ctypes.data_as(ctypes.c_void_p), HOST, a.size


def _check(ctx, rc, allow=()):
    if rc < 0 and rc not in allow:
        raise SubError(rc, lib().sub_last_error(ctx).decode())
    return rc


def sub_params_default(**overrides) -> sub_params:
    p = sub_params()
    _check(None, lib().sub_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def sub_create(params: sub_params, stream=None):
    ctx = ctypes.c_void_p()
    st = ctypes.c_void_p(int(stream) if stream else 0)
    rc = lib().sub_create(ctypes.byref(params), st, ctypes.byref(ctx))
    if rc != OK:
        raise SubError(rc, lib().sub_last_error(None).decode())
    return ctx


def sub_load_catalog(ctx, A, f, fdot, mapped=False):
    """mapped: the arrays are page-locked host memory that every run reads in place
    (SUB_HOST_MAPPED); the caller keeps them alive and unchanged until the next load."""
    (pa, wa, na), (pf, wf, nf), (pd, wd, nd) = (_ptr(A, np.float64), _ptr(f, np.float64),
                                                _ptr(fdot, np.float64))
    if not (na == nf == nd) or not (wa == wf == wd):
        raise ValueError("A, f, fdot must have the same length and location")
    if mapped:
        if wa != HOST:
            raise ValueError("a mapped catalog lives in host memory")
        wa = HOST_MAPPED
    return _check(ctx, lib().sub_load_catalog(ctx, pa, pf, pd, na, wa))


def sub_load_generated(ctx, n, seed, gamma=11.0 / 3.0, shape=2.0, fused=True):
    """A catalog generated on the device (the single-precision recipe; synth.catalog_single
    is the same recipe on the host).  fused: every run generates the sources inside its
    catalog pass; otherwise they are generated once into device memory."""
    return _check(ctx, lib().sub_load_generated(ctx, int(n), int(seed) & (2**64 - 1),
                                                float(gamma), float(shape), int(bool(fused))))


def sub_load_population(ctx, n, seed, pop, fused=True):
    """A catalog of the paper's population model (synth.PaperPopulation fields) drawn on the
    device."""
    ps = _population_struct(pop)
    _check(ctx, lib().sub_load_population(ctx, int(n), int(seed) & (2**64 - 1),
                                          ctypes.byref(ps), int(bool(fused))))


def sub_get_catalog(ctx, start, n, device=False):
    """(A, f, fdot) of sources start .. start+n-1 of the current catalog."""
    if device:
        import torch
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3)]
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in outs]
        where = DEVICE
    else:
        outs = [np.empty(n) for _ in range(3)]
        ptrs = [t.ctypes.data_as(ctypes.c_void_p) for t in outs]
        where = HOST
    _check(ctx, lib().sub_get_catalog(ctx, *ptrs, int(start), int(n), where))
    return tuple(outs)


def sub_run(ctx, wait: bool = True):
    if not wait:
        _check(ctx, lib().sub_run(ctx, None))
        return None
    st = sub_stats()
    _check(ctx, lib().sub_run(ctx, ctypes.byref(st)), allow=(ENOTCONVERGED,))
    return st


def sub_get_stats(ctx):
    st = sub_stats()
    _check(ctx, lib().sub_get_stats(ctx, ctypes.byref(st)), allow=(ENOTCONVERGED,))
    return st


def sub_get_history(ctx, cap: int = 1024):
    h = np.zeros(cap, np.int32)
    m = _check(ctx, lib().sub_get_history(ctx, h.ctypes.data_as(ctypes.c_void_p), cap))
    return h[:m]


def n_bins_of(ctx):
    n = ctypes.c_int64()
    k = ctypes.c_int64()
    _check(ctx, lib().sub_get_spectrum(ctx, None, 0, ctypes.byref(n), ctypes.byref(k), HOST))
    return n.value, k.value


def sub_get_spectrum(ctx, out=None):
    nb, _ = n_bins_of(ctx)
    if out is None:
        out = np.empty(nb)
    p, w, n = _ptr(out, np.float64)
    _check(ctx, lib().sub_get_spectrum(ctx, p, n, None, None, w))
    return out


def sub_get_resolved_mask(ctx, n: int, out=None):
    if out is None:
        out = np.empty(n, np.uint8)
    p, w, m = _ptr(out, np.uint8)
    _check(ctx, lib().sub_get_resolved_mask(ctx, p, m, w))
    return out


def sub_estimate(ctx, P, out=None):
    if out is None:
        out = np.empty_like(P) if not _is_torch(P) else P.new_empty(P.shape)
    pi, wi, n = _ptr(P, np.float64)
    po, wo, m = _ptr(out, np.float64)
    if wi != wo or n != m:
        raise ValueError("P and out must have the same length and location")
    _check(ctx, lib().sub_estimate(ctx, pi, po, n, wi))
    return out


def sub_get_power(ctx, out=None):
    nb, _ = n_bins_of(ctx)
    if out is None:
        out = np.empty(nb)
    p, w, n = _ptr(out, np.float64)
    _check(ctx, lib().sub_get_power(ctx, p, n, w))
    return out


def sub_get_tables(ctx):
    nb, _ = n_bins_of(ctx)
    S = np.empty(nb)
    R = np.empty(nb)
    _check(ctx, lib().sub_get_tables(ctx, S.ctypes.data_as(ctypes.c_void_p),
                                     R.ctypes.data_as(ctypes.c_void_p), nb, HOST))
    return S, R


def sub_coarse_grain(ctx, x=None, nbins=100, add_instr=False):
    """(S_k, f_k, N_k): bin averages over nbins log-spaced bins of x (n_bins values, host or
    device), or of the last run's S_gal when x is None; of S_instr + x with add_instr."""
    where = HOST
    px = None
    if x is not None:
        px, where, n = _ptr(x, np.float64)
        nb, _ = n_bins_of(ctx)
        if n != nb:
            raise ValueError("x must hold n_bins (%d) values" % nb)
    if where == DEVICE:
        import torch
        dev = x.device
        S = torch.empty(nbins, dtype=torch.float64, device=dev)
        f = torch.empty(nbins, dtype=torch.float64, device=dev)
        c = torch.empty(nbins, dtype=torch.int64, device=dev)
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (S, f, c)]
    else:
        S, f, c = np.empty(nbins), np.empty(nbins), np.empty(nbins, dtype=np.int64)
        ptrs = [t.ctypes.data_as(ctypes.c_void_p) for t in (S, f, c)]
    _check(ctx, lib().sub_coarse_grain(ctx, px, int(bool(add_instr)), nbins, *ptrs, where))
    return S, f, c


def sub_get_work(ctx):
    """Work-list items the loop kernels of the last run were handed, by list: chunks whose
    values changed, chunks within one and within two of them, median tiles."""
    w = (ctypes.c_int64 * 4)()
    _check(ctx, lib().sub_get_work(ctx, w, 4))
    return {"changed": w[0], "within1": w[1], "within2": w[2], "tiles": w[3]}


def sub_get_timing(ctx):
    """(prepass_ms, loop_ms, total_ms) of the last run, from events inside its graph."""
    a, b, t = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(ctx, lib().sub_get_timing(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)))
    return a.value, b.value, t.value


def sub_profile(ctx):
    """Per-kernel device time (ms) and launch counts of one host-driven run."""
    ms = (ctypes.c_float * len(KERNELS))()
    n = (ctypes.c_int32 * len(KERNELS))()
    st = sub_stats()
    _check(ctx, lib().sub_profile(ctx, ms, n, ctypes.byref(st)), allow=(ENOTCONVERGED,))
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNELS)}, st


def sub_get_profile_iterations(ctx, cap=4096):
    """Per iteration of the last sub_profile: {kernel: ms}."""
    buf = (ctypes.c_float * (cap * len(KERNELS)))()
    m = _check(ctx, lib().sub_get_profile_iterations(ctx, buf, cap))
    return [{k: buf[i * len(KERNELS) + j] for j, k in enumerate(KERNELS)}
            for i in range(min(m, cap))]


def sub_device_bytes(ctx) -> int:
    return lib().sub_device_bytes(ctx)


def sub_snr_check(ctx):
    """rho^2 of every kept candidate against the last run's S_gal, two ways: the FP32 screen
    and FP64 in the oracle's order.  Returns dict of numpy arrays src, screen, exact, nbins."""
    n = ctypes.c_int64()
    _check(ctx, lib().sub_snr_check(ctx, None, None, None, None, 0, ctypes.byref(n)),
           allow=(EINVAL,))
    m = n.value
    src = np.empty(m, dtype=np.int64)
    sc = np.empty(m, dtype=np.float32)
    ex = np.empty(m, dtype=np.float64)
    nb = np.empty(m, dtype=np.int32)
    if m:
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in (src, sc, ex, nb)]
        _check(ctx, lib().sub_snr_check(ctx, *ptrs, m, ctypes.byref(n)))
    return {"src": src, "screen": sc, "exact": ex, "nbins": nb}


def sub_destroy(ctx):
    if ctx:
        lib().sub_destroy(ctx)


def _default_population():
    from . import synth
    return synth.Population()


class Subtraction:
    """One context: ``Subtraction(T_obs=..., window=..., estimator=...)``."""

    def __init__(self, params: sub_params | None = None, stream=None, **kw):
        self.params = params if params is not None else sub_params_default(**kw)
        self.ctx = sub_create(self.params, stream)
        self.n_sources = None

    def load(self, A, f, fdot, mapped=False):
        sub_load_catalog(self.ctx, A, f, fdot, mapped)
        self.n_sources = int(len(A))
        self._mapped = (A, f, fdot) if mapped else None  # kept alive while runs read them
        return self

    def load_generated(self, n, seed, pop=None, fused=True):
        pop = pop if pop is not None else _default_population()
        sub_load_generated(self.ctx, n, seed, pop.gamma, pop.shape, fused)
        self.n_sources = int(n)
        self._mapped = None
        return self

    def load_population(self, n, seed, pop, fused=True):
        sub_load_population(self.ctx, n, seed, pop, fused)
        self.n_sources = int(n)
        self._mapped = None
        return self

    def catalog(self, start=0, n=None, device=False):
        n = self.n_sources - start if n is None else n
        return sub_get_catalog(self.ctx, start, n, device)

    def run(self, wait=True):
        return sub_run(self.ctx, wait)

    def spectrum(self, out=None):
        return sub_get_spectrum(self.ctx, out)

    def resolved(self, out=None):
        return sub_get_resolved_mask(self.ctx, self.n_sources, out)

    def history(self):
        return sub_get_history(self.ctx)

    def estimate(self, P, out=None):
        return sub_estimate(self.ctx, P, out)

    def tables(self):
        return sub_get_tables(self.ctx)

    def power(self, out=None):
        return sub_get_power(self.ctx, out)

    def timing(self):
        return sub_get_timing(self.ctx)

    def work(self):
        return sub_get_work(self.ctx)

    def coarse_grain(self, x=None, nbins=100, add_instr=False):
        return sub_coarse_grain(self.ctx, x, nbins, add_instr)

    def snr_check(self):
        return sub_snr_check(self.ctx)

    def profile(self):
        return sub_profile(self.ctx)

    def profile_iterations(self):
        return sub_get_profile_iterations(self.ctx)

    @property
    def grid(self):
        return n_bins_of(self.ctx)

    def close(self):
        if self.ctx:
            sub_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches

def sub_set_grid_div(ctx, div: int):
    return _check(ctx, lib().sub_set_grid_div(ctx, int(div)))


TUNE_GRID_DIV, TUNE_SORT_E, TUNE_MEDIAN_THREADS = 0, 1, 2


def sub_set_tuning(ctx, knob: int, value: int):
    """A launch setting that leaves results unchanged (TUNE_*; value 0: automatic)."""
    return _check(ctx, lib().sub_set_tuning(ctx, int(knob), int(value)))


TEST_SKIP_CATALOG_COPIES = 1


def sub_test_hooks(ctx, flags: int):
    return _check(ctx, lib().sub_test_hooks(ctx, int(flags)))


class Batch:
    """Several ``Subtraction`` contexts run together in one graph launch
    (``sub_batch_*``).  The contexts must outlive the batch."""

    def __init__(self, subs):
        self.subs = list(subs)
        arr = (ctypes.c_void_p * len(self.subs))(*[s.ctx.value for s in self.subs])
        self._arr = arr
        b = ctypes.c_void_p()
        rc = lib().sub_batch_create(arr, len(self.subs), ctypes.byref(b))
        if rc != OK:
            raise SubError(rc, lib().sub_last_error(None).decode())
        self.b = b

    def run(self):
        """Run every catalog; returns the list of sub_stats."""
        st = (sub_stats * len(self.subs))()
        rc = lib().sub_batch_run(self.b, st)
        if rc < 0 and rc != ENOTCONVERGED:
            raise SubError(rc, lib().sub_batch_last_error(self.b).decode())
        return list(st)

    @property
    def last_ms(self):
        return float(lib().sub_batch_last_ms(self.b))

    def close(self):
        if self.b:
            lib().sub_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

def sub_server_params_default(**overrides) -> sub_server_params:
    p = sub_server_params()
    _check(None, lib().sub_server_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Server:
    """A request loop (``sub_server_*``): ``submit`` queues a job whose host buffers must stay
    alive until ``poll`` returns its result."""

    def __init__(self, params: sub_server_params | None = None, **kw):
        self.params = params if params is not None else sub_server_params_default(**kw)
        s = ctypes.c_void_p()
        rc = lib().sub_server_create(ctypes.byref(self.params), ctypes.byref(s))
        if rc != OK:
            raise SubError(rc, lib().sub_last_error(None).decode())
        self.s = s
        self._keep = {}

    def submit(self, job_id, T_obs, A, f, fdot, S_gal_out=None, mask_out=None):
        """Queue a job; A, f, fdot, S_gal_out, mask_out are host arrays (numpy, or pinned
        torch CPU tensors) kept referenced until the job comes back."""
        (pa, wa, na), (pf, _, nf), (pd, _, nd) = (_ptr(A, np.float64), _ptr(f, np.float64),
                                                  _ptr(fdot, np.float64))
        if not (na == nf == nd) or wa != HOST:
            raise ValueError("A, f, fdot must be host arrays of one length")
        ps, ws_, ncap = _ptr(S_gal_out, np.float64)
        pm, wm, nm = _ptr(mask_out, np.uint8)
        if (S_gal_out is not None and ws_ != HOST) or (mask_out is not None and wm != HOST):
            raise ValueError("result buffers must be host memory")
        if mask_out is not None and nm < na:
            raise ValueError("mask buffer smaller than the catalog")
        rc = lib().sub_server_submit(self.s, int(job_id), float(T_obs), pa, pf, pd, na, ps,
                                     ncap, pm)
        if rc != OK:
            raise SubError(rc, lib().sub_server_last_error(self.s).decode())
        self._keep[int(job_id)] = (A, f, fdot, S_gal_out, mask_out)

    def submit_generated(self, job_id, T_obs, n, seed, pop=None, S_gal_out=None,
                         mask_out=None):
        """Queue a job whose catalog (n sources of population pop, this seed) is drawn on
        the device; the result buffers are host arrays kept referenced until it returns."""
        pop = pop if pop is not None else _default_population()
        ps, ws_, ncap = _ptr(S_gal_out, np.float64)
        pm, wm, nm = _ptr(mask_out, np.uint8)
        if (S_gal_out is not None and ws_ != HOST) or (mask_out is not None and wm != HOST):
            raise ValueError("result buffers must be host memory")
        if mask_out is not None and nm < n:
            raise ValueError("mask buffer smaller than the catalog")
        rc = lib().sub_server_submit_generated(self.s, int(job_id), float(T_obs), int(n),
                                               int(seed) & (2**64 - 1), float(pop.gamma),
                                               float(pop.shape), ps, ncap, pm)
        if rc != OK:
            raise SubError(rc, lib().sub_server_last_error(self.s).decode())
        self._keep[int(job_id)] = (S_gal_out, mask_out)

    def submit_population(self, job_id, T_obs, n, seed, pop, S_gal_out=None, mask_out=None):
        """Queue a job whose catalog is drawn on the device from the paper's population model
        (synth.PaperPopulation); result buffers as submit_generated."""
        ps, ws_, ncap = _ptr(S_gal_out, np.float64)
        pm, wm, nm = _ptr(mask_out, np.uint8)
        if (S_gal_out is not None and ws_ != HOST) or (mask_out is not None and wm != HOST):
            raise ValueError("result buffers must be host memory")
        if mask_out is not None and nm < n:
            raise ValueError("mask buffer smaller than the catalog")
        pst = _population_struct(pop)
        rc = lib().sub_server_submit_population(self.s, int(job_id), float(T_obs), int(n),
                                                int(seed) & (2**64 - 1), ctypes.byref(pst),
                                                ps, ncap, pm)
        if rc != OK:
            raise SubError(rc, lib().sub_server_last_error(self.s).decode())
        self._keep[int(job_id)] = (S_gal_out, mask_out)

    def poll(self, timeout_ms=0, cap=256):
        """Finished jobs: a list of dicts (job_id, status, stats, latency_ms, queue_ms,
        gpu_ms)."""
        buf = (sub_job_result * cap)()
        k = lib().sub_server_poll(self.s, buf, cap, int(timeout_ms))
        out = []
        for i in range(k):
            r = buf[i]
            self._keep.pop(int(r.job_id), None)
            out.append({"job_id": int(r.job_id), "status": int(r.status),
                        "stats": r.stats.as_dict(), "latency_ms": r.latency_ms,
                        "queue_ms": r.queue_ms, "gpu_ms": r.gpu_ms})
        return out

    def prewarm(self, T_obs, n_sources, count):
        """Idle contexts for T_obs with room for n_sources, created before traffic arrives."""
        rc = lib().sub_server_prewarm(self.s, float(T_obs), int(n_sources), int(count))
        if rc != OK:
            raise SubError(rc, lib().sub_server_last_error(self.s).decode())

    def info(self):
        st = sub_server_stats()
        lib().sub_server_info(self.s, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if self.s:
            lib().sub_server_destroy(self.s)
            self.s = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
