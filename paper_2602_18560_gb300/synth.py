"""Seeded synthetic galactic-binary catalogs (inputs only; none of the subtraction's arithmetic).

Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
written from its published definition.  Every number a catalog needs is a pure
function of (seed, source index, stream), so any slice of a catalog can be
regenerated independently.  The same catalog is produced bit for bit on any
machine: the elementary functions used below (log, exp, pow) are written here
with IEEE basic operations only (+, -, *, /, sqrt, exact scalings), so they do not
depend on the platform's math library, and normal deviates come from Marsaglia's
polar method (no trigonometric function).

Distributions (the synthetic stand-in for the paper's population catalogs):
  f     : truncated power law p(f) ~ f^-gamma on [1e-4, 1e-2] Hz, by inverse CDF
  A     : 1e-23 X (f / 1e-3 Hz)^(2/3), X ~ Gamma(shape k, scale 1) (Marsaglia-Tsang)
  fdot  : (96/5) pi^(8/3) (G Mc / c^3)^(5/3) f^(11/3), Mc ~ U(0.2, 0.8) Msun
          (the GW-driven chirp of Sec. II.A)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

YEAR = 365.25 * 86400.0
GMSUN_C3 = 4.925490947e-6  # G Msun / c^3 in seconds
F_MIN, F_MAX = 1e-4, 1e-2

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds over arrays of 32-bit counters; returns 4 uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 &= 0xFFFFFFFF
    k1 &= 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32),
            c3.astype(np.uint32))


def u53(a, b):
    """Uniform double in (0, 1) from two 32-bit words (53 random bits, centred)."""
    a = np.asarray(a, dtype=np.uint64) >> np.uint64(5)
    b = np.asarray(b, dtype=np.uint64) >> np.uint64(6)
    return ((a * np.uint64(67108864) + b).astype(np.float64) + 0.5) / 9007199254740992.0


def u32(a):
    """Uniform double in (0, 1) from one 32-bit word."""
    return (np.asarray(a, dtype=np.float64) + 0.5) / 4294967296.0


# Stream identifiers (third counter word).
_STREAM_FM = 0          # f and chirp mass
_STREAM_GAMMA = 1       # Gamma attempts use streams 1..16
_MAX_GAMMA_TRIES = 24
_STREAM_POP = 0xFFFFFFF0  # per-catalog population parameters


# ------------------------------------------------------------------ portable elementary functions
# Natural log: x = m 2^e with m in [sqrt(1/2), sqrt(2)), log m = 2 atanh((m-1)/(m+1)) by its
# series; exp: x = k ln2 + r with |r| <= ln2/2, exp r by its Taylor series, then scaled by 2^k.
# ln 2 is split in a part with a short mantissa (exact products with k) and a correction.
_LN2_HI = 6.93147180369123816490e-01
_LN2_LO = 1.90821492927058770002e-10
_SQRT_HALF = 0.70710678118654752440


def plog(x):
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    small = m < _SQRT_HALF
    m = np.where(small, m * 2.0, m)
    e = (e - small.astype(np.int64)).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    acc = np.full(t.shape, 1.0 / 27.0)
    for k in range(25, 0, -2):
        acc = acc * t2 + 1.0 / k
    return e * _LN2_HI + (e * _LN2_LO + 2.0 * t * acc)


def pexp(x):
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x / (_LN2_HI + _LN2_LO))
    r = (x - k * _LN2_HI) - k * _LN2_LO
    acc = np.full(r.shape, 1.0 / math.factorial(18))
    for i in range(17, -1, -1):
        acc = acc * r + 1.0 / math.factorial(i)
    return np.ldexp(acc, k.astype(np.int64))


_LOG_1E3 = float(plog(1e-3))


def ppow(x, y):
    """x^y for x > 0 (y scalar or array)."""
    return pexp(np.asarray(y, dtype=np.float64) * plog(x))


def _power_law_icdf(u, gamma, fmin=F_MIN, fmax=F_MAX):
    if abs(gamma - 1.0) < 1e-12:
        return fmin * pexp(u * float(plog(fmax / fmin)))
    e = 1.0 - gamma
    a, b = float(ppow(fmin, e)), float(ppow(fmax, e))
    return ppow(a + u * (b - a), 1.0 / e)


def _gamma(k: float, idx: np.ndarray, k0: int, k1: int):
    """Gamma(k, 1), k >= 1, by Marsaglia-Tsang with counter-based attempts; the normal
    deviate of each attempt comes from Marsaglia's polar method."""
    if k < 1.0:
        raise ValueError("shape must be >= 1")
    d = k - 1.0 / 3.0
    c = 1.0 / math.sqrt(9.0 * d)
    out = np.full(idx.shape, d, dtype=np.float64)
    todo = np.arange(idx.size)
    lo = (idx & 0xFFFFFFFF).astype(np.uint64)
    hi = (idx >> 32).astype(np.uint64)
    for t in range(_MAX_GAMMA_TRIES):
        if todo.size == 0:
            break
        x0, x1, x2, x3 = philox4x32_10(lo[todo], hi[todo], _STREAM_GAMMA + t, 0, k0, k1)
        p = 2.0 * u32(x0) - 1.0
        q = 2.0 * u32(x1) - 1.0
        s2 = p * p + q * q
        inside = (s2 < 1.0) & (s2 > 0.0)
        s2 = np.where(inside, s2, 0.5)
        z = p * np.sqrt(-2.0 * plog(s2) / s2)
        v = 1.0 + c * z
        ok = inside & (v > 0.0)
        v = np.where(ok, v * v * v, 1.0)
        ua = u53(x2, x3)
        acc = ok & (plog(ua) < 0.5 * z * z + d - d * v + d * plog(v))
        out[todo[acc]] = d * v[acc]
        todo = todo[~acc]
    return out


@dataclass
class Population:
    gamma: float = 11.0 / 3.0    # power-law index of p(f) ~ f^-gamma
    shape: float = 2.0           # Gamma shape of the amplitude factor X


def catalog(n: int, seed: int, pop: Population | None = None, start: int = 0,
            chunk: int = 1 << 22):
    """Sources start .. start+n-1 of the catalog with this seed: returns (A, f, fdot) FP64."""
    pop = pop or Population()
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    A = np.empty(n)
    f = np.empty(n)
    fdot = np.empty(n)
    pref = 96.0 / 5.0 * float(ppow(math.pi, 8.0 / 3.0))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(start + s, start + e, dtype=np.int64)
        lo = (idx & 0xFFFFFFFF).astype(np.uint64)
        hi = (idx >> 32).astype(np.uint64)
        x0, x1, x2, x3 = philox4x32_10(lo, hi, _STREAM_FM, 0, k0, k1)
        fs = _power_law_icdf(u53(x0, x1), pop.gamma)
        mc = (0.2 + 0.6 * u53(x2, x3)) * GMSUN_C3
        X = _gamma(pop.shape, idx, k0, k1)
        lf = plog(fs)
        f[s:e] = fs
        fdot[s:e] = pref * pexp(5.0 / 3.0 * plog(mc) + 11.0 / 3.0 * lf)
        A[s:e] = 1e-23 * X * pexp(2.0 / 3.0 * (lf - _LOG_1E3))
    return A, f, fdot


# ------------------------------------------------------------------ single-precision recipe
# The catalog recipe of the device generator: the same counters and distributions as
# catalog(), evaluated in IEEE single precision with basic operations only (no fused
# multiply-add), so that numpy float32 here and the GPU produce the same bits.  Values are
# returned as FP64 (exact conversions).  log: the atanh series up to t^13; exp: Taylor to r^8.
_F = np.float32
_LN2_HI32 = _F(0.693145751953125)        # 16 significant bits: exact products with |k| < 256
_LN2_LO32 = _F(1.4286067653301870e-06)
_LN2_32 = _F(0.6931471805599453)
_SQRT_HALF32 = _F(0.7071067811865476)
_TINY32 = _F(1.1754943508222875e-38)      # smallest normal float
_LOG_C32 = [_F(1.0 / k) for k in (13, 11, 9, 7, 5, 3, 1)]
_EXP_C32 = [_F(1.0 / math.factorial(i)) for i in range(8, -1, -1)]


def plog32(x):
    x = np.maximum(np.asarray(x, dtype=np.float32), _TINY32)
    m, e = np.frexp(x)
    small = m < _SQRT_HALF32
    m = np.where(small, m * _F(2.0), m).astype(np.float32)
    e = (e - small.astype(e.dtype)).astype(np.float32)
    t = (m - _F(1.0)) / (m + _F(1.0))
    t2 = t * t
    acc = np.full(t.shape, _LOG_C32[0], dtype=np.float32)
    for c in _LOG_C32[1:]:
        acc = acc * t2 + c
    return e * _LN2_HI32 + (e * _LN2_LO32 + _F(2.0) * t * acc)


def pexp32(x):
    x = np.asarray(x, dtype=np.float32)
    k = np.rint(x / _LN2_32)
    r = (x - k * _LN2_HI32) - k * _LN2_LO32
    acc = np.full(r.shape, _EXP_C32[0], dtype=np.float32)
    for c in _EXP_C32[1:]:
        acc = acc * r + c
    return np.ldexp(acc, k.astype(np.int32)).astype(np.float32)


def u32f(a):
    """Uniform float in (0, 1) from one 32-bit word (single precision)."""
    return (np.asarray(a, dtype=np.uint32).astype(np.float32) + _F(0.5)) / _F(4294967296.0)


def single_constants(pop: Population):
    """Per-population constants of the single-precision recipe (all in float32).  The
    inverse CDF is f = f0 (rho + u (1 - rho))^(1/e), e = 1 - gamma, with f0 the end where
    the density is highest and rho = (f1/f0)^e < 1: the sparse tail comes from small u,
    where the uniform keeps its full relative precision, and nothing cancels.  Within 1e-3
    of gamma = 1 the density is taken as log-uniform."""
    e = _F(1.0 - pop.gamma)
    lmin, lmax = plog32(_F(F_MIN)), plog32(_F(F_MAX))
    power = abs(pop.gamma - 1.0) >= 1e-3
    lf0, lf1 = (lmin, lmax) if e < 0 else (lmax, lmin)
    rho = pexp32(e * (lf1 - lf0)) if power else _F(0.0)
    omr = _F(1.0) - rho
    inv_e = _F(1.0) / e if power else _F(0.0)
    span = lmax - lmin  # log-uniform case
    d = _F(pop.shape) - _F(1.0 / 3.0)
    c = _F(1.0) / np.sqrt(_F(9.0) * d)
    pref = _F(19.2) * pexp32(_F(8.0 / 3.0) * plog32(_F(math.pi)))
    return dict(power=power, lf0=_F(lf0), rho=_F(rho), omr=_F(omr), inv_e=_F(inv_e),
                lmin=_F(lmin), span=_F(span),
                d=_F(d), c=_F(c), pref=_F(pref), log1e3=_F(plog32(_F(1e-3))))


def _gamma32(d, c, lo, hi, k0, k1):
    """Gamma(d + 1/3, 1) in single precision (Marsaglia-Tsang with constants d, c), a
    polar-method normal per counter-based attempt; d itself when every attempt is refused."""
    X = np.full(lo.shape, d, dtype=np.float32)
    todo = np.arange(lo.size)
    for t in range(_MAX_GAMMA_TRIES):
        if todo.size == 0:
            break
        y0, y1, y2, y3 = philox4x32_10(lo[todo], hi[todo], _STREAM_GAMMA + t, 0, k0, k1)
        p = _F(2.0) * u32f(y0) - _F(1.0)
        q = _F(2.0) * u32f(y1) - _F(1.0)
        s2 = p * p + q * q
        inside = (s2 < _F(1.0)) & (s2 > _F(0.0))
        s2 = np.where(inside, s2, _F(0.5)).astype(np.float32)
        z = p * np.sqrt(_F(-2.0) * plog32(s2) / s2)
        v = _F(1.0) + c * z
        ok = inside & (v > _F(0.0))
        v = np.where(ok, v * v * v, _F(1.0)).astype(np.float32)
        ua = u32f(y2)
        acc = ok & (plog32(ua) < _F(0.5) * z * z + d - d * v + d * plog32(v))
        X[todo[acc]] = (d * v)[acc]
        todo = todo[~acc]
    return X


def catalog_single(n: int, seed: int, pop: Population | None = None, start: int = 0,
                   chunk: int = 1 << 22):
    """Sources start .. start+n-1 of the single-precision recipe with this seed, as FP64
    (A, f, fdot): the catalog the device generator produces."""
    pop = pop or Population()
    if pop.shape < 1.0:
        raise ValueError("shape must be >= 1")
    k = single_constants(pop)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    A = np.empty(n)
    f = np.empty(n)
    fdot = np.empty(n)
    gm = _F(GMSUN_C3)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(start + s, start + e, dtype=np.int64)
        lo = (idx & 0xFFFFFFFF).astype(np.uint64)
        hi = (idx >> 32).astype(np.uint64)
        x0, x1, x2, x3 = philox4x32_10(lo, hi, _STREAM_FM, 0, k0, k1)
        u = u32f(x0)
        # log f is the exponent that f comes from (no second logarithm)
        if k["power"]:
            lf = k["lf0"] + k["inv_e"] * plog32(k["rho"] + u * k["omr"])
        else:
            lf = k["lmin"] + u * k["span"]
        fs = pexp32(lf)
        mc = (_F(0.2) + _F(0.6) * u32f(x2)) * gm
        X = _gamma32(k["d"], k["c"], lo, hi, k0, k1)
        f[s:e] = fs
        fdot[s:e] = k["pref"] * pexp32(_F(5.0 / 3.0) * plog32(mc) + _F(11.0 / 3.0) * lf)
        A[s:e] = (_F(1e-23) * X) * pexp32(_F(2.0 / 3.0) * (lf - k["log1e3"]))
    return A, f, fdot


# ------------------------------------------------------------------ the paper's population model
# Sec. II.B "Population model" and Table I: f from a power law p(f) ~ f^alpha_pl on
# [0.1, 10] mHz; the rescaled log frequency derivative xi = log10(fdot) - mu_g ~ Gamma with
# concentration alpha_g and rate beta_g; the rescaled log amplitude
# log10(f^(-2/3) A) - mu ~ log-normal of width sigma; f and xi tied by a Gaussian copula of
# correlation rho (App. A).  The copula is sampled by conditioning, which gives the joint
# distribution of App. A's four steps: xi from its marginal, z2 = Phi^-1(F_Gamma(xi)), then
# z1 = rho z2 + sqrt(1 - rho^2) n with an independent normal n, and f = F_f^-1(Phi(z1)) (the
# tail probability Phi(-z1) enters the inverse CDF, so the sparse high-frequency end keeps
# its precision).  Single precision with basic operations only, as the device generator;
# special functions from published methods: the inverse normal CDF by Wichura's AS241 in
# its single-precision form PPND7 (Applied Statistics 37, 1988), erfc by the Chebyshev fit of Numerical Recipes (Press et al., 2nd ed., Sec. 6.2), the
# regularized incomplete gamma function by its series and its continued fraction (modified
# Lentz), log Gamma by the Lanczos form with g = 5 (Sec. 6.1 there).

# Table I prior ranges of the population parameters (and N_b).
PAPER_PRIOR = {"alpha_pl": (-4.0, -2.0), "alpha_g": (1.0, 3.0), "beta_g": (1.0, 3.0),
               "mu_g": (-22.0, -20.0), "mu": (-23.0, -21.0), "sigma": (0.1, 0.3),
               "rho": (0.0, 1.0), "n_b": (5e6, 3e7)}

_STREAM_PAPER = 32  # the copula's and the amplitude's uniforms
_LN10_32 = _F(2.302585092994046)
# AS241 (Wichura 1988, Applied Statistics 37, 477), the single-precision version PPND7
_PP_A = [_F(x) for x in (59.109374720, 159.29113202, 50.434271938, 3.3871327179)]
_PP_B = [_F(x) for x in (67.187563600, 78.757757664, 17.895169469)]
_PP_C = [_F(x) for x in (0.17023821103, 1.3067284816, 2.7568153900, 1.4234372777)]
_PP_D = [_F(x) for x in (0.12021132975, 0.73700164250)]
_PP_E = [_F(x) for x in (0.017337203997, 0.42868294337, 3.0812263860, 6.6579051150)]
_PP_F = [_F(x) for x in (0.012258202635, 0.24197894225)]
_ERFC_C = [_F(x) for x in (0.17087277, -0.82215223, 1.48851587, -1.13520398, 0.27886807,
                           -0.18628806, 0.09678418, 0.37409196, 1.00002368, -1.26551223)]
_LANCZOS = [_F(x) for x in (76.18009172947146, -86.50532032941677, 24.01409824083091,
                            -1.231739572450155, 0.1208650973866179e-2, -0.5395239384953e-5)]
_GAMMA_ITERS = 64
_EPS32 = _F(5.9604644775390625e-08)     # 2^-24
_FPMIN32 = _F(1e-30)


def _horner32(x, coefs, one_last=False):
    acc = np.full(x.shape, coefs[0], dtype=np.float32)
    for c in coefs[1:]:
        acc = acc * x + c
    if one_last:
        acc = acc * x + _F(1.0)
    return acc


def u23f(a):
    """Uniform float in [2^-24, 1 - 2^-24] from the top 23 bits of a 32-bit word: never 0 or 1
    (normal deviates from it stay within 5.3 standard deviations)."""
    return ((np.asarray(a, dtype=np.uint32) >> np.uint32(9)).astype(np.float32) + _F(0.5)) * \
        _F(1.0 / 8388608.0)


def norm_ppf_lower32(t):
    """Phi^-1(t) for 0 < t <= 1/2 (AS241 PPND7), single precision."""
    t = np.asarray(t, dtype=np.float32)
    q = t - _F(0.5)
    central = np.abs(q) <= _F(0.425)
    r = _F(0.180625) - q * q
    x_c = q * _horner32(r, _PP_A) / _horner32(r, _PP_B, True)
    rt = np.sqrt(_F(0.0) - plog32(np.where(central, _F(0.5), t)))
    near = rt <= _F(5.0)
    r1 = rt - _F(1.6)
    r2 = rt - _F(5.0)
    v = np.where(near, _horner32(r1, _PP_C) / _horner32(r1, _PP_D, True),
                 _horner32(r2, _PP_E) / _horner32(r2, _PP_F, True))
    return np.where(central, x_c, _F(0.0) - v).astype(np.float32)


def norm_ppf32(u):
    """Phi^-1(u) for 0 < u < 1: the lower half directly, the upper one by symmetry (1 - u is
    exact in single precision for u >= 1/2)."""
    u = np.asarray(u, dtype=np.float32)
    low = u <= _F(0.5)
    return np.where(low, norm_ppf_lower32(np.where(low, u, _F(0.5))),
                    -norm_ppf_lower32(np.where(low, _F(0.5), _F(1.0) - u))).astype(np.float32)


def erfc32(x):
    """erfc(x) for x >= 0 (fractional error below 1.2e-7), single precision."""
    x = np.asarray(x, dtype=np.float32)
    t = _F(1.0) / (_F(1.0) + _F(0.5) * x)
    acc = np.full(x.shape, _ERFC_C[0], dtype=np.float32)
    for c in _ERFC_C[1:]:
        acc = acc * t + c
    arg = np.maximum(_F(0.0) - x * x + acc, _F(-87.0))
    return t * pexp32(arg)


def norm_sf32(z):
    """Phi(-z) = 1 - Phi(z), the upper tail probability, single precision."""
    z = np.asarray(z, dtype=np.float32)
    pos = z >= _F(0.0)
    e = _F(0.5) * erfc32(np.abs(z) * _F(0.7071067811865476))
    return np.where(pos, e, _F(1.0) - e).astype(np.float32)


def lgamma32(a):
    """log Gamma(a) for a > 0 (Lanczos, g = 5, six terms), single precision."""
    x = _F(a)
    y = x
    tmp = x + _F(5.5)
    tmp = tmp - (x + _F(0.5)) * plog32(tmp)
    ser = _F(1.000000000190015)
    for c in _LANCZOS:
        y = y + _F(1.0)
        ser = ser + c / y
    return _F(-tmp + plog32(_F(2.5066282746310005) * ser / x))


def gamma_pq32(a, x, gln):
    """(P, Q) = regularized lower and upper incomplete gamma functions of shape a at x >= 0,
    single precision: the series for x < a + 1 (then Q = 1 - P), the continued fraction
    for Q otherwise (then P = 1 - Q); at most 64 terms.  gln = lgamma32(a)."""
    a = _F(a)
    x = np.asarray(x, dtype=np.float32)
    xs = np.maximum(x, _F(1e-30))
    pref_arg = np.maximum((_F(0.0) - x + a * plog32(xs)) - _F(gln), _F(-87.0))
    pref = pexp32(pref_arg)
    use_ser = x < a + _F(1.0)
    # series: sum_n x^n / (a (a+1) ... (a+n))
    ap = np.full(x.shape, a, dtype=np.float32)
    ssum = np.full(x.shape, _F(1.0) / a, dtype=np.float32)
    dl = ssum.copy()
    act = use_ser.copy()
    for _ in range(_GAMMA_ITERS):
        if not act.any():
            break
        ap_n = ap + _F(1.0)
        dl_n = dl * x / ap_n
        s_n = ssum + dl_n
        ap = np.where(act, ap_n, ap)
        dl = np.where(act, dl_n, dl)
        ssum = np.where(act, s_n, ssum)
        act = act & ~(np.abs(dl_n) < np.abs(s_n) * _EPS32)
    P_ser = ssum * pref
    # continued fraction for Q (modified Lentz)
    b = x + _F(1.0) - a
    c = np.full(x.shape, _F(1.0) / _FPMIN32, dtype=np.float32)
    d = _F(1.0) / np.where(use_ser, _F(1.0), b)
    h = d.copy()
    act = ~use_ser
    for i in range(1, _GAMMA_ITERS + 1):
        if not act.any():
            break
        an = _F(-i) * (_F(i) - a)
        b_n = b + _F(2.0)
        d_n = an * d + b_n
        d_n = np.where(np.abs(d_n) < _FPMIN32, _FPMIN32, d_n)
        c_n = b_n + an / c
        c_n = np.where(np.abs(c_n) < _FPMIN32, _FPMIN32, c_n)
        d_n = _F(1.0) / d_n
        de = d_n * c_n
        h_n = h * de
        b = np.where(act, b_n, b)
        d = np.where(act, d_n, d)
        c = np.where(act, c_n, c)
        h = np.where(act, h_n, h)
        act = act & ~(np.abs(de - _F(1.0)) < _EPS32)
    Q_cf = pref * h
    P = np.where(use_ser, P_ser, _F(1.0) - Q_cf).astype(np.float32)
    Q = np.where(use_ser, _F(1.0) - P_ser, Q_cf).astype(np.float32)
    return P, Q


@dataclass
class PaperPopulation:
    """Population parameters Lambda of the paper (Table I), N_b aside."""
    alpha_pl: float = -2.9    # p(f) ~ f^alpha_pl
    alpha_g: float = 1.96     # Gamma concentration of xi = log10 fdot - mu_g
    beta_g: float = 1.8       # Gamma rate
    mu_g: float = -21.0
    mu: float = -22.0         # log10(f^(-2/3) A) - mu ~ log-normal(sigma)
    sigma: float = 0.18
    rho: float = 0.99         # copula correlation of f and xi


def paper_constants(pop: PaperPopulation):
    """Per-population constants of the paper recipe (float32, as the device computes them)."""
    k = single_constants(Population(gamma=-pop.alpha_pl, shape=pop.alpha_g))
    rho = _F(pop.rho)
    k.update(beta=_F(pop.beta_g), alpha=_F(pop.alpha_g), gln=lgamma32(pop.alpha_g),
             mu_g=_F(pop.mu_g), mu=_F(pop.mu), sigma=_F(pop.sigma), rho=rho,
             rho_c=np.sqrt(_F(1.0) - rho * rho))
    return k


def catalog_paper(n: int, seed: int, pop: PaperPopulation | None = None, start: int = 0,
                  chunk: int = 1 << 21, with_latent: bool = False):
    """Sources start .. start+n-1 of the paper's population model with this seed, in single
    precision, as FP64 (A, f, fdot): the catalog the device generator produces.  With
    with_latent, also (xi, log-normal amplitude factor, z1, z2) for tests."""
    pop = pop or PaperPopulation()
    if pop.alpha_g < 1.0:
        raise ValueError("alpha_g must be >= 1")
    k = paper_constants(pop)
    kp = single_constants(Population(gamma=-pop.alpha_pl))
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    A, f, fdot = np.empty(n), np.empty(n), np.empty(n)
    lat = [np.empty(n, dtype=np.float32) for _ in range(4)] if with_latent else None
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(start + s, start + e, dtype=np.int64)
        lo = (idx & 0xFFFFFFFF).astype(np.uint64)
        hi = (idx >> 32).astype(np.uint64)
        # xi = G / beta, G ~ Gamma(alpha_g, 1); its CDF value as a standard normal z2
        G = _gamma32(k["d"], k["c"], lo, hi, k0, k1)
        xi = G / k["beta"]
        P, Q = gamma_pq32(k["alpha"], G, k["gln"])
        low = P <= _F(0.5)
        z2 = np.where(low, norm_ppf_lower32(np.where(low, P, _F(0.5))),
                      -norm_ppf_lower32(np.where(low, _F(0.5), Q))).astype(np.float32)
        x0, x1, x2, x3 = philox4x32_10(lo, hi, _STREAM_PAPER, 0, k0, k1)
        z1 = k["rho"] * z2 + k["rho_c"] * norm_ppf32(u23f(x0))
        # f from the tail probability of z1 (small: the sparse high-frequency end)
        ut = norm_sf32(z1)
        if kp["power"]:
            lf = kp["lf0"] + kp["inv_e"] * plog32(kp["rho"] + ut * kp["omr"])
        else:
            lf = kp["lmin"] + (_F(1.0) - ut) * kp["span"]
        fs = pexp32(lf)
        fd = pexp32(_LN10_32 * (k["mu_g"] + xi))
        am = pexp32(k["sigma"] * norm_ppf32(u23f(x1)))
        a = pexp32(_F(2.0 / 3.0) * lf + _LN10_32 * (k["mu"] + am))
        A[s:e], f[s:e], fdot[s:e] = a, fs, fd
        if with_latent:
            for arr, v in zip(lat, (xi, am, z1, z2)):
                arr[s:e] = v
    if with_latent:
        return A, f, fdot, lat
    return A, f, fdot


def paper_population_draw(seed: int, index: int):
    """Lambda and N_b from the Table I priors (independent uniforms), for draw `index`."""
    x0, x1, x2, x3 = philox4x32_10(index & 0xFFFFFFFF, index >> 32, _STREAM_POP + 2, 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    y0, y1, y2, y3 = philox4x32_10(index & 0xFFFFFFFF, index >> 32, _STREAM_POP + 3, 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    us = [float(u32(w)) for w in (x0, x1, x2, x3, y0, y1, y2, y3)]
    names = ("alpha_pl", "alpha_g", "beta_g", "mu_g", "mu", "sigma", "rho", "n_b")
    v = {nm: PAPER_PRIOR[nm][0] + u * (PAPER_PRIOR[nm][1] - PAPER_PRIOR[nm][0])
         for nm, u in zip(names, us)}
    n_b = int(round(v.pop("n_b")))
    return PaperPopulation(**v), n_b


def population_draw(seed: int, index: int, gamma_range=(3.0, 4.5), shape_range=(1.5, 3.0)):
    """Per-catalog population parameters drawn uniformly from the given ranges."""
    x0, x1, x2, x3 = philox4x32_10(index & 0xFFFFFFFF, index >> 32, _STREAM_POP, 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    ug, uk = float(u53(x0, x1)), float(u53(x2, x3))
    return Population(gamma=gamma_range[0] + ug * (gamma_range[1] - gamma_range[0]),
                      shape=shape_range[0] + uk * (shape_range[1] - shape_range[0]))


def job_draw(seed: int, index: int, n_range=(1e5, 3e7), years=(1, 2, 4)):
    """Size and observation time of a batched catalog or served job: N log-uniform, T from a set."""
    x0, x1, x2, x3 = philox4x32_10(index & 0xFFFFFFFF, index >> 32, _STREAM_POP + 1, 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    un, ut = float(u53(x0, x1)), float(u32(x2))
    lo, hi = float(plog(n_range[0])), float(plog(n_range[1]))
    n = int(round(float(pexp(lo + un * (hi - lo)))))
    T = years[min(len(years) - 1, int(ut * len(years)))] * YEAR
    return n, T, float(u32(x3))


# The benchmark and parity workloads (sizes, observation times, populations).
@dataclass
class Workload:
    name: str
    n_sources: int
    T_obs: float
    seed: int
    pop: Population


def workload(name: str) -> Workload:
    if name == "nb1e4_1yr":
        return Workload(name, 10_000, 1 * YEAR, 0, Population(11.0 / 3.0, 2.0))
    if name == "nb1e6_4yr":
        return Workload(name, 1_000_000, 4 * YEAR, 1, Population(11.0 / 3.0, 2.0))
    if name == "nb1e7_4yr":  # profiling size: the full-size population, a third of the sources
        return Workload(name, 10_000_000, 4 * YEAR, 2, population_draw(2, 0))
    if name == "nb3e7_4yr":
        return Workload(name, 30_000_000, 4 * YEAR, 2, population_draw(2, 0))
    raise KeyError(name)


def _catalog_task(args):
    n, seed, pop, start = args
    return catalog(n, seed, pop, start=start)


def catalogs_parallel(specs, procs=None, slice_size=1 << 21):
    """catalog(n, seed, pop) for every (n, seed, pop) of specs, computed by spawned worker
    processes over slices of each index range.  Every source is a pure function of its
    seed and index, so the result is identical to calling catalog() in this process."""
    import multiprocessing as mp
    import os
    procs = procs or min(16, os.cpu_count() or 1)
    tasks, owners = [], []
    for i, (n, seed, pop) in enumerate(specs):
        for s in range(0, n, slice_size):
            tasks.append((min(slice_size, n - s), seed, pop, s))
            owners.append(i)
    if procs <= 1 or len(tasks) <= 1:
        parts = [_catalog_task(t) for t in tasks]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            parts = pool.map(_catalog_task, tasks, chunksize=1)
    out = []
    for i, (n, _, _) in enumerate(specs):
        mine = [p for p, o in zip(parts, owners) if o == i]
        if not mine:
            out.append((np.empty(0), np.empty(0), np.empty(0)))
        else:
            out.append(tuple(np.concatenate([p[k] for p in mine]) for k in range(3)))
    return out
