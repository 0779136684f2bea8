// On-device catalog generation: the single-precision catalog recipe.
//
// Counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published
// definition: every number a source needs is a pure function of (seed, source index,
// stream), so any source can be generated, or generated again, on its own.
// Distributions (the synthetic stand-in for the paper's population catalogs):
//   f    : truncated power law p(f) ~ f^-gamma on [1e-4, 1e-2] Hz, by inverse CDF in a form
//          without cancellation: f = f0 (rho + u (1 - rho))^(1/(1-gamma)), f0 the end of
//          highest density and rho = (f1/f0)^(1-gamma) < 1, so the sparse tail comes from
//          small u (log-uniform within 1e-3 of gamma = 1)
//   A    : 1e-23 X (f / 1e-3 Hz)^(2/3), X ~ Gamma(shape, 1) (Marsaglia-Tsang, with a
//          polar-method normal per attempt)
//   fdot : (96/5) pi^(8/3) Mc^(5/3) f^(11/3), Mc ~ U(0.2, 0.8) G Msun / c^3 (the GW-driven
//          chirp of Sec. II.A)
// All arithmetic is IEEE single precision with round-to-nearest intrinsics and no fused
// multiply-add; log and exp are series evaluations (atanh series to t^13 after a binary
// reduction; Taylor series to r^8 after reduction by ln 2), so the host's float32
// evaluation of the same steps gives the same bits.  The values are returned as FP64.
#pragma once

#include <cstdint>

namespace gbsub {

struct GenParams {
  unsigned k0, k1;       // seed (low, high word)
  int power;             // 1: power law; 0: log-uniform (gamma within 1e-3 of 1)
  float lf0, rho, omr;   // power law: f = exp(lf0 + inv_e log(rho + u omr)), omr = 1 - rho
  float inv_e;
  float lmin, span;      // log-uniform: f = exp(lmin + u span)
  float d, c;            // Marsaglia-Tsang constants of Gamma(shape, 1)
  float pref, log1e3;    // (96/5) pi^(8/3); log(1e-3)
  // the paper's population (kind 1; the power law above is p(f) ~ f^alpha_pl, the Gamma
  // above has shape alpha_g)
  int kind;              // 0: the synthetic recipe above; 1: the paper's population
  float beta, alpha, gln;       // Gamma rate, shape, log Gamma(shape)
  float mu_g, mu, sigma;        // offsets of log10 fdot and of the rescaled log amplitude;
                                // log-normal width
  float rho_cop, rho_c;         // copula correlation, sqrt(1 - rho^2)
};

// The paper's population parameters (Table I), as doubles.
struct PaperPop {
  double alpha_pl, alpha_g, beta_g, mu_g, mu, sigma, rho;
};

constexpr unsigned kStreamFM = 0u;      // f and chirp mass
constexpr unsigned kStreamGamma = 1u;   // Gamma attempts use streams 1 .. kGammaTries
constexpr int kGammaTries = 24;
constexpr unsigned kStreamPaper = 32u;  // the paper population's copula and amplitude

__host__ __device__ __forceinline__ void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned long long p0 = 0xD2511F53ull * c[0];
    const unsigned long long p1 = 0xCD9E8D57ull * c[2];
    const unsigned hi0 = (unsigned)(p0 >> 32), lo0 = (unsigned)p0;
    const unsigned hi1 = (unsigned)(p1 >> 32), lo1 = (unsigned)p1;
    const unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

#ifdef __CUDACC__
__device__ __forceinline__ float gen_u32f(unsigned x) {
  // (x + 1/2) / 2^32: dividing by a power of two is the exact product with its inverse
  return __fmul_rn(__fadd_rn(__uint2float_rn(x), 0.5f), 2.3283064365386963e-10f);
}

// Uniform in [2^-24, 1 - 2^-24] from the top 23 bits of a word: never 0 or 1, so that a
// normal deviate from it stays within 5.3 standard deviations (gen_u32f can round to 1).
__device__ __forceinline__ float gen_u23f(unsigned x) {
  return __fmul_rn(__fadd_rn(__uint2float_rn(x >> 9), 0.5f), 1.1920928955078125e-07f);
}

__device__ __forceinline__ float gen_log(float x) {
  const float tiny = (float)1.1754943508222875e-38;  // smallest normal
  if (!(x >= tiny)) x = tiny;
  const unsigned bits = __float_as_uint(x);
  int e = (int)((bits >> 23) & 0xFFu) - 126;                       // x = m 2^e, m in [1/2, 1)
  float m = __uint_as_float((bits & 0x807FFFFFu) | 0x3F000000u);
  if (m < (float)0.7071067811865476) {
    m = __fmul_rn(m, 2.0f);
    e -= 1;
  }
  const float ef = (float)e;
  const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float t2 = __fmul_rn(t, t);
  float acc = (float)(1.0 / 13.0);
  acc = __fadd_rn(__fmul_rn(acc, t2), (float)(1.0 / 11.0));
  acc = __fadd_rn(__fmul_rn(acc, t2), (float)(1.0 / 9.0));
  acc = __fadd_rn(__fmul_rn(acc, t2), (float)(1.0 / 7.0));
  acc = __fadd_rn(__fmul_rn(acc, t2), (float)(1.0 / 5.0));
  acc = __fadd_rn(__fmul_rn(acc, t2), (float)(1.0 / 3.0));
  acc = __fadd_rn(__fmul_rn(acc, t2), 1.0f);
  const float hi = __fmul_rn(ef, (float)0.693145751953125);
  const float lo = __fadd_rn(__fmul_rn(ef, (float)1.4286067653301870e-06),
                             __fmul_rn(__fmul_rn(2.0f, t), acc));
  return __fadd_rn(hi, lo);
}

__device__ __forceinline__ float gen_exp(float x) {
  const float k = rintf(__fdiv_rn(x, (float)0.6931471805599453));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(k, (float)0.693145751953125)),
                            __fmul_rn(k, (float)1.4286067653301870e-06));
  float acc = (float)(1.0 / 40320.0);
  acc = __fadd_rn(__fmul_rn(acc, r), (float)(1.0 / 5040.0));
  acc = __fadd_rn(__fmul_rn(acc, r), (float)(1.0 / 720.0));
  acc = __fadd_rn(__fmul_rn(acc, r), (float)(1.0 / 120.0));
  acc = __fadd_rn(__fmul_rn(acc, r), (float)(1.0 / 24.0));
  acc = __fadd_rn(__fmul_rn(acc, r), (float)(1.0 / 6.0));
  acc = __fadd_rn(__fmul_rn(acc, r), 0.5f);
  acc = __fadd_rn(__fmul_rn(acc, r), 1.0f);
  acc = __fadd_rn(__fmul_rn(acc, r), 1.0f);
  // times 2^k, exact: k stays within [-126, 127] and every result here is a normal float
  return __fmul_rn(acc, __uint_as_float((unsigned)((int)k + 127) << 23));
}

// Gamma(d + 1/3, 1): Marsaglia-Tsang over counter-based attempts (a polar-method normal
// each); d itself when every attempt is refused.
__device__ __forceinline__ float gen_gamma(const GenParams& p, unsigned lo, unsigned hi) {
  float X = p.d;
  for (int t = 0; t < kGammaTries; ++t) {
    unsigned y[4] = {lo, hi, kStreamGamma + (unsigned)t, 0u};
    philox4x32_10(y, p.k0, p.k1);
    const float pp = __fsub_rn(__fmul_rn(2.0f, gen_u32f(y[0])), 1.0f);
    const float qq = __fsub_rn(__fmul_rn(2.0f, gen_u32f(y[1])), 1.0f);
    float s2 = __fadd_rn(__fmul_rn(pp, pp), __fmul_rn(qq, qq));
    const bool inside = (s2 < 1.0f) && (s2 > 0.0f);
    if (!inside) s2 = 0.5f;
    const float z = __fmul_rn(pp, __fsqrt_rn(__fdiv_rn(__fmul_rn(-2.0f, gen_log(s2)), s2)));
    float v = __fadd_rn(1.0f, __fmul_rn(p.c, z));
    const bool ok = inside && (v > 0.0f);
    v = ok ? __fmul_rn(__fmul_rn(v, v), v) : 1.0f;
    const float ua = gen_u32f(y[2]);
    const float rhs = __fadd_rn(__fsub_rn(__fadd_rn(__fmul_rn(__fmul_rn(0.5f, z), z), p.d),
                                          __fmul_rn(p.d, v)),
                                __fmul_rn(p.d, gen_log(v)));
    if (ok && gen_log(ua) < rhs) {
      X = __fmul_rn(p.d, v);
      break;
    }
  }
  return X;
}

__device__ __forceinline__ float gen_horner(float x, const float* c, int n, bool one_last) {
  float acc = c[0];
  for (int i = 1; i < n; ++i) acc = __fadd_rn(__fmul_rn(acc, x), c[i]);
  if (one_last) acc = __fadd_rn(__fmul_rn(acc, x), (float)1.0);
  return acc;
}

// Phi^-1(t) for 0 < t <= 1/2: Wichura's AS241 in its single-precision form PPND7 (Applied
// Statistics 37, 1988).
__device__ __forceinline__ float gen_ppf_lower(float t) {
  const float A[4] = {(float)59.109374720, (float)159.29113202, (float)50.434271938, (float)3.3871327179};
  const float B[3] = {(float)67.187563600, (float)78.757757664, (float)17.895169469};
  const float C[4] = {(float)0.17023821103, (float)1.3067284816, (float)2.7568153900, (float)1.4234372777};
  const float D[2] = {(float)0.12021132975, (float)0.73700164250};
  const float E[4] = {(float)0.017337203997, (float)0.42868294337, (float)3.0812263860, (float)6.6579051150};
  const float F[2] = {(float)0.012258202635, (float)0.24197894225};
  const float q = __fsub_rn(t, (float)0.5);
  if (fabsf(q) <= (float)0.425) {
    const float r = __fsub_rn((float)0.180625, __fmul_rn(q, q));
    return __fdiv_rn(__fmul_rn(q, gen_horner(r, A, 4, false)), gen_horner(r, B, 3, true));
  }
  const float rt = __fsqrt_rn(__fsub_rn((float)0.0, gen_log(t)));
  float v;
  if (rt <= (float)5.0) {
    const float r1 = __fsub_rn(rt, (float)1.6);
    v = __fdiv_rn(gen_horner(r1, C, 4, false), gen_horner(r1, D, 2, true));
  } else {
    const float r2 = __fsub_rn(rt, (float)5.0);
    v = __fdiv_rn(gen_horner(r2, E, 4, false), gen_horner(r2, F, 2, true));
  }
  return __fsub_rn((float)0.0, v);
}

// Phi^-1(u), 0 < u < 1 (the upper half by symmetry; 1 - u is exact there).
__device__ __forceinline__ float gen_ppf(float u) {
  return u <= (float)0.5 ? gen_ppf_lower(u) : -gen_ppf_lower(__fsub_rn((float)1.0, u));
}

// erfc(x), x >= 0: the Chebyshev fit of Numerical Recipes (Press et al., 2nd ed., Sec. 6.2),
// fractional error below 1.2e-7.
__device__ __forceinline__ float gen_erfc(float x) {
  const float Cc[10] = {(float)0.17087277, (float)-0.82215223, (float)1.48851587, (float)-1.13520398, (float)0.27886807,
                        (float)-0.18628806, (float)0.09678418, (float)0.37409196, (float)1.00002368, (float)-1.26551223};
  const float t = __fdiv_rn((float)1.0, __fadd_rn((float)1.0, __fmul_rn((float)0.5, x)));
  const float acc = gen_horner(t, Cc, 10, false);
  const float arg = fmaxf(__fadd_rn(__fsub_rn((float)0.0, __fmul_rn(x, x)), acc), (float)-87.0);
  return __fmul_rn(t, gen_exp(arg));
}

// Phi(-z): the upper tail probability of a standard normal.
__device__ __forceinline__ float gen_sf(float z) {
  const float e = __fmul_rn((float)0.5, gen_erfc(__fmul_rn(fabsf(z), (float)0.7071067811865476)));
  return z >= (float)0.0 ? e : __fsub_rn((float)1.0, e);
}

// log Gamma(a), a > 0: the Lanczos form with g = 5 and six terms (Numerical Recipes,
// Sec. 6.1).
__device__ __forceinline__ float gen_lgamma(float a) {
  const float cof[6] = {(float)76.18009172947146, (float)-86.50532032941677, (float)24.01409824083091,
                        (float)-1.231739572450155, (float)0.1208650973866179e-2, (float)-0.5395239384953e-5};
  float y = a;
  float tmp = __fadd_rn(a, (float)5.5);
  tmp = __fsub_rn(tmp, __fmul_rn(__fadd_rn(a, (float)0.5), gen_log(tmp)));
  float ser = (float)1.000000000190015;
  for (int i = 0; i < 6; ++i) {
    y = __fadd_rn(y, (float)1.0);
    ser = __fadd_rn(ser, __fdiv_rn(cof[i], y));
  }
  return __fadd_rn(-tmp, gen_log(__fdiv_rn(__fmul_rn((float)2.5066282746310005, ser), a)));
}

// (P, Q): the regularized lower and upper incomplete gamma functions of shape a at x >= 0,
// by the series for x < a + 1 (Q = 1 - P) and the continued fraction (modified Lentz) for Q
// otherwise (P = 1 - Q), at most 64 terms; gln = log Gamma(a).
__device__ __forceinline__ void gen_gamma_pq(float a, float x, float gln, float* P, float* Q) {
  const float eps = (float)5.9604644775390625e-08, fpmin = 1e-30f;
  const float xs = fmaxf(x, 1e-30f);
  const float parg =
      fmaxf(__fsub_rn(__fadd_rn(__fsub_rn((float)0.0, x), __fmul_rn(a, gen_log(xs))), gln), (float)-87.0);
  const float pref = gen_exp(parg);
  if (x < __fadd_rn(a, (float)1.0)) {
    float ap = a, ssum = __fdiv_rn((float)1.0, a), dl = ssum;
    for (int i = 0; i < 64; ++i) {
      ap = __fadd_rn(ap, (float)1.0);
      dl = __fdiv_rn(__fmul_rn(dl, x), ap);
      ssum = __fadd_rn(ssum, dl);
      if (fabsf(dl) < __fmul_rn(fabsf(ssum), eps)) break;
    }
    const float ps = __fmul_rn(ssum, pref);
    *P = ps;
    *Q = __fsub_rn((float)1.0, ps);
    return;
  }
  float b = __fsub_rn(__fadd_rn(x, (float)1.0), a);
  float c = __fdiv_rn((float)1.0, fpmin);
  float d = __fdiv_rn((float)1.0, b);
  float h = d;
  for (int i = 1; i <= 64; ++i) {
    const float an = __fmul_rn((float)(-i), __fsub_rn((float)i, a));
    b = __fadd_rn(b, (float)2.0);
    d = __fadd_rn(__fmul_rn(an, d), b);
    if (fabsf(d) < fpmin) d = fpmin;
    c = __fadd_rn(b, __fdiv_rn(an, c));
    if (fabsf(c) < fpmin) c = fpmin;
    d = __fdiv_rn((float)1.0, d);
    const float de = __fmul_rn(d, c);
    h = __fmul_rn(h, de);
    if (fabsf(__fsub_rn(de, (float)1.0)) < eps) break;
  }
  const float qc = __fmul_rn(pref, h);
  *P = __fsub_rn((float)1.0, qc);
  *Q = qc;
}

// Source s of the paper's population (Sec. II.B, Table I; App. A): xi = G / beta with
// G ~ Gamma(alpha_g, 1), z2 = Phi^-1(F_Gamma(xi)), z1 = rho z2 + sqrt(1 - rho^2) n, f from the
// power law at tail probability Phi(-z1), fdot = 10^(mu_g + xi),
// A = f^(2/3) 10^(mu + exp(sigma n')) with n, n' independent standard normals.
__device__ __forceinline__ void gen_source_paper(const GenParams& p, long long s, double* A,
                                                 double* f, double* fdot) {
  const unsigned lo = (unsigned)(unsigned long long)s, hi = (unsigned)((unsigned long long)s >> 32);
  const float G = gen_gamma(p, lo, hi);
  const float xi = __fdiv_rn(G, p.beta);
  float P, Q;
  gen_gamma_pq(p.alpha, G, p.gln, &P, &Q);
  const float z2 = P <= (float)0.5 ? gen_ppf_lower(P) : -gen_ppf_lower(Q);
  unsigned x[4] = {lo, hi, kStreamPaper, 0u};
  philox4x32_10(x, p.k0, p.k1);
  const float z1 = __fadd_rn(__fmul_rn(p.rho_cop, z2), __fmul_rn(p.rho_c, gen_ppf(gen_u23f(x[0]))));
  const float ut = gen_sf(z1);
  const float lf = p.power
                       ? __fadd_rn(p.lf0, __fmul_rn(p.inv_e, gen_log(__fadd_rn(p.rho, __fmul_rn(ut, p.omr)))))
                       : __fadd_rn(p.lmin, __fmul_rn(__fsub_rn((float)1.0, ut), p.span));
  const float ln10 = (float)2.302585092994046;
  const float fs = gen_exp(lf);
  const float fd = gen_exp(__fmul_rn(ln10, __fadd_rn(p.mu_g, xi)));
  const float am = gen_exp(__fmul_rn(p.sigma, gen_ppf(gen_u23f(x[1]))));
  const float a = gen_exp(__fadd_rn(__fmul_rn((float)(2.0 / 3.0), lf),
                                    __fmul_rn(ln10, __fadd_rn(p.mu, am))));
  *A = (double)a;
  *f = (double)fs;
  *fdot = (double)fd;
}

// Source s of the catalog: (A, f, fdot) in FP64.
__device__ __forceinline__ void gen_source(const GenParams& p, long long s, double* A, double* f,
                                           double* fdot) {
  if (p.kind == 1) {
    gen_source_paper(p, s, A, f, fdot);
    return;
  }
  const unsigned lo = (unsigned)(unsigned long long)s, hi = (unsigned)((unsigned long long)s >> 32);
  unsigned x[4] = {lo, hi, kStreamFM, 0u};
  philox4x32_10(x, p.k0, p.k1);
  const float u = gen_u32f(x[0]);
  // log f is the exponent that f comes from (no second logarithm)
  const float lf = p.power
                       ? __fadd_rn(p.lf0, __fmul_rn(p.inv_e, gen_log(__fadd_rn(p.rho, __fmul_rn(u, p.omr)))))
                       : __fadd_rn(p.lmin, __fmul_rn(u, p.span));
  const float fs = gen_exp(lf);
  const float mc = __fmul_rn(__fadd_rn((float)0.2, __fmul_rn((float)0.6, gen_u32f(x[2]))),
                             (float)4.925490947e-6);
  const float X = gen_gamma(p, lo, hi);
  const float fd = __fmul_rn(p.pref, gen_exp(__fadd_rn(__fmul_rn((float)(5.0 / 3.0), gen_log(mc)),
                                                      __fmul_rn((float)(11.0 / 3.0), lf))));
  const float a = __fmul_rn(__fmul_rn((float)1e-23, X),
                            gen_exp(__fmul_rn((float)(2.0 / 3.0), __fsub_rn(lf, p.log1e3))));
  *A = (double)a;
  *f = (double)fs;
  *fdot = (double)fd;
}
#endif

}  // namespace gbsub
