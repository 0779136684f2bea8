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
};

constexpr unsigned kStreamFM = 0u;      // f and chirp mass
constexpr unsigned kStreamGamma = 1u;   // Gamma attempts use streams 1 .. kGammaTries
constexpr int kGammaTries = 24;

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

// Source s of the catalog: (A, f, fdot) in FP64.
__device__ __forceinline__ void gen_source(const GenParams& p, long long s, double* A, double* f,
                                           double* fdot) {
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
