// Device-side helpers shared by the subtraction kernels (arXiv 2602.18560, App. D).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbsub {

typedef unsigned long long u64;
typedef long long i64;

// ---------------------------------------------------------------- constants
constexpr double kC = 299792458.0;  // m/s
constexpr double kL = 2.5e9;        // LISA arm, m (Sec. III.A)
constexpr double kPi = 3.14159265358979323846;
// Chi^2_2 bias of the running median, (1 - 2/(9*2))^-3 = (8/9)^-3 = 729/512 (App. D).
constexpr double kMedianBias = 729.0 / 512.0;
// Scale of the deposited power in the catalog pass and the SNR thresholds: q = (P_k /
// S_instr,k) 2^96, i.e. units of 2^-96 of the instrument noise in that bin (the spectrum
// itself keeps q 2^-32, see q_parts).  A contribution must stay below 2^159 units (P/S below
// 2^63 in one bin).
constexpr double kQScale = 79228162514264337593543950336.0;                   // 2^96
// bits of 2^159, the first value of q beyond the fixed-point range
constexpr unsigned long long kQLimitBits = 0x49E0000000000000ull;
constexpr int kMaxWindow = 8192;

// Error bits raised on the device.
enum : unsigned { ERR_RANGE = 1u, ERR_INPUT = 2u, ERR_TIMEOUT = 8u };

// All three finite (exponent field not all ones), from the bits: no FP64 instruction.
__device__ __forceinline__ bool finite3(double a, double b, double c) {
  const unsigned long long m = 0x7FF0000000000000ull;
  return ((__double_as_longlong(a) & m) != m) && ((__double_as_longlong(b) & m) != m) &&
         ((__double_as_longlong(c) & m) != m);
}

// ---------------------------------------------------------------- 128-bit unsigned
struct U128 {
  u64 lo, hi;
};

__device__ __forceinline__ U128 u128_add(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ U128 u128_sub(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ bool u128_is_zero(U128 a) { return (a.lo | a.hi) == 0ull; }

// floor(x * 2^sh) for x >= 0 finite and the result below 2^127.
__device__ __forceinline__ U128 dbl_to_u128_scaled(double x, int sh) {
  U128 r{0ull, 0ull};
  u64 b = (u64)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7FF);
  u64 m = b & 0x000FFFFFFFFFFFFFull;
  if (e == 0) {
    if (m == 0) return r;
    e = 1;
  } else {
    m |= 0x0010000000000000ull;
  }
  int s = e - 1075 + sh;  // value = m * 2^s
  if (s >= 0) {
    if (s >= 64) {
      r.hi = m << (s - 64);
    } else {
      r.lo = m << s;
      r.hi = (s == 0) ? 0ull : (m >> (64 - s));
    }
  } else {
    int t = -s;
    r.lo = (t >= 64) ? 0ull : (m >> t);
  }
  return r;
}

// x 2^k for 1 <= x <= 2^64: k added to the exponent field (exact, no FP64 instruction)
// when the result is a normal number (-1022 <= k <= 959); otherwise ldexp.
__device__ __forceinline__ double scale_pow2(double x, int k) {
  if (k >= -1022 && k <= 959)
    return __longlong_as_double(__double_as_longlong(x) + ((long long)k << 52));
  return ldexp(x, k);
}

// Round-to-nearest double of v * 2^-sh.
__device__ __forceinline__ double u128_to_dbl_scaled(U128 v, int sh) {
  if (v.hi == 0ull) {
    if (v.lo == 0ull) return 0.0;
    return scale_pow2(__ull2double_rn(v.lo), -sh);
  }
  int lz = __clzll((i64)v.hi);      // 0..63
  int shift = 64 - lz;              // bits to drop so the top 64 bits remain
  u64 top = (v.hi << lz) | (lz ? (v.lo >> (64 - lz)) : 0ull);
  // the discarded low bits become a sticky bit so that rounding stays correct
  u64 low_mask = (lz == 0) ? ~0ull : ((1ull << (64 - lz)) - 1ull);
  u64 sticky = ((v.lo & low_mask) != 0ull) ? 1ull : 0ull;
  top |= sticky;
  return scale_pow2(__ull2double_rn(top), shift - sh);
}

// A bin of the spectrum is three 64-bit words holding Q = w2 2^64 + w1 2^32 + w0 in units of
// 2^-64 S_instr of the bin (a fourth word pads the bin to 32 bytes).  Each contribution, an
// integer number of units (q 2^-32 of its value q in units of 2^-96 S_instr, truncated), is
// split in bits 0-31 (into w0), bits 32-63 (w1) and bits 64-127 (w2): w0 and w1 take fewer
// than 2^32 terms below 2^32, so no word overflows while Q stays below 2^127 (P/S_instr below
// 2^63), and Q is exact whatever the order of the additions; removing a contribution
// subtracts the same three parts.  w2 takes a part only for a contribution of at least
// S_instr, so most deposits are two 64-bit atomics.
__device__ __forceinline__ void q_parts(double q, u64* c0, u64* c1, u64* c2) {
  U128 v = dbl_to_u128_scaled(q, -32);
  *c0 = v.lo & 0xFFFFFFFFull;
  *c1 = v.lo >> 32;
  *c2 = v.hi;
}

// The deposit of a single-bin source, q = A^2 gq (units of 2^-96 of the bin's S_instr;
// gq = 2^96 (T/5) R / S_instr), from the integer mantissas: the top 64 bits of A's mantissa
// squared, times gq's, the products truncated.  It is within 2^-61 of the exact A^2 gq (the
// FP64 product RN(RN(A A) gq) is within 2^-52) and takes no FP64 instruction, which on this
// GPU runs at a small fraction of the integer rate.
//   c0, c1, c2 : the parts the spectrum words take (q_parts: bits 0-31, 32-63 and 64-127 of
//                Q = q 2^-32)
//   qbits      : q as the bits of a double (mantissa truncated), for comparisons with the
//                bits of non-negative doubles
// Returns false when q >= 2^159 (beyond the fixed-point range).  A finite (its sign does not
// matter), gq > 0 finite; A or gq zero or subnormal gives q = 0.
__device__ __forceinline__ bool q_single(double A, double gq, u64* c0, u64* c1, u64* c2,
                                         u64* qbits) {
  const u64 ba = (u64)__double_as_longlong(A), bg = (u64)__double_as_longlong(gq);
  const int ea = (int)((ba >> 52) & 0x7FF), eg = (int)((bg >> 52) & 0x7FF);
  *c0 = 0ull;
  *c1 = 0ull;
  *c2 = 0ull;
  *qbits = 0ull;
  if (ea == 0 || eg == 0) return true;
  const u64 a = ((ba & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  const u64 g = ((bg & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  const u64 a2 = __umul64hi(a, a);  // in [2^62, 2^64)
  const u64 p = __umul64hi(a2, g);  // in [2^61, 2^64)
  const int sh = 2 * ea + eg - 3130;  // q = p 2^sh
  const int lz = __clzll((long long)p);
  const int E = sh + 63 - lz;         // q in [2^E, 2^(E+1))
  if (E >= 159) return false;
  if (E >= -1022) *qbits = ((u64)(E + 1023) << 52) | ((p << (lz + 1)) >> 12);
  const int t = sh - 32;              // Q = q 2^-32 = p 2^t, Q = hi 2^64 + lo
  u64 lo = 0ull, hi = 0ull;
  if (t >= 64) {
    hi = p << (t - 64);
  } else if (t > 0) {
    lo = p << t;
    hi = p >> (64 - t);
  } else if (t == 0) {
    lo = p;
  } else if (t > -64) {
    lo = p >> (-t);
  }
  *c0 = lo & 0xFFFFFFFFull;
  *c1 = lo >> 32;
  *c2 = hi;
  return true;
}

// f * T rounded to nearest (ties to even), computed exactly in integer arithmetic, returned
// as x = u + 1/2 split into its integer part k and the top 24 bits of its fraction.  T is
// given by its 53-bit integer mantissa mT and exponent eT (T = mT 2^eT).  Returns false when
// the product is out of the range handled here (f not a positive normal number, or
// f T >= 2^30), in which case the caller uses plain FP64.
__device__ __forceinline__ bool ft_bin(double f, u64 mT, int eT, long long* k, unsigned* frac24,
                                       int* fracbits) {
  u64 b = (u64)__double_as_longlong(f);
  int e = (int)((b >> 52) & 0x7FF);
  if ((b >> 63) || e == 0 || e == 0x7FF) return false;
  u64 mf = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  u64 lo = mf * mT;
  u64 hi = __umul64hi(mf, mT);  // product in [2^104, 2^106)
  int sh = ((hi >> 41) & 1ull) ? 53 : 52;
  // M = p >> sh with round-to-nearest-even on the dropped bits
  u64 M = (hi << (64 - sh)) | (lo >> sh);
  u64 rmask = (1ull << sh) - 1ull;
  u64 r = lo & rmask;
  u64 half = 1ull << (sh - 1);
  if (r > half || (r == half && (M & 1ull))) {
    ++M;
    if (M >> 53) {
      M >>= 1;
      ++sh;
    }
  }
  int E = (e - 1075) + eT + sh;  // f T = M 2^E
  if (E > -23 || E < -62) return false;
  int F = -E;                    // fraction bits of M
  u64 x = M + (1ull << (F - 1)); // (f T + 1/2) 2^F
  *k = (long long)(x >> F);
  u64 fr = x & ((1ull << F) - 1ull);
  *frac24 = (F >= 24) ? (unsigned)(fr >> (F - 24)) : (unsigned)(fr << (24 - F));
  *fracbits = F;
  return true;
}

// Signed FP32 value of a double (truncated mantissa); 0 below the FP32 normal range.
__device__ __forceinline__ float dbl_to_f32_signed(double v) {
  u64 b = (u64)__double_as_longlong(v);
  int e = (int)((b >> 52) & 0x7FF);
  int ef = e - 1023 + 127;
  if (e == 0 || ef <= 0) return 0.0f;
  if (ef >= 255) return __int_as_float(0x7FC00000);
  unsigned fb = ((unsigned)(b >> 63) << 31) | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7FFFFFu);
  return __uint_as_float(fb);
}

__device__ __forceinline__ U128 q_combine3(u64 w0, u64 w1, u64 w2) {
  U128 r;
  r.lo = w0 + (w1 << 32);
  r.hi = w2 + (w1 >> 32) + (r.lo < w0 ? 1ull : 0ull);
  return r;
}

// v * 2^sh as an FP32 number, truncated (relative error < 2^-23), flushed to 0 below
// the normal range and saturated at the largest float.  Integer operations only.
__device__ __forceinline__ float dbl_to_f32_scaled(double v, int sh) {
  u64 b = (u64)__double_as_longlong(v);
  int e = (int)((b >> 52) & 0x7FF);
  if (e == 0 || (b >> 63)) return 0.0f;
  int ef = e - 1023 + 127 + sh;
  if (ef <= 0) return 0.0f;
  if (ef >= 255) return 3.4028234e38f;
  unsigned fb = ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7FFFFFu);
  return __uint_as_float(fb);
}

// ---------------------------------------------------------------- source pieces
// Sweep of a source in bin units (Eqs. GB waveform / phase Taylor expansion):
// the instantaneous frequency f + fdot t over [0, T] spans [u0, u1] =
// [f T, f T + fdot T^2]; the weight of bin k is the fraction of the sweep inside
// the cell [k - 1/2, k + 1/2).  Products and sums use explicit round-to-nearest
// intrinsics so that no multiply-add is fused.
struct Sweep {
  double lo, hi;  // sorted endpoints in bin units
  i64 ka, kb;     // first and last cell touched
};

__device__ __forceinline__ Sweep make_sweep(double f, double fdot, double T, double T2) {
  Sweep s;
  double u0 = __dmul_rn(f, T);
  double du = __dmul_rn(fdot, T2);
  double u1 = __dadd_rn(u0, du);
  s.lo = fmin(u0, u1);
  s.hi = fmax(u0, u1);
  s.ka = (i64)floor(__dadd_rn(s.lo, 0.5));
  s.kb = (i64)floor(__dadd_rn(s.hi, 0.5));
  return s;
}

// Weight of cell k for a sweep that touches more than one cell (the FP64 decision of the
// SNR uses this, the oracle's own division).
__device__ __forceinline__ double sweep_weight(const Sweep& s, i64 k) {
  double a = fmax(s.lo, __dsub_rn((double)k, 0.5));
  double b = fmin(s.hi, __dadd_rn((double)k, 0.5));
  if (!(b > a)) return 0.0;
  return __ddiv_rn(__dsub_rn(b, a), __dsub_rn(s.hi, s.lo));
}

// The same weight as (b - a) times inv = RN(1 / (hi - lo)), one division per sweep instead of
// one per cell (an FP64 division is a dozen FP64-pipe operations on this GPU).  Within one
// rounding of sweep_weight; the deposits and the removals both use it, so a removal still
// cancels its deposit exactly.
__device__ __forceinline__ double sweep_inv_len(const Sweep& s) {
  return __drcp_rn(__dsub_rn(s.hi, s.lo));
}
__device__ __forceinline__ double sweep_weight_inv(const Sweep& s, i64 k, double inv) {
  double a = fmax(s.lo, __dsub_rn((double)k, 0.5));
  double b = fmin(s.hi, __dadd_rn((double)k, 0.5));
  if (!(b > a)) return 0.0;
  return __dmul_rn(__dsub_rn(b, a), inv);
}

}  // namespace gbsub
