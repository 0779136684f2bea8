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
// Per-bin fixed point of the deposited power: q = (P_k / S_instr,k) * 2^64, i.e. the
// unit is 2^-64 of the instrument noise in that bin.  A contribution must stay below
// 2^95 units (P/S < 2^31); the accumulator of a bin holds < 2^96 units.
constexpr double kQScale = 18446744073709551616.0;        // 2^64
constexpr double kQLimit = 39614081257132168796771975168.0;  // 2^95
constexpr int kMaxWindow = 8192;
constexpr int kSnapStride = 32;   // positions between stored active-set snapshots

// Error bits raised on the device.
enum : unsigned { ERR_RANGE = 1u, ERR_WINDOW = 2u, ERR_CAND = 4u };

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

// Round-to-nearest double of v * 2^-sh.
__device__ __forceinline__ double u128_to_dbl_scaled(U128 v, int sh) {
  if (v.hi == 0ull) {
    if (v.lo == 0ull) return 0.0;
    return ldexp(__ull2double_rn(v.lo), -sh);
  }
  int lz = __clzll((i64)v.hi);      // 0..63
  int shift = 64 - lz;              // bits to drop so the top 64 bits remain
  u64 top = (v.hi << lz) | (lz ? (v.lo >> (64 - lz)) : 0ull);
  // the discarded low bits become a sticky bit so that rounding stays correct
  u64 low_mask = (lz == 0) ? ~0ull : ((1ull << (64 - lz)) - 1ull);
  u64 sticky = ((v.lo & low_mask) != 0ull) ? 1ull : 0ull;
  top |= sticky;
  return ldexp(__ull2double_rn(top), shift - sh);
}

// Split a fixed-point contribution q (a double holding an integer-valued
// amount of units, q < 2^95) into the part below 2^32 and the part above.
// Both halves are accumulated in 64-bit words: the low word takes fewer than
// 2^32 terms below 2^32 each, so neither word overflows and the sum
// acc_hi * 2^32 + acc_lo is exact whatever the order of the additions.
__device__ __forceinline__ void q_split(double q, u64* lo32, u64* hi64) {
  U128 v = dbl_to_u128_scaled(q, 0);
  *lo32 = v.lo & 0xFFFFFFFFull;
  *hi64 = (v.lo >> 32) | (v.hi << 32);
}

__device__ __forceinline__ U128 q_combine(u64 acc_lo, u64 acc_hi) {
  U128 r;
  r.lo = acc_lo + (acc_hi << 32);
  r.hi = (acc_hi >> 32) + (r.lo < acc_lo ? 1ull : 0ull);
  return r;
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

// Weight of cell k for a sweep that touches more than one cell.
__device__ __forceinline__ double sweep_weight(const Sweep& s, i64 k) {
  double a = fmax(s.lo, __dsub_rn((double)k, 0.5));
  double b = fmin(s.hi, __dadd_rn((double)k, 0.5));
  if (!(b > a)) return 0.0;
  return __ddiv_rn(__dsub_rn(b, a), __dsub_rn(s.hi, s.lo));
}

// ---------------------------------------------------------------- bitsets
// Smallest set bit index >= i in words[0 .. nw), stride-addressed (word w at
// words[w * stride]); returns limit if none below limit.
__device__ __forceinline__ int bs_next(const uint32_t* words, int stride, int nw, int i, int limit) {
  if (i >= limit) return limit;
  int w = i >> 5;
  uint32_t bits = words[w * stride] & (0xFFFFFFFFu << (i & 31));
  while (bits == 0u) {
    ++w;
    if (w >= nw) return limit;
    bits = words[w * stride];
  }
  int r = (w << 5) + __ffs(bits) - 1;
  return r < limit ? r : limit;
}

// Largest set bit index < i; -1 if none.
__device__ __forceinline__ int bs_prev(const uint32_t* words, int stride, int i) {
  if (i <= 0) return -1;
  int w = (i - 1) >> 5;
  int sh = (i - 1) & 31;
  uint32_t mask = (sh == 31) ? 0xFFFFFFFFu : ((2u << sh) - 1u);
  uint32_t bits = words[w * stride] & mask;
  while (bits == 0u) {
    --w;
    if (w < 0) return -1;
    bits = words[w * stride];
  }
  return (w << 5) + 31 - __clz(bits);
}

}  // namespace gbsub
