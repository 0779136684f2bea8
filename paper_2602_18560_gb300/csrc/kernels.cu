// CUDA kernels of the iterative galactic-binary subtraction (arXiv 2602.18560, App. D),
// written for sm_103a (GB300).
//
// Steps of one run:
//   tables   : S_instr(f_k) (App. C, SciRDv1 A channel, TDI-2 factor), R(f_k) (App. B)
//              and the scales derived from them.                              [per context]
//   prepass  : one pass over the catalog: the bins each chirp sweeps, its power deposited
//              into an exact fixed-point spectrum, rho_0 against S_instr, the paper's
//              candidates (rho_0 >= kappa rho_th) counted and the ones that can still be
//              resolved (rho_0 > rho_th) kept.                                [per run]
//   loop     : S_gal = estimator of P_k = S_k Q_k 2^-96 (running mean / running median /
//              median then mean, Eqs. running mean, running median); rho of each kept
//              candidate against S_instr + S_gal (Eqs. SNR inner product, inner product);
//              sources with rho > rho_th removed from the spectrum exactly; loop control
//              on the device.
//
// No floating-point atomics: the spectrum is an integer (units of 2^-96 S_instr,k per bin),
// so deposits and removals commute and every run gives the same bits.  GB300 runs FP64 at
// 1/58 of the FP32 rate, so per-iteration work avoids FP64: medians select on the integer
// bits of the doubles, window sums are integer, and the SNR test is screened in FP32 with
// a proven error margin (exact FP64 recomputation inside the margin).

#include <cuda_runtime.h>
#include <cuda_device_runtime_api.h>

#include "common.cuh"
#include "kernels.cuh"

namespace gbsub {

// ============================================================================ tables

__global__ void k_tables(Grid g, int tdi2, double* __restrict__ S, double* __restrict__ R,
                         double* __restrict__ gq, float* __restrict__ Gf,
                         float* __restrict__ invSf) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= g.nb) return;
  const double fstar = kC / (2.0 * kPi * kL);
  double f = (double)(g.k_lo + j) / g.T;
  double x = f / fstar;
  double sx, cx;
  sincos(x, &sx, &cx);
  // P_OMS = (15 pm)^2 [1 + (2 mHz/f)^4] (2 pi f / c)^2
  double r = 2.0e-3 / f;
  double w = 2.0 * kPi * f / kC;
  double p_oms = 15.0e-12 * 15.0e-12 * (1.0 + r * r * r * r) * w * w;
  // P_TM = (3 fm/s^2)^2 [1 + (0.4 mHz/f)^2][1 + (f / 8 mHz)^4] (2 pi f)^-4 (2 pi f / c)^2
  double r1 = 0.4e-3 / f, r2 = f / 8.0e-3;
  double om = 2.0 * kPi * f;
  double p_tm = 3.0e-15 * 3.0e-15 * (1.0 + r1 * r1) * (1.0 + r2 * r2 * r2 * r2) /
                (om * om * om * om) * w * w;
  double s_aa = 8.0 * sx * sx * (4.0 * (1.0 + cx + cx * cx) * p_tm + (2.0 + cx) * p_oms);
  double resp = 16.0 * sx * sx * x * x * (9.0 / 20.0) / (1.0 + 0.7 * x * x);
  if (tdi2) {
    double s2 = sin(2.0 * x);
    double t2 = 4.0 * s2 * s2;
    s_aa *= t2;
    resp *= t2;
  }
  S[j] = s_aa;
  R[j] = resp;
  double ratio = g.t5 * resp / s_aa;          // P / S per unit of A^2 w
  gq[j] = kQScale * ratio;                    // fixed-point units per unit of A^2 w
  // FP32 screen factors; outside the normal FP32 range they are NaN, which sends every
  // SNR decision touching the bin to the exact FP64 path.
  double gs = ldexp(4.0 * ratio, -160);       // rho^2 against S_instr per unit A^2 w 2^160
  double is = 1.0 / ldexp(s_aa, 150);
  const double fmin_n = 1.1754943508222875e-38, fmax_n = 3.4028234663852886e38;
  Gf[j] = (gs >= fmin_n && gs <= fmax_n) ? (float)gs : __int_as_float(0x7FC00000);
  invSf[j] = (is >= fmin_n && is <= fmax_n) ? (float)is : __int_as_float(0x7FC00000);
}

void launch_tables(const Grid& g, int tdi2, double* S, double* R, double* gq, float* Gf,
                   float* invSf, cudaStream_t st) {
  int th = 256;
  long long bl = (g.nb + th - 1) / th;
  k_tables<<<(unsigned)bl, th, 0, st>>>(g, tdi2, S, R, gq, Gf, invSf);
}

// ============================================================================ spectrum I/O

__device__ __forceinline__ void deposit_q(unsigned long long* acc, long long j, double q,
                                          unsigned* err) {
  // q >= 0: compare the bits with those of 2^127 (no FP64 instruction)
  if ((u64)__double_as_longlong(q) >= 0x47E0000000000000ull) {
    atomicOr(err, ERR_RANGE);
    return;
  }
  u64 c0, c1, c2;
  q_parts(q, &c0, &c1, &c2);
  u64* a = acc + 4 * j;
  if (c0) atomicAdd(a + 0, c0);
  if (c1) atomicAdd(a + 1, c1);
  if (c2) atomicAdd(a + 2, c2);
}

__device__ __forceinline__ void remove_q(unsigned long long* acc, long long j, double q) {
  if ((u64)__double_as_longlong(q) >= 0x47E0000000000000ull) return;  // never deposited
  u64 c0, c1, c2;
  q_parts(q, &c0, &c1, &c2);
  u64* a = acc + 4 * j;
  if (c0) atomicAdd(a + 0, (u64)(0ull - c0));
  if (c1) atomicAdd(a + 1, (u64)(0ull - c1));
  if (c2) atomicAdd(a + 2, (u64)(0ull - c2));
}

// Estimator input of bin j: P_j = S_j Q_j 2^-96, or x[j].
__device__ __forceinline__ double spec_value(const SpecIn& in, long long j) {
  if (in.acc) {
    const ulonglong2* a = reinterpret_cast<const ulonglong2*>(in.acc + 4 * j);
    ulonglong2 w01 = a[0];
    u64 w2 = in.acc[4 * j + 2];
    U128 Q = q_combine3(w01.x, w01.y, w2);
    return __dmul_rn(in.S[j], u128_to_dbl_scaled(Q, 96));
  }
  return in.x[j];
}

__global__ void k_power_out(const unsigned long long* __restrict__ acc, const double* __restrict__ S,
                            long long n, double* __restrict__ P) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  SpecIn in;
  in.acc = acc;
  in.S = S;
  in.x = nullptr;
  P[j] = spec_value(in, j);
}

void launch_power_out(const unsigned long long* acc, const double* S, long long n, double* P,
                      cudaStream_t st) {
  int th = 256;
  k_power_out<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(acc, S, n, P);
}

// ============================================================================ prepass

// FP64 path of the catalog pass: the sweep of one source, its pieces deposited; returns
// the sum of its contributions.  Kept out of line so that none of it is speculated into
// the common path.
__device__ __noinline__ double prepass_slow(double a2, double fs, double fds, const Grid g,
                                            const Tables tb, unsigned long long* acc,
                                            unsigned* err) {
  Sweep sw = make_sweep(fs, fds, g.T, g.T2);
  double r = 0.0;
  if (sw.ka == sw.kb) {
    long long j = sw.ka - g.k_lo;
    if (j >= 0 && j < g.nb) {
      double q = __dmul_rn(a2, tb.gq[j]);
      deposit_q(acc, j, q, err);
      r = q;
    }
  } else {
    long long k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
    long long k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
    for (long long k = k0; k <= k1; ++k) {
      double w = sweep_weight(sw, k);
      if (w > 0.0) {
        long long j = k - g.k_lo;
        double q = __dmul_rn(__dmul_rn(a2, w), tb.gq[j]);
        deposit_q(acc, j, q, err);
        r = __dadd_rn(r, q);
      }
    }
  }
  return r;
}

// Record of a kept candidate (rare; out of line).
__device__ __noinline__ void emit_candidate(Cands cd, long long c, long long s, double a2,
                                            double fs, double fds, const Grid g) {
  Sweep sw = make_sweep(fs, fds, g.T, g.T2);
  cd.src[c] = s;
  cd.ka[c] = (int)(sw.ka - g.k_lo);
  cd.nbin[c] = (int)(sw.kb - sw.ka + 1);
  cd.a2f[c] = dbl_to_f32_scaled(a2, 160);
  cd.flo[c] = (float)(sw.lo - (double)sw.ka);
  cd.len[c] = (float)(sw.hi - sw.lo);
  cd.a2[c] = a2;
  cd.lo[c] = sw.lo;
  cd.hi[c] = sw.hi;
  cd.res[c] = 0;
}

__global__ void __launch_bounds__(256) k_prepass(
    const double* __restrict__ A, const double* __restrict__ f, const double* __restrict__ fdot,
    long long N, Grid g, Tables tb, double thr_kappa, double thr_live,
    unsigned long long* __restrict__ acc, Cands cd, RunState* rs) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // thresholds on r >= 0 compared as the integer bits of non-negative doubles
  const u64 tk_bits = (u64)__double_as_longlong(thr_kappa);
  const u64 tl_bits = (u64)__double_as_longlong(thr_live);
  unsigned long long nkappa = 0;
  for (long long base = warp0; base < N; base += stride) {
    long long s = base + lane;
    bool live = false;
    double a2 = 0.0, fs = 0.0, fds = 0.0;
    if (s < N) {
      double a = A[s];
      fs = f[s];
      fds = fdot[s];
      a2 = __dmul_rn(a, a);
      // Common case without FP64: bin of f T + 1/2 exactly, and an FP32 bound on the sweep
      // fdot T^2 proving that f T + fdot T^2 + 1/2 stays in the same bin (the FP64 path
      // takes every case the bound cannot settle).
      long long k0;
      unsigned fr24;
      int fb;
      bool single = false;
      if (ft_bin(fs, g.mT, g.eT, &k0, &fr24, &fb)) {
        float du = __fmul_rn(dbl_to_f32_signed(fds), g.T2f);
        float phi = __fmul_rn((float)fr24, 5.9604644775390625e-8f);  // 2^-24
        float m = __fadd_rn(9.5367431640625e-7f, __fmul_rn(4e-7f, fabsf(du)));  // 2^-20 + ...
        float x = __fadd_rn(phi, du);
        single = (x >= m) && (x < __fsub_rn(1.0f, m));
      }
      double r = 0.0;  // sum of q: rho_0^2 = 4 r 2^-96
      if (single) {
        long long j = k0 - g.k_lo;
        if (j >= 0 && j < g.nb) {
          double q = __dmul_rn(a2, tb.gq[j]);
          deposit_q(acc, j, q, &rs->err);
          r = q;
        }
      } else {
        r = prepass_slow(a2, fs, fds, g, tb, acc, &rs->err);
      }
      u64 rb = (u64)__double_as_longlong(r);
      if (rb >= tk_bits) ++nkappa;
      live = (rb > tl_bits) && (rb >= tk_bits);
    }
    unsigned m = __ballot_sync(0xFFFFFFFFu, live);
    if (m) {
      unsigned long long b0 = 0;
      int leader = __ffs(m) - 1;
      if (lane == leader) b0 = atomicAdd(&rs->nlive, (unsigned long long)__popc(m));
      b0 = __shfl_sync(0xFFFFFFFFu, b0, leader);
      if (live) {
        long long c = (long long)b0 + __popc(m & ((1u << lane) - 1u));
        emit_candidate(cd, c, s, a2, fs, fds, g);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) nkappa += __shfl_xor_sync(0xFFFFFFFFu, nkappa, o);
  if (lane == 0 && nkappa) atomicAdd(&rs->ncand, nkappa);
}

void launch_prepass(const double* A, const double* f, const double* fdot, long long N,
                    const Grid& g, const Tables& tb, double thr_kappa, double thr_live,
                    unsigned long long* acc, Cands cd, RunState* rs, int nsm, cudaStream_t st) {
  if (N <= 0) return;
  int th = 256;
  long long want = (N + th - 1) / th;
  long long cap = (long long)nsm * 8;
  int bl = (int)(want < cap ? want : cap);
  k_prepass<<<bl, th, 0, st>>>(A, f, fdot, N, g, tb, thr_kappa, thr_live, acc, cd, rs);
}

// ============================================================================ reductions

__device__ __forceinline__ void warp_max_atomic(u64 v, u64* target) {
  // v are bits of non-negative doubles: their integer order is the value order.
  for (int o = 16; o > 0; o >>= 1) {
    u64 t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = t > v ? t : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(target, v);
}

__global__ void k_max_bits(const double* __restrict__ x, long long n, unsigned long long* max_bits) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  u64 b = 0;
  if (j < n) {
    b = (u64)__double_as_longlong(x[j]);
    if (b >> 63) b = 0ull;
  }
  warp_max_atomic(b, max_bits);
}

void launch_max_bits(const double* x, long long n, unsigned long long* max_bits, cudaStream_t st) {
  int th = 256;
  k_max_bits<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(x, n, max_bits);
}

// S_gal epilogue: store, fold the relative change of S_n for conv_rtol, and the FP32
// factor 1 / (1 + S_gal / S_instr) that the SNR screen multiplies rho_0^2 by.
__device__ __forceinline__ double sg_store(const SgOut& o, long long j, double v) {
  double rel = 0.0;
  if (o.rtol_on) {
    double a = __dadd_rn(o.S[j], v), b = __dadd_rn(o.S[j], o.out[j]);
    rel = fabs(__dsub_rn(a, b)) / a;
  }
  o.out[j] = v;
  if (o.inv_f) {
    float ratio = __fmul_rn(dbl_to_f32_scaled(v, 150), o.invSf[j]);
    o.inv_f[j] = __frcp_rn(__fadd_rn(1.0f, ratio));
  }
  return rel;
}

// ============================================================================ chunk sort
// Chunks of Kc >= W consecutive bins: any window of at most W bins lies in at most two
// consecutive chunks.  Each chunk is sorted once (keys: the bits of the non-negative
// doubles, whose integer order is their value order; ties broken by position), and
// for every kSnapStride-th position t the set of sorted indices whose position is >= t
// is stored as a bitset ("snapshot") so that a thread can build the active set of any
// window quickly.

__global__ void k_chunk_sort(SpecIn in, long long n, SmoothPlan pl,
                             unsigned long long* __restrict__ skey, uint16_t* __restrict__ srank,
                             uint32_t* __restrict__ snap, Dirty d) {
  extern __shared__ unsigned long long sm_keys[];
  uint16_t* sm_idx = (uint16_t*)(sm_keys + pl.kpad);
  const int b = blockIdx.x;
  if (!d.any(b, 0)) return;  // unchanged input: keys, ranks and snapshots still hold
  const long long base = (long long)b * pl.Kc;
  const int len = (int)((n - base) < pl.Kc ? (n - base) : pl.Kc);
  for (int i = threadIdx.x; i < pl.kpad; i += blockDim.x) {
    u64 k = ~0ull;
    if (i < len) {
      k = (u64)__double_as_longlong(spec_value(in, base + i));
      if (k >> 63) k = 0ull;  // -0.0 (or a negative value) sorts as zero
    }
    sm_keys[i] = k;
    sm_idx[i] = (uint16_t)i;
  }
  __syncthreads();
  // bitonic sort of (key, position)
  for (int kk = 2; kk <= pl.kpad; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < pl.kpad; i += blockDim.x) {
        int ixj = i ^ jj;
        if (ixj > i) {
          u64 ki = sm_keys[i], kj = sm_keys[ixj];
          uint16_t ii = sm_idx[i], ij = sm_idx[ixj];
          bool gt = (ki > kj) || (ki == kj && ii > ij);
          bool asc = ((i & kk) == 0);
          if (gt == asc) {
            sm_keys[i] = kj;
            sm_keys[ixj] = ki;
            sm_idx[i] = ij;
            sm_idx[ixj] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int s = threadIdx.x; s < len; s += blockDim.x) {
    skey[base + s] = sm_keys[s];
    srank[base + sm_idx[s]] = (uint16_t)s;
  }
  // snapshots: word w of snapshot m has bit i set iff sorted index 32w+i < len and its
  // position is >= m * kSnapStride.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int w = warp; w < pl.nw; w += nwarp) {
    int s = w * 32 + lane;
    int pos = (s < len) ? (int)sm_idx[s] : -1;
    uint32_t* dst = snap + (size_t)b * pl.nsnap * pl.nw + w;
    for (int m = 0; m < pl.nsnap; ++m) {
      unsigned bits = __ballot_sync(0xFFFFFFFFu, pos >= m * kSnapStride);
      if (lane == 0) dst[(size_t)m * pl.nw] = bits;
    }
  }
}

void launch_chunk_sort(SpecIn in, long long n, const SmoothPlan& pl, unsigned long long* skey,
                       uint16_t* srank, uint32_t* snap, Dirty d, cudaStream_t st) {
  size_t smem = (size_t)pl.kpad * (sizeof(u64) + sizeof(uint16_t));
  int th = pl.kpad >= 1024 ? 1024 : (pl.kpad < 64 ? 64 : pl.kpad);
  k_chunk_sort<<<pl.nch, th, smem, st>>>(in, n, pl, skey, srank, snap, d);
}

// ============================================================================ median slide
// Each thread produces L consecutive outputs.  The window of output j is
// [s(j), e(j)] = [max(0, j - W/2), min(n-1, j - W/2 + W - 1)] and lies in chunk A (the
// chunk of s(j)) and chunk B = A + 1.  The thread keeps, for A and B, a bitset over
// sorted indices marking the elements inside the window, and a "merge cut" (cA, cB):
// the first cA sorted elements of A and first cB of B are exactly the elements that
// precede the cut in the merged order of A and B (ties: A first, then by position).
// pc counts the active elements before the cut; it is kept at c/2 + 1 (c = window
// size), so the last active element before the cut is the upper median.  Sliding the
// window by one bin clears one bit and sets one bit, and moves the cut by O(1) active
// elements.  The initial cut comes from a binary search over the merged order.

struct SlideSide {
  const u64* key;        // sorted keys of the chunk
  const uint16_t* rank;  // position -> sorted index
  const uint32_t* snap;  // snapshots of the chunk
  uint32_t* bs;          // bitset words (strided)
  int len;               // elements in the chunk (0 if none)
  long long base;        // first bin of the chunk
};

__device__ __forceinline__ void side_bind(SlideSide& sd, const u64* skey, const uint16_t* srank,
                                          const uint32_t* snap, const SmoothPlan& pl, long long n,
                                          long long chunk) {
  sd.base = chunk * pl.Kc;
  long long rem = n - sd.base;
  sd.len = rem <= 0 ? 0 : (rem < pl.Kc ? (int)rem : pl.Kc);
  if (chunk >= pl.nch) chunk = pl.nch - 1;  // unused when len == 0
  sd.key = skey + chunk * (long long)pl.Kc;
  sd.rank = srank + chunk * (long long)pl.Kc;
  sd.snap = snap + chunk * (long long)pl.nsnap * pl.nw;
}

__device__ __forceinline__ void bs_set(uint32_t* bs, int stride, int s) {
  bs[(s >> 5) * stride] |= (1u << (s & 31));
}
__device__ __forceinline__ void bs_clear(uint32_t* bs, int stride, int s) {
  bs[(s >> 5) * stride] &= ~(1u << (s & 31));
}

// Active positions [p0, p1) of a chunk as a bitset over sorted indices.
__device__ void side_fill(SlideSide& sd, int stride, int nw, int p0, int p1) {
  if (sd.len == 0 || p1 <= p0) {
    for (int w = 0; w < nw; ++w) sd.bs[w * stride] = 0u;
    return;
  }
  int m0 = p0 / kSnapStride, m1 = p1 / kSnapStride;
  const uint32_t* s0 = sd.snap + (size_t)m0 * nw;
  const uint32_t* s1 = sd.snap + (size_t)m1 * nw;
  for (int w = 0; w < nw; ++w) sd.bs[w * stride] = __ldg(s0 + w) & ~__ldg(s1 + w);
  for (int p = m0 * kSnapStride; p < p0; ++p) bs_clear(sd.bs, stride, __ldg(sd.rank + p));
  int q0 = m1 * kSnapStride > p0 ? m1 * kSnapStride : p0;
  for (int p = q0; p < p1; ++p) bs_set(sd.bs, stride, __ldg(sd.rank + p));
}

__device__ __forceinline__ int popc_prefix(const uint32_t* bs, int stride, int c) {
  int r = 0;
  int w = c >> 5;
  for (int i = 0; i < w; ++i) r += __popc(bs[i * stride]);
  if (c & 31) r += __popc(bs[w * stride] & ((1u << (c & 31)) - 1u));
  return r;
}

// Number of A elements among the first P of the merged order.
__device__ __forceinline__ int merge_path(const SlideSide& A, const SlideSide& B, int P) {
  int lo = P - B.len > 0 ? P - B.len : 0;
  int hi = P < A.len ? P : A.len;
  while (lo < hi) {
    int x = (lo + hi + 1) >> 1;  // try taking x elements of A
    int y = P - x;
    bool ok = (y >= B.len) || (__ldg(A.key + x - 1) <= __ldg(B.key + y));
    if (ok) lo = x; else hi = x - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_median_slide(
    const unsigned long long* __restrict__ skey, const uint16_t* __restrict__ srank,
    const uint32_t* __restrict__ snap, long long n, SmoothPlan pl, SgOut o, Dirty d) {
  extern __shared__ uint32_t sm_bits[];
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  const int nw = pl.nw;
  uint32_t* bsX = sm_bits + tid;               // word w at bsX[w * T]
  uint32_t* bsY = sm_bits + (size_t)nw * T + tid;
  const long long g = blockIdx.x * (long long)T + tid;
  const long long j0 = g * pl.L;
  double relmax = 0.0;
  // the outputs of this thread lie in one chunk (L divides Kc); their windows read chunks
  // within one of it
  if (j0 < n && d.any(j0 / pl.Kc, 1)) {
    const long long j1 = (j0 + pl.L < n) ? j0 + pl.L : n;
    const int h = pl.W / 2;
    long long s_cur = j0 - h > 0 ? j0 - h : 0;
    long long e_cur = j0 - h + pl.W - 1 < n - 1 ? j0 - h + pl.W - 1 : n - 1;
    long long chA = s_cur / pl.Kc;
    SlideSide A, B;
    side_bind(A, skey, srank, snap, pl, n, chA);
    side_bind(B, skey, srank, snap, pl, n, chA + 1);
    A.bs = bsX;
    B.bs = bsY;
    {
      int pa0 = (int)(s_cur - A.base);
      long long ea = e_cur - A.base + 1;
      int pa1 = (int)(ea < A.len ? ea : A.len);
      side_fill(A, T, nw, pa0, pa1);
      long long eb = e_cur - B.base + 1;
      int pb1 = eb <= 0 ? 0 : (int)(eb < B.len ? eb : B.len);
      side_fill(B, T, nw, 0, pb1);
    }
    int c = (int)(e_cur - s_cur + 1);
    int kq = c / 2 + 1;
    // initial cut: smallest merged position with kq active elements before it
    int lo = kq, hi = A.len + B.len;
    while (lo < hi) {
      int P = (lo + hi) >> 1;
      int x = merge_path(A, B, P);
      int cnt = popc_prefix(A.bs, T, x) + popc_prefix(B.bs, T, P - x);
      if (cnt >= kq) hi = P; else lo = P + 1;
    }
    int cA = merge_path(A, B, lo);
    int cB = lo - cA;
    int pc = kq;

    for (long long j = j0; j < j1; ++j) {
      if (j > j0) {
        long long sj = j - h > 0 ? j - h : 0;
        long long ej = j - h + pl.W - 1 < n - 1 ? j - h + pl.W - 1 : n - 1;
        if (sj > s_cur) {
          int sx = __ldg(A.rank + (s_cur - A.base));
          bs_clear(A.bs, T, sx);
          --c;
          if (sx < cA) --pc;
          s_cur = sj;
          if (s_cur >= A.base + A.len && B.len > 0) {
            // chunk A is empty: B becomes A, the next chunk becomes B
            uint32_t* freed = A.bs;
            A = B;
            cA = cB;
            ++chA;
            side_bind(B, skey, srank, snap, pl, n, chA + 1);
            B.bs = freed;  // all zero: every element of the old A has left
            // cB = number of B elements preceding A[cA] (B after A on ties)
            int lo2 = 0, hi2 = B.len;
            if (cA < A.len) {
              u64 ka = __ldg(A.key + cA);
              while (lo2 < hi2) {
                int mid = (lo2 + hi2) >> 1;
                if (__ldg(B.key + mid) < ka) lo2 = mid + 1; else hi2 = mid;
              }
              cB = lo2;
            } else {
              cB = B.len;
            }
          }
        }
        if (ej > e_cur) {
          e_cur = ej;
          if (ej < A.base + A.len) {
            int sx = __ldg(A.rank + (ej - A.base));
            bs_set(A.bs, T, sx);
            ++c;
            if (sx < cA) ++pc;
          } else {
            int sx = __ldg(B.rank + (ej - B.base));
            bs_set(B.bs, T, sx);
            ++c;
            if (sx < cB) ++pc;
          }
        }
        kq = c / 2 + 1;
        while (pc < kq) {
          // advance over the next active element of the merged order
          int nA = bs_next(A.bs, T, nw, cA, A.len);
          int nB = bs_next(B.bs, T, nw, cB, B.len);
          bool takeA = (nB >= B.len) || (nA < A.len && __ldg(A.key + nA) <= __ldg(B.key + nB));
          if (takeA) {
            u64 ka = __ldg(A.key + nA);
            cA = nA + 1;
            while (cB < B.len && __ldg(B.key + cB) < ka) ++cB;
          } else {
            u64 kb = __ldg(B.key + nB);
            cB = nB + 1;
            while (cA < A.len && __ldg(A.key + cA) <= kb) ++cA;
          }
          ++pc;
        }
        while (pc > kq) {
          // retreat over the last active element before the cut
          int pA = bs_prev(A.bs, T, cA);
          int pB = bs_prev(B.bs, T, cB);
          bool takeB = (pA < 0) || (pB >= 0 && __ldg(B.key + pB) >= __ldg(A.key + pA));
          if (takeB) {
            u64 kb = __ldg(B.key + pB);
            cB = pB;
            while (cA > 0 && __ldg(A.key + cA - 1) > kb) --cA;
          } else {
            u64 ka = __ldg(A.key + pA);
            cA = pA;
            while (cB > 0 && __ldg(B.key + cB - 1) >= ka) --cB;
          }
          --pc;
        }
      }
      // the upper median is the last active element before the cut
      int pA = bs_prev(A.bs, T, cA);
      int pB = bs_prev(B.bs, T, cB);
      u64 khi, klo = 0;
      bool hiB = (pA < 0) || (pB >= 0 && __ldg(B.key + pB) >= __ldg(A.key + pA));
      if (hiB) khi = __ldg(B.key + pB); else khi = __ldg(A.key + pA);
      double med;
      if (c & 1) {
        med = __longlong_as_double((i64)khi);
      } else {
        // lower median: the larger of the other side's last active and this side's previous
        int q1, q2;
        u64 k1 = 0, k2 = 0;
        bool h1 = false, h2 = false;
        if (hiB) {
          q1 = pA;
          q2 = bs_prev(B.bs, T, pB);
          if (q1 >= 0) { k1 = __ldg(A.key + q1); h1 = true; }
          if (q2 >= 0) { k2 = __ldg(B.key + q2); h2 = true; }
        } else {
          q1 = pB;
          q2 = bs_prev(A.bs, T, pA);
          if (q1 >= 0) { k1 = __ldg(B.key + q1); h1 = true; }
          if (q2 >= 0) { k2 = __ldg(A.key + q2); h2 = true; }
        }
        klo = (h1 && h2) ? (k1 > k2 ? k1 : k2) : (h1 ? k1 : k2);
        med = __dmul_rn(__dadd_rn(__longlong_as_double((i64)klo), __longlong_as_double((i64)khi)),
                        0.5);
      }
      double v = __dmul_rn(kMedianBias, med);
      double rel = sg_store(o, j, v);
      relmax = rel > relmax ? rel : relmax;
    }
  }
  if (o.rtol_on) warp_max_atomic((u64)__double_as_longlong(relmax), &o.rs->relchg_bits);
}

// Same algorithm with the sorted keys and ranks of the three chunks a window of output
// chunk c can touch (c-1, c, c+1) staged in shared memory: one CTA per output chunk, so
// the dependent loads of each thread's merge-cut walk hit shared memory.  Snapshots are
// read from global memory (a few independent loads per thread at set-up).
__global__ void __launch_bounds__(256) k_median_slide_smem(
    const unsigned long long* __restrict__ skey, const uint16_t* __restrict__ srank,
    const uint32_t* __restrict__ snap, long long n, SmoothPlan pl, SgOut o, Dirty d) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  const int nw = pl.nw;
  const int Kc = pl.Kc;
  const long long c = blockIdx.x;
  if (!d.any(c, 1)) return;  // no window of this chunk changed
  u64* sk = (u64*)sm_raw;                                   // [3][Kc]
  uint16_t* sr = (uint16_t*)(sk + 3 * (size_t)Kc);          // [3][Kc]
  uint32_t* sb = (uint32_t*)(sr + 3 * (size_t)Kc);          // [2][nw][T]
  uint16_t* sp = (uint16_t*)(sb + 2 * (size_t)nw * T);      // [2][nw + 1][T] word prefixes
  const long long c0 = c - 1;  // chunk held in slot 0
  for (int slot = 0; slot < 3; ++slot) {
    long long ch = c0 + slot;
    if (ch < 0 || ch >= pl.nch) continue;
    long long base = ch * (long long)Kc;
    int len = (int)((n - base) < Kc ? (n - base) : Kc);
    const ulonglong2* gk = reinterpret_cast<const ulonglong2*>(skey + base);
    ulonglong2* dk = reinterpret_cast<ulonglong2*>(sk + (size_t)slot * Kc);
    for (int i = tid; i < (len + 1) / 2; i += T) dk[i] = gk[i];
    for (int i = tid; i < len; i += T) sr[(size_t)slot * Kc + i] = srank[base + i];
  }
  __syncthreads();
  uint32_t* bsX = sb + tid;
  uint32_t* bsY = sb + (size_t)nw * T + tid;
  const long long j0 = c * Kc + (long long)tid * pl.L;
  double relmax = 0.0;
  if (j0 < n) {
    long long jend = (c + 1) * (long long)Kc;
    long long j1 = j0 + pl.L < jend ? j0 + pl.L : jend;
    if (j1 > n) j1 = n;
    const int h = pl.W / 2;
    long long s_cur = j0 - h > 0 ? j0 - h : 0;
    long long e_cur = j0 - h + pl.W - 1 < n - 1 ? j0 - h + pl.W - 1 : n - 1;
    long long chA = s_cur / Kc;
    auto bind = [&](SlideSide& sd, long long ch) {
      sd.base = ch * Kc;
      long long rem = n - sd.base;
      sd.len = rem <= 0 ? 0 : (rem < Kc ? (int)rem : Kc);
      long long slot = ch - c0;
      if (slot < 0) slot = 0;
      if (slot > 2) slot = 2;
      sd.key = sk + slot * Kc;
      sd.rank = sr + slot * Kc;
      long long chs = ch < pl.nch ? ch : pl.nch - 1;
      sd.snap = snap + chs * (long long)pl.nsnap * nw;
    };
    SlideSide A, B;
    bind(A, chA);
    bind(B, chA + 1);
    A.bs = bsX;
    B.bs = bsY;
    {
      int pa0 = (int)(s_cur - A.base);
      long long ea = e_cur - A.base + 1;
      int pa1 = (int)(ea < A.len ? ea : A.len);
      int m0 = pa0 / kSnapStride, m1 = pa1 / kSnapStride;
      if (A.len == 0 || pa1 <= pa0) {
        for (int w = 0; w < nw; ++w) A.bs[w * T] = 0u;
      } else {
        const uint32_t* s0 = A.snap + (size_t)m0 * nw;
        const uint32_t* s1 = A.snap + (size_t)m1 * nw;
        for (int w = 0; w < nw; ++w) A.bs[w * T] = __ldg(s0 + w) & ~__ldg(s1 + w);
        for (int p = m0 * kSnapStride; p < pa0; ++p) bs_clear(A.bs, T, A.rank[p]);
        int q0 = m1 * kSnapStride > pa0 ? m1 * kSnapStride : pa0;
        for (int p = q0; p < pa1; ++p) bs_set(A.bs, T, A.rank[p]);
      }
      long long eb = e_cur - B.base + 1;
      int pb1 = eb <= 0 ? 0 : (int)(eb < B.len ? eb : B.len);
      if (B.len == 0 || pb1 <= 0) {
        for (int w = 0; w < nw; ++w) B.bs[w * T] = 0u;
      } else {
        int mb = pb1 / kSnapStride;
        const uint32_t* s0 = B.snap;
        const uint32_t* s1 = B.snap + (size_t)mb * nw;
        for (int w = 0; w < nw; ++w) B.bs[w * T] = __ldg(s0 + w) & ~__ldg(s1 + w);
        for (int p = mb * kSnapStride; p < pb1; ++p) bs_set(B.bs, T, B.rank[p]);
      }
    }
    int cnt = (int)(e_cur - s_cur + 1);
    int kq = cnt / 2 + 1;
    // word prefixes of the active counts (valid until the first slide step), so that the
    // count of active elements below a sorted index is one lookup and one popcount
    uint16_t* pA = sp + tid;
    uint16_t* pB = sp + (size_t)(nw + 1) * T + tid;
    {
      int ra = 0, rb = 0;
      for (int w = 0; w < nw; ++w) {
        pA[w * T] = (uint16_t)ra;
        pB[w * T] = (uint16_t)rb;
        ra += __popc(A.bs[w * T]);
        rb += __popc(B.bs[w * T]);
      }
      pA[nw * T] = (uint16_t)ra;
      pB[nw * T] = (uint16_t)rb;
    }
    auto cnt_below = [&](const uint32_t* bs, const uint16_t* pf, int x) {
      int w = x >> 5;
      int r = pf[w * T];
      if (x & 31) r += __popc(bs[w * T] & ((1u << (x & 31)) - 1u));
      return r;
    };
    // initial cut: smallest merged position with kq active elements before it
    int lo = kq, hi = A.len + B.len;
    while (lo < hi) {
      int P = (lo + hi) >> 1;
      int lo2 = P - B.len > 0 ? P - B.len : 0, hi2 = P < A.len ? P : A.len;
      while (lo2 < hi2) {
        int x = (lo2 + hi2 + 1) >> 1;
        int y = P - x;
        bool ok = (y >= B.len) || (A.key[x - 1] <= B.key[y]);
        if (ok) lo2 = x; else hi2 = x - 1;
      }
      int k2 = cnt_below(A.bs, pA, lo2) + cnt_below(B.bs, pB, P - lo2);
      if (k2 >= kq) hi = P; else lo = P + 1;
    }
    int cA, cB;
    {
      int P = lo;
      int lo2 = P - B.len > 0 ? P - B.len : 0, hi2 = P < A.len ? P : A.len;
      while (lo2 < hi2) {
        int x = (lo2 + hi2 + 1) >> 1;
        int y = P - x;
        bool ok = (y >= B.len) || (A.key[x - 1] <= B.key[y]);
        if (ok) lo2 = x; else hi2 = x - 1;
      }
      cA = lo2;
      cB = P - lo2;
    }
    int pc = kq;
    for (long long j = j0; j < j1; ++j) {
      if (j > j0) {
        long long sj = j - h > 0 ? j - h : 0;
        long long ej = j - h + pl.W - 1 < n - 1 ? j - h + pl.W - 1 : n - 1;
        if (sj > s_cur) {
          int sx = A.rank[s_cur - A.base];
          bs_clear(A.bs, T, sx);
          --cnt;
          if (sx < cA) --pc;
          s_cur = sj;
          if (s_cur >= A.base + A.len && B.len > 0) {
            uint32_t* freed = A.bs;
            A = B;
            cA = cB;
            ++chA;
            bind(B, chA + 1);
            B.bs = freed;
            if (cA < A.len) {
              u64 ka = A.key[cA];
              int lo3 = 0, hi3 = B.len;
              while (lo3 < hi3) {
                int mid = (lo3 + hi3) >> 1;
                if (B.key[mid] < ka) lo3 = mid + 1; else hi3 = mid;
              }
              cB = lo3;
            } else {
              cB = B.len;
            }
          }
        }
        if (ej > e_cur) {
          e_cur = ej;
          if (ej < A.base + A.len) {
            int sx = A.rank[ej - A.base];
            bs_set(A.bs, T, sx);
            ++cnt;
            if (sx < cA) ++pc;
          } else {
            int sx = B.rank[ej - B.base];
            bs_set(B.bs, T, sx);
            ++cnt;
            if (sx < cB) ++pc;
          }
        }
        kq = cnt / 2 + 1;
        while (pc < kq) {
          int nA = bs_next(A.bs, T, nw, cA, A.len);
          int nB = bs_next(B.bs, T, nw, cB, B.len);
          bool takeA = (nB >= B.len) || (nA < A.len && A.key[nA] <= B.key[nB]);
          if (takeA) {
            u64 ka = A.key[nA];
            cA = nA + 1;
            while (cB < B.len && B.key[cB] < ka) ++cB;
          } else {
            u64 kb = B.key[nB];
            cB = nB + 1;
            while (cA < A.len && A.key[cA] <= kb) ++cA;
          }
          ++pc;
        }
        while (pc > kq) {
          int pA = bs_prev(A.bs, T, cA);
          int pB = bs_prev(B.bs, T, cB);
          bool takeB = (pA < 0) || (pB >= 0 && B.key[pB] >= A.key[pA]);
          if (takeB) {
            u64 kb = B.key[pB];
            cB = pB;
            while (cA > 0 && A.key[cA - 1] > kb) --cA;
          } else {
            u64 ka = A.key[pA];
            cA = pA;
            while (cB > 0 && B.key[cB - 1] >= ka) --cB;
          }
          --pc;
        }
      }
      int pA = bs_prev(A.bs, T, cA);
      int pB = bs_prev(B.bs, T, cB);
      bool hiB = (pA < 0) || (pB >= 0 && B.key[pB] >= A.key[pA]);
      u64 khi = hiB ? B.key[pB] : A.key[pA];
      double med;
      if (cnt & 1) {
        med = __longlong_as_double((i64)khi);
      } else {
        int q1, q2;
        u64 k1 = 0, k2 = 0;
        bool h1 = false, h2 = false;
        if (hiB) {
          q1 = pA;
          q2 = bs_prev(B.bs, T, pB);
          if (q1 >= 0) { k1 = A.key[q1]; h1 = true; }
          if (q2 >= 0) { k2 = B.key[q2]; h2 = true; }
        } else {
          q1 = pB;
          q2 = bs_prev(A.bs, T, pA);
          if (q1 >= 0) { k1 = B.key[q1]; h1 = true; }
          if (q2 >= 0) { k2 = A.key[q2]; h2 = true; }
        }
        u64 klo = (h1 && h2) ? (k1 > k2 ? k1 : k2) : (h1 ? k1 : k2);
        med = __dmul_rn(__dadd_rn(__longlong_as_double((i64)klo), __longlong_as_double((i64)khi)),
                        0.5);
      }
      double v = __dmul_rn(kMedianBias, med);
      double rel = sg_store(o, j, v);
      relmax = rel > relmax ? rel : relmax;
    }
  }
  if (o.rtol_on) warp_max_atomic((u64)__double_as_longlong(relmax), &o.rs->relchg_bits);
}

// Threads per chunk for the shared-memory slide (each takes Kc / T consecutive outputs:
// short chains of dependent steps), and its shared-memory size.
static int smem_slide_threads(const SmoothPlan& pl) {
  int t = pl.Kc / 8;
  if (t < 32) t = 32;
  if (t > 128) t = 128;
  return t;
}
static size_t smem_slide_bytes(const SmoothPlan& pl, int T) {
  return (size_t)3 * pl.Kc * (sizeof(u64) + sizeof(uint16_t)) + (size_t)2 * pl.nw * T * 4 +
         (size_t)2 * (pl.nw + 1) * T * 2;
}

void launch_median_slide(const unsigned long long* skey, const uint16_t* srank,
                         const uint32_t* snap, long long n, const SmoothPlan& pl, SgOut o,
                         Dirty d, cudaStream_t st) {
  int ts = smem_slide_threads(pl);
  size_t ss = smem_slide_bytes(pl, ts);
  if (ss <= 160 * 1024) {
    SmoothPlan p2 = pl;
    p2.L = (pl.Kc + ts - 1) / ts;
    k_median_slide_smem<<<pl.nch, ts, ss, st>>>(skey, srank, snap, n, p2, o, d);
    return;
  }
  int th = pl.slide_threads;
  long long threads = (n + pl.L - 1) / pl.L;
  long long bl = (threads + th - 1) / th;
  size_t smem = (size_t)2 * pl.nw * th * sizeof(uint32_t);
  k_median_slide<<<(unsigned)bl, th, smem, st>>>(skey, srank, snap, n, pl, o, d);
}

// ============================================================================ window mean
// Exact window sums: inside chunk b every value becomes a 128-bit integer number of units
// 2^-sig[b], sig[b] chosen from the chunk's maximum so that a sum over the chunk fits;
// each chunk stores its inclusive prefix sums.  A window (at most two chunks) is one
// difference of prefixes per chunk, each converted to double once, so there is no
// cancellation however large the dynamic range of the spectrum.

__device__ __forceinline__ int sigma_from_max(u64 maxbits) {
  // max < 2^(e - 1022) with e the biased exponent; Kc <= 2^13 terms stay below 2^127.
  int e = (int)((maxbits >> 52) & 0x7FF);
  if (e == 0) e = 1;
  return 1136 - e;
}

__global__ void k_chunk_prefix(SpecIn in, long long n, SmoothPlan pl,
                               unsigned long long* __restrict__ pre_lo,
                               unsigned long long* __restrict__ pre_hi, int* __restrict__ sig,
                               unsigned* __restrict__ uflow, double* __restrict__ x_out, Dirty d,
                               int in_radius) {
  __shared__ U128 warp_tot[32];
  __shared__ u64 warp_max[32];
  __shared__ int any_uf;
  const int b = blockIdx.x;
  if (!d.any(b, in_radius)) return;  // unchanged input: prefix sums still hold
  const long long base = (long long)b * pl.Kc;
  const int len = (int)((n - base) < pl.Kc ? (n - base) : pl.Kc);
  const int per = (pl.Kc + blockDim.x - 1) / blockDim.x;
  const int p0 = threadIdx.x * per;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // pass 1: values and the chunk maximum
  double v[8];  // per <= 8 (Kc <= 8192 with 1024 threads)
  u64 mb = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < per) {
      int p = p0 + i;
      double x = 0.0;
      if (p < len) {
        x = spec_value(in, base + p);
        if (x_out) x_out[base + p] = x;
      }
      v[i] = x;
      u64 bits = (u64)__double_as_longlong(x);
      if (!(bits >> 63) && bits > mb) mb = bits;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    u64 t = __shfl_xor_sync(0xFFFFFFFFu, mb, o);
    mb = t > mb ? t : mb;
  }
  if (lane == 0) warp_max[warp] = mb;
  if (threadIdx.x == 0) any_uf = 0;
  __syncthreads();
  if (threadIdx.x < 32) {
    u64 t = threadIdx.x < nwarp ? warp_max[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      u64 u = __shfl_xor_sync(0xFFFFFFFFu, t, o);
      t = u > t ? u : t;
    }
    if (threadIdx.x == 0) warp_max[0] = t;
  }
  __syncthreads();
  const int sigma = sigma_from_max(warp_max[0]);
  // pass 2: thread totals in fixed point; note inputs > 0 below one unit
  U128 run{0ull, 0ull};
  int uf = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < per && p0 + i < len) {
      U128 q = dbl_to_u128_scaled(v[i], sigma);
      if (v[i] > 0.0 && u128_is_zero(q)) uf = 1;
      run = u128_add(run, q);
    }
  }
  if (uf) any_uf = 1;
  // exclusive scan of thread totals
  U128 inc = run;
  for (int o = 1; o < 32; o <<= 1) {
    U128 t;
    t.lo = __shfl_up_sync(0xFFFFFFFFu, inc.lo, o);
    t.hi = __shfl_up_sync(0xFFFFFFFFu, inc.hi, o);
    if (lane >= o) inc = u128_add(inc, t);
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    U128 t2 = lane < nwarp ? warp_tot[lane] : U128{0ull, 0ull};
    for (int o = 1; o < 32; o <<= 1) {
      U128 t;
      t.lo = __shfl_up_sync(0xFFFFFFFFu, t2.lo, o);
      t.hi = __shfl_up_sync(0xFFFFFFFFu, t2.hi, o);
      if (lane >= o) t2 = u128_add(t2, t);
    }
    if (lane < nwarp) warp_tot[lane] = t2;  // inclusive over warps
  }
  __syncthreads();
  U128 offs = u128_sub(inc, run);  // exclusive within warp
  if (warp > 0) offs = u128_add(offs, warp_tot[warp - 1]);
  // pass 3: write inclusive prefixes
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < per && p0 + i < len) {
      offs = u128_add(offs, dbl_to_u128_scaled(v[i], sigma));
      pre_lo[base + p0 + i] = offs.lo;
      pre_hi[base + p0 + i] = offs.hi;
    }
  }
  if (threadIdx.x == 0) {
    uflow[b] = (unsigned)any_uf;
    sig[b] = sigma;
  }
}

void launch_chunk_prefix(SpecIn in, long long n, const SmoothPlan& pl, unsigned long long* pre_lo,
                         unsigned long long* pre_hi, int* sig, unsigned* uflow, double* x_out,
                         Dirty d, int in_radius, cudaStream_t st) {
  int th = pl.Kc < 1024 ? pl.Kc : 1024;  // at most 8 values per thread
  k_chunk_prefix<<<pl.nch, th, 0, st>>>(in, n, pl, pre_lo, pre_hi, sig, uflow, x_out, d,
                                        in_radius);
}

// Sum of x[a .. e] inside one chunk as a double (a, e in the chunk, a <= e).
__device__ __forceinline__ double part_sum(const double* __restrict__ x, long long cbase, long long a,
                                           long long e, const unsigned long long* __restrict__ pre_lo,
                                           const unsigned long long* __restrict__ pre_hi, int sigma,
                                           unsigned uf) {
  U128 pe{pre_lo[e], pre_hi[e]};
  U128 sum = pe;
  if (a > cbase) sum = u128_sub(pe, U128{pre_lo[a - 1], pre_hi[a - 1]});
  long long cnt = e - a + 1;
  // Each input lost less than one unit; if the sum holds fewer than cnt * 2^40 units the
  // relative error could exceed 2^-40, so add the doubles directly instead.  A zero sum
  // is exact only if no input of the chunk fell below one unit.
  if (u128_is_zero(sum) && !uf) return 0.0;
  bool small = (sum.hi == 0ull) && (sum.lo < ((unsigned long long)cnt << 40));
  if (small) {
    double acc = 0.0;
    for (long long i = a; i <= e; ++i) acc = __dadd_rn(acc, x[i]);
    return acc;
  }
  return u128_to_dbl_scaled(sum, sigma);
}

__global__ void k_window_mean(const double* __restrict__ x, long long n, SmoothPlan pl,
                              const unsigned long long* __restrict__ pre_lo,
                              const unsigned long long* __restrict__ pre_hi,
                              const int* __restrict__ sig, const unsigned* __restrict__ uflow,
                              SgOut o, Dirty d, int out_radius) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double relmax = 0.0;
  if (j < n && d.any(j / pl.Kc, out_radius)) {
    const int h = pl.W / 2;
    long long s = j - h > 0 ? j - h : 0;
    long long e = j - h + pl.W - 1 < n - 1 ? j - h + pl.W - 1 : n - 1;
    long long cs = s / pl.Kc, ce = e / pl.Kc;
    long long cnt = e - s + 1;
    double sum;
    if (cs == ce) {
      sum = part_sum(x, cs * pl.Kc, s, e, pre_lo, pre_hi, sig[cs], uflow[cs]);
    } else {
      long long last = cs * pl.Kc + pl.Kc - 1;
      double s1 = part_sum(x, cs * pl.Kc, s, last, pre_lo, pre_hi, sig[cs], uflow[cs]);
      double s2 = part_sum(x, ce * pl.Kc, ce * pl.Kc, e, pre_lo, pre_hi, sig[ce], uflow[ce]);
      sum = __dadd_rn(s1, s2);
    }
    double v = (cnt == pl.W) ? __dmul_rn(sum, 1.0 / (double)pl.W) : __ddiv_rn(sum, (double)cnt);
    relmax = sg_store(o, j, v);
  }
  if (o.rtol_on) warp_max_atomic((u64)__double_as_longlong(relmax), &o.rs->relchg_bits);
}

void launch_window_mean(const double* x, long long n, const SmoothPlan& pl,
                        const unsigned long long* pre_lo, const unsigned long long* pre_hi,
                        const int* sig, const unsigned* uflow, SgOut o, Dirty d, int out_radius,
                        cudaStream_t st) {
  int th = 256;
  k_window_mean<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(x, n, pl, pre_lo, pre_hi, sig, uflow,
                                                               o, d, out_radius);
}

// ============================================================================ SNR + resolve
// rho^2 = 4 (T/5) A^2 sum_k w_k R_k / (S_k + S_gal,k) = sum_k rho0_k / (1 + S_gal,k / S_k).
// The screen evaluates it in FP32 as sum_k a2f w_k Gf_k inv_f_k; its relative error is
// below 2.2e-6 + 2e-7 per bin (FP32 roundings of the inputs, the ratio, the reciprocal,
// the products and the sum of positive terms), so outside a margin of 1e-5 + 4e-7 per
// bin around rho_th^2 the FP64 decision is known.  Inside it, and always when the
// caller asks for the strict path, rho^2 is recomputed in FP64 exactly as the oracle
// does.  In the mixed-precision mode the FP32 value decides alone.

__device__ __forceinline__ bool rtol_stop(const RunState* rs, double rtol) {
  if (!(rtol > 0.0) || rs->iter < 1) return false;
  double r = __longlong_as_double((i64)rs->relchg_bits);
  return r <= rtol;
}

__device__ double rho2_exact(const Grid& g, const Tables& tb, const double* __restrict__ Sg,
                             double a2, double lo, double hi) {
  Sweep sw;
  sw.lo = lo;
  sw.hi = hi;
  sw.ka = (i64)floor(__dadd_rn(lo, 0.5));
  sw.kb = (i64)floor(__dadd_rn(hi, 0.5));
  bool single = (sw.ka == sw.kb);
  long long k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
  long long k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
  double acc = 0.0;
  for (long long k = k0; k <= k1; ++k) {
    double w = single ? 1.0 : sweep_weight(sw, k);
    if (w > 0.0) {
      long long j = k - g.k_lo;
      double sn = __dadd_rn(tb.S[j], Sg[j]);
      double psk = __dmul_rn(__dmul_rn(__dmul_rn(g.t5, tb.R[j]), a2), w);
      acc = __dadd_rn(acc, __ddiv_rn(psk, sn));
    }
  }
  return __dmul_rn(4.0, acc);
}

__global__ void __launch_bounds__(256) k_snr_resolve(
    Cands cd, Grid g, Tables tb, const double* __restrict__ Sg, const float* __restrict__ inv_f,
    double th2, double rtol, int mode, unsigned char* __restrict__ resolved,
    unsigned long long* __restrict__ acc, RunState* rs, Dirty d, int Kc, int sg_radius) {
  if (rs->final_pass || rtol_stop(rs, rtol)) return;
  const long long nlive = (long long)rs->nlive;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const float th2f = (float)th2;
  unsigned local_new = 0, local_exact = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nlive; c += stride) {
    if (cd.res[c]) continue;
    const int ka = cd.ka[c];
    const int nbin = cd.nbin[c];
    {
      // S_n unchanged on every bin of the sweep: rho is the value already found below rho_th
      long long c0 = ka < 0 ? 0 : ka / Kc;
      long long kl = (long long)ka + nbin - 1;
      if (kl > g.nb - 1) kl = g.nb - 1;
      if (kl < 0) continue;
      long long c1 = kl / Kc;
      bool changed = false;
      for (long long cc = c0; cc <= c1 && !changed; ++cc) changed = d.any(cc, sg_radius);
      if (!changed) continue;
    }
    const float a2f = cd.a2f[c];
    float r2 = 0.0f;
    int kcount = 0;
    if (nbin == 1) {
      if (ka >= 0 && ka < g.nb) {
        r2 = __fmul_rn(__fmul_rn(a2f, tb.Gf[ka]), inv_f[ka]);
        kcount = 1;
      }
    } else {
      const float flo = cd.flo[c], fhi = __fadd_rn(flo, cd.len[c]), invlen = 1.0f / cd.len[c];
      int t0 = ka < 0 ? -ka : 0;
      int t1 = (long long)ka + nbin > g.nb ? (int)(g.nb - ka) : nbin;
      for (int t = t0; t < t1; ++t) {
        float a = fmaxf(flo, (float)t - 0.5f);
        float b = fminf(fhi, (float)t + 0.5f);
        if (b > a) {
          float w = __fmul_rn(__fsub_rn(b, a), invlen);
          int k = ka + t;
          r2 = __fadd_rn(r2, __fmul_rn(__fmul_rn(__fmul_rn(a2f, w), tb.Gf[k]), inv_f[k]));
          ++kcount;
        }
      }
    }
    bool resolve;
    if (mode == 1) {
      resolve = r2 > th2f;
    } else {
      float m = 1e-5f + 4e-7f * (float)kcount;
      if (mode == 0 && r2 > th2f * (1.0f + m)) {
        resolve = true;
      } else if (mode == 0 && r2 < th2f * (1.0f - m)) {
        resolve = false;
      } else {
        ++local_exact;
        resolve = rho2_exact(g, tb, Sg, cd.a2[c], cd.lo[c], cd.hi[c]) > th2;
      }
    }
    if (resolve) {
      cd.res[c] = 1;
      resolved[cd.src[c]] = 1;
      ++local_new;
      // remove exactly the parts the prepass deposited
      Sweep sw;
      sw.lo = cd.lo[c];
      sw.hi = cd.hi[c];
      sw.ka = (i64)floor(__dadd_rn(sw.lo, 0.5));
      sw.kb = (i64)floor(__dadd_rn(sw.hi, 0.5));
      double a2 = cd.a2[c];
      if (sw.ka == sw.kb) {
        long long j = sw.ka - g.k_lo;
        if (j >= 0 && j < g.nb) {
          remove_q(acc, j, __dmul_rn(a2, tb.gq[j]));
          d.mark_next(j / Kc);
        }
      } else {
        long long k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
        long long k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
        for (long long k = k0; k <= k1; ++k) {
          double w = sweep_weight(sw, k);
          if (w > 0.0) {
            long long j = k - g.k_lo;
            remove_q(acc, j, __dmul_rn(__dmul_rn(a2, w), tb.gq[j]));
            d.mark_next(j / Kc);
          }
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    local_new += __shfl_xor_sync(0xFFFFFFFFu, local_new, o);
    local_exact += __shfl_xor_sync(0xFFFFFFFFu, local_exact, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (local_new) atomicAdd(&rs->count_new, (unsigned long long)local_new);
    if (local_exact) atomicAdd(&rs->nexact, (unsigned long long)local_exact);
  }
}

void launch_snr_resolve(Cands cd, long long ncap, const Grid& g, const Tables& tb,
                        const double* Sg, const float* inv_f, double th2, double rtol, int mode,
                        unsigned char* resolved, unsigned long long* acc, RunState* rs,
                        Dirty d, int Kc, int sg_radius, int nsm, cudaStream_t st) {
  int th = 256;
  long long want = (ncap + th - 1) / th;
  long long cap = (long long)nsm * 8;
  int bl = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  k_snr_resolve<<<bl, th, 0, st>>>(cd, g, tb, Sg, inv_f, th2, rtol, mode, resolved, acc, rs, d, Kc,
                                   sg_radius);
}

// ============================================================================ loop control

__global__ void k_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                          unsigned long long cond_handle, int use_cond, unsigned char* dirty,
                          int nch) {
  // every thread clears part of the dirty set this iteration read (rs->iter still holds
  // the previous count); the new set was marked by this iteration's removals
  if (dirty) {
    unsigned char* cur = dirty + (size_t)(rs->iter & 1) * nch;
    for (int i = threadIdx.x; i < nch; i += blockDim.x) cur[i] = 0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned go = 1u;
  if (rs->final_pass) {
    go = 0u;
  } else {
    bool rstop = rtol_stop(rs, rtol);
    int it = rs->iter + 1;
    rs->iter = it;
    unsigned long long nn = rs->count_new;
    if (new_hist && it <= max_iter) new_hist[it - 1] = (int)nn;
    rs->nres += nn;
    if (rstop || nn == 0ull) {
      rs->converged = 1;
      go = 0u;
    } else if (it >= max_iter) {
      rs->final_pass = 1;  // one more estimate of S_gal from the final resolved set
      go = 1u;
    }
  }
  rs->count_new = 0ull;
  rs->relchg_bits = 0ull;
  if (!go) rs->stopped = 1;
  if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, go);
}

void launch_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                    unsigned long long cond_handle, int use_cond, unsigned char* dirty, int nch,
                    cudaStream_t st) {
  k_control<<<1, 256, 0, st>>>(rs, max_iter, rtol, new_hist, cond_handle, use_cond, dirty, nch);
}

void configure_kernels() {
  cudaFuncSetAttribute(k_chunk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  cudaFuncSetAttribute(k_median_slide, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(k_median_slide_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
}

}  // namespace gbsub
