// CUDA kernels of the iterative galactic-binary subtraction (arXiv 2602.18560, App. D),
// written for sm_103a (GB300).
//
// Steps of one run:
//   tables   : S_instr(f_k) (App. C, SciRDv1 A channel, TDI-2 factor), R(f_k) (App. B)
//              and the fixed-point scale of each bin.                       [once per context]
//   prepass  : one pass over the catalog: the bins each chirp sweeps, its power deposited
//              into an exact fixed-point spectrum, rho_0 against S_instr, candidates
//              rho_0 >= kappa rho_th compacted.                            [once per run]
//   loop     : P_k = S_k Q_k 2^-64; S_gal = estimator of P (running mean / running median /
//              median then mean, Eqs. running mean, running median); rho of each unresolved
//              candidate against S_instr + S_gal (Eqs. SNR inner product, inner product);
//              sources with rho > rho_th removed from the spectrum exactly; loop control on
//              the device.
//
// No floating-point atomics: the spectrum is an integer (units of 2^-64 S_instr,k per bin),
// so deposits and removals commute and every run gives the same bits.

#include <cuda_runtime.h>
#include <cuda_device_runtime_api.h>

#include "common.cuh"
#include "kernels.cuh"

namespace gbsub {

// ============================================================================ tables

__global__ void k_tables(Grid g, int tdi2, double* __restrict__ S, double* __restrict__ R,
                         double* __restrict__ gq) {
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
  // q = A^2 w * gq_k is the contribution in units of 2^-64 S_instr,k:
  // P / S = (T/5) R A^2 w / S.
  gq[j] = kQScale * (g.t5 * resp / s_aa);
}

void launch_tables(const Grid& g, int tdi2, double* S, double* R, double* gq, cudaStream_t st) {
  int th = 256;
  long long bl = (g.nb + th - 1) / th;
  k_tables<<<(unsigned)bl, th, 0, st>>>(g, tdi2, S, R, gq);
}

// ============================================================================ prepass

__device__ __forceinline__ void deposit_q(unsigned long long* acc_lo, unsigned long long* acc_hi,
                                          long long j, double q, unsigned* err) {
  if (!(q < kQLimit)) {
    atomicOr(err, ERR_RANGE);
    return;
  }
  u64 lo, hi;
  q_split(q, &lo, &hi);
  if (lo) atomicAdd(acc_lo + j, lo);
  if (hi) atomicAdd(acc_hi + j, hi);
}

__global__ void __launch_bounds__(256) k_prepass(
    const double* __restrict__ A, const double* __restrict__ f, const double* __restrict__ fdot,
    long long N, Grid g, const double* __restrict__ gq, double thr_q,
    unsigned long long* __restrict__ acc_lo, unsigned long long* __restrict__ acc_hi,
    Cand* __restrict__ cand, RunState* rs) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = warp0; base < N; base += stride) {
    long long s = base + lane;
    bool is_cand = false;
    Cand rec;
    if (s < N) {
      double a = A[s];
      Sweep sw = make_sweep(f[s], fdot[s], g.T, g.T2);
      double a2 = __dmul_rn(a, a);
      double r = 0.0;  // sum of q: rho_0^2 = 4 r 2^-64
      if (sw.ka == sw.kb) {
        long long j = sw.ka - g.k_lo;
        if (j >= 0 && j < g.nb) {
          double q = __dmul_rn(a2, gq[j]);
          deposit_q(acc_lo, acc_hi, j, q, &rs->err);
          r = q;
        }
      } else {
        long long k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
        long long k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
        for (long long k = k0; k <= k1; ++k) {
          double w = sweep_weight(sw, k);
          if (w > 0.0) {
            long long j = k - g.k_lo;
            double q = __dmul_rn(__dmul_rn(a2, w), gq[j]);
            deposit_q(acc_lo, acc_hi, j, q, &rs->err);
            r = __dadd_rn(r, q);
          }
        }
      }
      if (r >= thr_q) {
        is_cand = true;
        rec.src = s;
        rec.a2 = a2;
        rec.lo = sw.lo;
        rec.hi = sw.hi;
      }
    }
    unsigned m = __ballot_sync(0xFFFFFFFFu, is_cand);
    if (m) {
      unsigned long long b0 = 0;
      if (lane == __ffs(m) - 1) b0 = atomicAdd(&rs->ncand, (unsigned long long)__popc(m));
      b0 = __shfl_sync(0xFFFFFFFFu, b0, __ffs(m) - 1);
      if (is_cand) cand[b0 + __popc(m & ((1u << lane) - 1u))] = rec;
    }
  }
}

void launch_prepass(const double* A, const double* f, const double* fdot, long long N,
                    const Grid& g, const double* gq, double thr_q, unsigned long long* acc_lo,
                    unsigned long long* acc_hi, Cand* cand, RunState* rs, int nsm,
                    cudaStream_t st) {
  if (N <= 0) return;
  int th = 256;
  long long want = (N + th - 1) / th;
  long long cap = (long long)nsm * 8;
  int bl = (int)(want < cap ? want : cap);
  k_prepass<<<bl, th, 0, st>>>(A, f, fdot, N, g, gq, thr_q, acc_lo, acc_hi, cand, rs);
}

// ============================================================================ spectrum

__device__ __forceinline__ void block_max_bits(u64 v, u64* target) {
  // v are bits of non-negative doubles: their integer order is the value order.
  for (int o = 16; o > 0; o >>= 1) {
    u64 t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = t > v ? t : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(target, v);
}

__global__ void k_q2p(const unsigned long long* __restrict__ acc_lo,
                      const unsigned long long* __restrict__ acc_hi, const double* __restrict__ S,
                      long long nb, double* __restrict__ P, RunState* rs) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  u64 bits = 0;
  if (j < nb) {
    U128 Q = q_combine(acc_lo[j], acc_hi[j]);
    double p = __dmul_rn(S[j], u128_to_dbl_scaled(Q, 64));
    P[j] = p;
    bits = (u64)__double_as_longlong(p);
  }
  block_max_bits(bits, &rs->max_p_bits);
}

void launch_q2p(const unsigned long long* acc_lo, const unsigned long long* acc_hi,
                const double* S, long long nb, double* P, RunState* rs, int, cudaStream_t st) {
  int th = 256;
  k_q2p<<<(unsigned)((nb + th - 1) / th), th, 0, st>>>(acc_lo, acc_hi, S, nb, P, rs);
}

__global__ void k_max_bits(const double* __restrict__ x, long long n, unsigned long long* max_bits) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  u64 b = 0;
  if (j < n) {
    b = (u64)__double_as_longlong(x[j]);
    if (b >> 63) b = 0ull;
  }
  block_max_bits(b, max_bits);
}

void launch_max_bits(const double* x, long long n, unsigned long long* max_bits, cudaStream_t st) {
  int th = 256;
  k_max_bits<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(x, n, max_bits);
}

// ============================================================================ chunk sort
// Chunks of Kc >= W consecutive bins: any window of at most W bins lies in at most two
// consecutive chunks.  Each chunk is sorted once (keys: the bits of the non-negative
// doubles, whose integer order is their value order; ties broken by position), and
// for every kSnapStride-th position t the set of sorted indices whose position is >= t
// is stored as a bitset ("snapshot") so that a thread can build the active set of any
// window quickly.

__global__ void k_chunk_sort(const double* __restrict__ x, long long n, SmoothPlan pl,
                             unsigned long long* __restrict__ skey, uint16_t* __restrict__ srank,
                             uint32_t* __restrict__ snap) {
  extern __shared__ unsigned long long sm_keys[];
  uint16_t* sm_idx = (uint16_t*)(sm_keys + pl.kpad);
  const int b = blockIdx.x;
  const long long base = (long long)b * pl.Kc;
  const int len = (int)((n - base) < pl.Kc ? (n - base) : pl.Kc);
  for (int i = threadIdx.x; i < pl.kpad; i += blockDim.x) {
    u64 k = ~0ull;
    if (i < len) {
      double v = x[base + i];
      k = (u64)__double_as_longlong(v);
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

void launch_chunk_sort(const double* x, long long n, const SmoothPlan& pl, unsigned long long* skey,
                       uint16_t* srank, uint32_t* snap, const RunState*, cudaStream_t st) {
  size_t smem = (size_t)pl.kpad * (sizeof(u64) + sizeof(uint16_t));
  int th = pl.kpad >= 1024 ? 1024 : (pl.kpad < 64 ? 64 : pl.kpad);
  k_chunk_sort<<<pl.nch, th, smem, st>>>(x, n, pl, skey, srank, snap);
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
    // valid iff A[x-1] precedes B[P-x] (or P-x == B.len)
    int y = P - x;
    bool ok = (y >= B.len) || (__ldg(A.key + x - 1) <= __ldg(B.key + y));
    if (ok) lo = x; else hi = x - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_median_slide(
    const unsigned long long* __restrict__ skey, const uint16_t* __restrict__ srank,
    const uint32_t* __restrict__ snap, long long n, SmoothPlan pl, double* __restrict__ out,
    unsigned long long* max_bits_out, const double* __restrict__ S, int rtol_on, RunState* rs) {
  extern __shared__ uint32_t sm_bits[];
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  const int nw = pl.nw;
  uint32_t* bsX = sm_bits + tid;               // word w at bsX[w * T]
  uint32_t* bsY = sm_bits + (size_t)nw * T + tid;
  const long long g = blockIdx.x * (long long)T + tid;
  const long long j0 = g * pl.L;
  u64 mbits = 0;
  double relmax = 0.0;
  if (j0 < n) {
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
      if (rtol_on) {
        double a = __dadd_rn(S[j], v), bprev = __dadd_rn(S[j], out[j]);
        double rel = fabs(__dsub_rn(a, bprev)) / a;
        relmax = rel > relmax ? rel : relmax;
      }
      out[j] = v;
      u64 vb = (u64)__double_as_longlong(v);
      mbits = vb > mbits ? vb : mbits;
    }
  }
  if (max_bits_out) block_max_bits(mbits, max_bits_out);
  if (rtol_on) block_max_bits((u64)__double_as_longlong(relmax), &rs->relchg_bits);
}

void launch_median_slide(const unsigned long long* skey, const uint16_t* srank,
                         const uint32_t* snap, long long n, const SmoothPlan& pl, double* out,
                         unsigned long long* max_bits_out, const double* S, int rtol_on,
                         RunState* rs, cudaStream_t st) {
  int th = pl.slide_threads;
  long long threads = (n + pl.L - 1) / pl.L;
  long long bl = (threads + th - 1) / th;
  size_t smem = (size_t)2 * pl.nw * th * sizeof(uint32_t);
  k_median_slide<<<(unsigned)bl, th, smem, st>>>(skey, srank, snap, n, pl, out, max_bits_out, S,
                                                 rtol_on, rs);
}

// ============================================================================ window mean
// Exact window sums: every value becomes a 128-bit integer number of units 2^-sigma,
// where sigma comes from the maximum of the input so that any sum of 2 Kc inputs fits;
// each chunk stores its inclusive prefix sums, and a window (at most two chunks) is a
// difference/sum of prefixes.  Integer sums are exact, so there is no cancellation
// however large the dynamic range of the spectrum.

__device__ __forceinline__ int sigma_from_max(u64 maxbits) {
  // max < 2^(e - 1022) with e the biased exponent; 2 Kc <= 2^14 terms stay below 2^127.
  int e = (int)((maxbits >> 52) & 0x7FF);
  if (e == 0) e = 1;
  return 1135 - e;
}

__global__ void k_chunk_prefix(const double* __restrict__ x, long long n, SmoothPlan pl,
                               const unsigned long long* max_bits,
                               unsigned long long* __restrict__ pre_lo,
                               unsigned long long* __restrict__ pre_hi,
                               unsigned* __restrict__ uflow) {
  __shared__ U128 warp_tot[32];
  __shared__ int any_uf;
  const int b = blockIdx.x;
  const long long base = (long long)b * pl.Kc;
  const int len = (int)((n - base) < pl.Kc ? (n - base) : pl.Kc);
  const int sigma = sigma_from_max(*max_bits);
  const int per = (pl.Kc + blockDim.x - 1) / blockDim.x;
  const int p0 = threadIdx.x * per;
  U128 run{0ull, 0ull};
  if (threadIdx.x == 0) any_uf = 0;
  __syncthreads();
  // pass 1: thread totals; note inputs > 0 that fall below one unit
  int uf = 0;
  for (int i = 0; i < per; ++i) {
    int p = p0 + i;
    if (p < len) {
      double v = x[base + p];
      U128 q = dbl_to_u128_scaled(v, sigma);
      if (v > 0.0 && u128_is_zero(q)) uf = 1;
      run = u128_add(run, q);
    }
  }
  if (uf) any_uf = 1;
  // exclusive scan of thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    int nwarp = blockDim.x >> 5;
    U128 v = lane < nwarp ? warp_tot[lane] : U128{0ull, 0ull};
    for (int o = 1; o < 32; o <<= 1) {
      U128 t;
      t.lo = __shfl_up_sync(0xFFFFFFFFu, v.lo, o);
      t.hi = __shfl_up_sync(0xFFFFFFFFu, v.hi, o);
      if (lane >= o) v = u128_add(v, t);
    }
    if (lane < nwarp) warp_tot[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  U128 offs = u128_sub(inc, run);  // exclusive within warp
  if (warp > 0) offs = u128_add(offs, warp_tot[warp - 1]);
  // pass 2: write inclusive prefixes
  for (int i = 0; i < per; ++i) {
    int p = p0 + i;
    if (p < len) {
      offs = u128_add(offs, dbl_to_u128_scaled(x[base + p], sigma));
      pre_lo[base + p] = offs.lo;
      pre_hi[base + p] = offs.hi;
    }
  }
  if (threadIdx.x == 0) uflow[b] = (unsigned)any_uf;
}

void launch_chunk_prefix(const double* x, long long n, const SmoothPlan& pl,
                         const unsigned long long* max_bits, unsigned long long* pre_lo,
                         unsigned long long* pre_hi, unsigned* uflow, const RunState*,
                         cudaStream_t st) {
  int th = 256;
  k_chunk_prefix<<<pl.nch, th, 0, st>>>(x, n, pl, max_bits, pre_lo, pre_hi, uflow);
}

__global__ void k_window_mean(const double* __restrict__ x, long long n, SmoothPlan pl,
                              const unsigned long long* max_bits,
                              const unsigned long long* __restrict__ pre_lo,
                              const unsigned long long* __restrict__ pre_hi,
                              const unsigned* __restrict__ uflow, double* __restrict__ out,
                              const double* __restrict__ S, int rtol_on, RunState* rs) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double relmax = 0.0;
  if (j < n) {
    const int sigma = sigma_from_max(*max_bits);
    const int h = pl.W / 2;
    long long s = j - h > 0 ? j - h : 0;
    long long e = j - h + pl.W - 1 < n - 1 ? j - h + pl.W - 1 : n - 1;
    long long cs = s / pl.Kc, ce = e / pl.Kc;
    U128 pe{pre_lo[e], pre_hi[e]};
    U128 sum;
    U128 before{0ull, 0ull};
    if (s > cs * pl.Kc) before = U128{pre_lo[s - 1], pre_hi[s - 1]};
    if (cs == ce) {
      sum = u128_sub(pe, before);
    } else {
      long long last = cs * pl.Kc + pl.Kc - 1;
      U128 tot{pre_lo[last], pre_hi[last]};
      sum = u128_add(u128_sub(tot, before), pe);
    }
    long long cnt = e - s + 1;
    double v;
    // Each input lost less than one unit; if the sum holds fewer than cnt * 2^40 units
    // the relative error could exceed 2^-40, so add the doubles directly instead.  A zero
    // sum is exact only if no input of these chunks fell below one unit.
    bool small = (sum.hi == 0ull) && (sum.lo < ((unsigned long long)cnt << 40));
    if (u128_is_zero(sum) && !(uflow[cs] | uflow[ce])) {
      v = 0.0;
    } else if (small) {
      double acc = 0.0;
      for (long long i = s; i <= e; ++i) acc = __dadd_rn(acc, x[i]);
      v = __ddiv_rn(acc, (double)cnt);
    } else {
      double sd = u128_to_dbl_scaled(sum, sigma);
      v = (cnt == pl.W) ? __dmul_rn(sd, 1.0 / (double)pl.W) : __ddiv_rn(sd, (double)cnt);
    }
    if (rtol_on) {
      double a = __dadd_rn(S[j], v), bprev = __dadd_rn(S[j], out[j]);
      relmax = fabs(__dsub_rn(a, bprev)) / a;
    }
    out[j] = v;
  }
  if (rtol_on) block_max_bits((u64)__double_as_longlong(relmax), &rs->relchg_bits);
}

void launch_window_mean(const double* x, long long n, const SmoothPlan& pl,
                        const unsigned long long* max_bits, const unsigned long long* pre_lo,
                        const unsigned long long* pre_hi, const unsigned* uflow, double* out,
                        const double* S, int rtol_on, RunState* rs, cudaStream_t st) {
  int th = 256;
  k_window_mean<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(x, n, pl, max_bits, pre_lo, pre_hi,
                                                               uflow, out, S, rtol_on, rs);
}

// ============================================================================ SNR + resolve

__device__ __forceinline__ bool rtol_stop(const RunState* rs, double rtol) {
  if (!(rtol > 0.0) || rs->iter < 1) return false;
  double r = __longlong_as_double((i64)rs->relchg_bits);
  return r <= rtol;
}

__device__ __forceinline__ void remove_q(unsigned long long* acc_lo, unsigned long long* acc_hi,
                                         long long j, double q) {
  if (!(q < kQLimit)) return;  // never deposited
  u64 lo, hi;
  q_split(q, &lo, &hi);
  if (lo) atomicAdd(acc_lo + j, (u64)(0ull - lo));
  if (hi) atomicAdd(acc_hi + j, (u64)(0ull - hi));
}

__global__ void __launch_bounds__(256) k_snr_resolve(
    const Cand* __restrict__ cand, Grid g, const double* __restrict__ S,
    const double* __restrict__ R, const double* __restrict__ gq, const double* __restrict__ Sg,
    double th2, double rtol, unsigned char* __restrict__ cres, unsigned char* __restrict__ resolved,
    unsigned long long* __restrict__ acc_lo, unsigned long long* __restrict__ acc_hi,
    RunState* rs) {
  if (rs->final_pass || rtol_stop(rs, rtol)) return;
  const long long ncand = (long long)rs->ncand;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned local_new = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncand; c += stride) {
    if (cres[c]) continue;
    Cand cd = cand[c];
    Sweep sw;
    sw.lo = cd.lo;
    sw.hi = cd.hi;
    sw.ka = (i64)floor(__dadd_rn(sw.lo, 0.5));
    sw.kb = (i64)floor(__dadd_rn(sw.hi, 0.5));
    double acc = 0.0;
    long long k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
    long long k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
    bool single = (sw.ka == sw.kb);
    for (long long k = k0; k <= k1; ++k) {
      double w = single ? 1.0 : sweep_weight(sw, k);
      if (w > 0.0) {
        long long j = k - g.k_lo;
        double sn = __dadd_rn(S[j], Sg[j]);
        double psk = __dmul_rn(__dmul_rn(__dmul_rn(g.t5, R[j]), cd.a2), w);
        acc = __dadd_rn(acc, __ddiv_rn(psk, sn));
      }
    }
    double rho2 = __dmul_rn(4.0, acc);
    if (rho2 > th2) {
      cres[c] = 1;
      resolved[cd.src] = 1;
      ++local_new;
      for (long long k = k0; k <= k1; ++k) {
        double w = single ? 1.0 : sweep_weight(sw, k);
        if (w > 0.0) {
          long long j = k - g.k_lo;
          double q = single ? __dmul_rn(cd.a2, gq[j]) : __dmul_rn(__dmul_rn(cd.a2, w), gq[j]);
          remove_q(acc_lo, acc_hi, j, q);
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) local_new += __shfl_xor_sync(0xFFFFFFFFu, local_new, o);
  if ((threadIdx.x & 31) == 0 && local_new) atomicAdd(&rs->count_new, (unsigned long long)local_new);
}

void launch_snr_resolve(const Cand* cand, long long ncand_cap, const Grid& g, const double* S,
                        const double* R, const double* gq, const double* Sg, double th2,
                        double rtol, unsigned char* cres, unsigned char* resolved,
                        unsigned long long* acc_lo, unsigned long long* acc_hi, RunState* rs,
                        int nsm, cudaStream_t st) {
  int th = 256;
  long long want = (ncand_cap + th - 1) / th;
  long long cap = (long long)nsm * 8;
  int bl = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  k_snr_resolve<<<bl, th, 0, st>>>(cand, g, S, R, gq, Sg, th2, rtol, cres, resolved, acc_lo, acc_hi,
                                   rs);
}

// ============================================================================ loop control

__global__ void k_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                          unsigned long long cond_handle, int use_cond) {
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
  rs->max_p_bits = 0ull;
  rs->max_m_bits = 0ull;
  rs->relchg_bits = 0ull;
  if (!go) rs->stopped = 1;
  if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, go);
}

void launch_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                    unsigned long long cond_handle, int use_cond, cudaStream_t st) {
  k_control<<<1, 1, 0, st>>>(rs, max_iter, rtol, new_hist, cond_handle, use_cond);
}

void configure_kernels() {
  cudaFuncSetAttribute(k_chunk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  cudaFuncSetAttribute(k_median_slide, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
}

}  // namespace gbsub
