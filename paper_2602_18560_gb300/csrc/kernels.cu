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
  // q >= 0: compare the bits with those of 2^159 (no FP64 instruction)
  if ((u64)__double_as_longlong(q) >= kQLimitBits) {
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
  if ((u64)__double_as_longlong(q) >= kQLimitBits) return;  // never deposited
  u64 c0, c1, c2;
  q_parts(q, &c0, &c1, &c2);
  u64* a = acc + 4 * j;
  if (c0) atomicAdd(a + 0, (u64)(0ull - c0));
  if (c1) atomicAdd(a + 1, (u64)(0ull - c1));
  if (c2) atomicAdd(a + 2, (u64)(0ull - c2));
}

// The parts of a single-bin deposit (q_single) added to, or taken from, bin j.
__device__ __forceinline__ void add_parts(unsigned long long* acc, long long j, u64 c0, u64 c1,
                                          u64 c2) {
  u64* a = acc + 4 * j;
  if (c0) atomicAdd(a + 0, c0);
  if (c1) atomicAdd(a + 1, c1);
  if (c2) atomicAdd(a + 2, c2);
}
__device__ __forceinline__ void sub_parts(unsigned long long* acc, long long j, u64 c0, u64 c1,
                                          u64 c2) {
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
    return __dmul_rn(in.S[j], u128_to_dbl_scaled(Q, 64));
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

// The catalog is dominated by the low-frequency end of the band (the number of sources
// falls steeply with f), so the 64-bit atomics of the deposits pile up on the cache lines
// of the first bins: an L2 line takes one atomic at a time.  The first rep.nbins bins
// therefore have kAccReplicas private copies (words 0 and 1 of every bin), a source
// picking one by its index; a fold adds them into the spectrum after the pass (word 2 takes
// a part only from a source of at least S_instr in the bin, rare, and goes to the spectrum
// directly).  Integer sums, so the result does not depend on the split.
__device__ __forceinline__ void add_parts_rep(AccReplicas rep, unsigned long long* acc,
                                              long long j, int r, u64 c0, u64 c1, u64 c2) {
  u64* a = rep.w + 2 * ((size_t)r * rep.nbins + j);
  if (c0) atomicAdd(a + 0, c0);
  if (c1) atomicAdd(a + 1, c1);
  if (c2) atomicAdd(acc + 4 * j + 2, c2);
}

__global__ void k_fold_replicas(unsigned long long* __restrict__ acc, AccReplicas rep) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= rep.nbins) return;
  u64 s1 = 0, s2 = 0;
#pragma unroll
  for (int r = 0; r < kAccReplicas; ++r) {
    const ulonglong2 v = reinterpret_cast<const ulonglong2*>(rep.w)[(size_t)r * rep.nbins + j];
    s1 += v.x;
    s2 += v.y;
  }
  acc[4 * j + 0] += s1;
  acc[4 * j + 1] += s2;
}


// FP64 path of the catalog pass: the sweep of one source, its pieces deposited; returns
// the sum of its contributions.  Kept out of line so that none of it is speculated into
// the common path.
// Bins of a source's sweep that the FP64 path walks: [k0, k1] (absolute bin numbers),
// empty when the sweep leaves the band.
__device__ __forceinline__ void sweep_bins(const Sweep& sw, const Grid& g, long long* k0,
                                           long long* k1) {
  *k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
  *k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
}

// Deposit bins k0 + off, k0 + off + step, ... <= k1 of a multi-bin sweep; returns the sum
// of their contributions in that order.
__device__ __forceinline__ double sweep_deposit(const Sweep& sw, const Grid& g, const Tables& tb,
                                                double a2, long long k0, long long k1, int off,
                                                int step, unsigned long long* acc,
                                                unsigned* err) {
  double r = 0.0;
  const double inv = sweep_inv_len(sw);
  for (long long k = k0 + off; k <= k1; k += step) {
    double w = sweep_weight_inv(sw, k, inv);
    if (w > 0.0) {
      long long j = k - g.k_lo;
      double q = __dmul_rn(__dmul_rn(a2, w), tb.gq[j]);
      deposit_q(acc, j, q, err);
      r = __dadd_rn(r, q);
    }
  }
  return r;
}

// FP64 path of the catalog pass for one source: the sweep, its pieces deposited; returns
// the sum of its contributions.  Kept out of line so that none of it is speculated into the
// common path.
// A single-bin sweep is deposited as q_single(A, gq) exactly as the common path deposits it, so
// that every single-bin source is removed the same way whichever path deposited it.
__device__ __noinline__ double prepass_slow(double A, double fs, double fds, const Grid g,
                                            const Tables tb, unsigned long long* acc,
                                            unsigned* err) {
  Sweep sw = make_sweep(fs, fds, g.T, g.T2);
  if (sw.ka == sw.kb) {
    long long j = sw.ka - g.k_lo;
    if (j >= 0 && j < g.nb) {
      u64 c0, c1, c2, qb;
      if (!q_single(A, tb.gq[j], &c0, &c1, &c2, &qb)) {
        atomicOr(err, ERR_RANGE);
        return 0.0;
      }
      add_parts(acc, j, c0, c1, c2);
      return __longlong_as_double((long long)qb);
    }
    return 0.0;
  }
  long long k0, k1;
  sweep_bins(sw, g, &k0, &k1);
  return sweep_deposit(sw, g, tb, __dmul_rn(A, A), k0, k1, 0, 1, acc, err);
}

// Bins the FP64 path of a source would walk (0 for a single-bin sweep).
__device__ __noinline__ long long slow_span(double fs, double fds, const Grid g) {
  Sweep sw = make_sweep(fs, fds, g.T, g.T2);
  if (sw.ka == sw.kb) return 0;
  long long k0, k1;
  sweep_bins(sw, g, &k0, &k1);
  return k1 >= k0 ? k1 - k0 + 1 : 0;
}

// The FP64 path of one long sweep, by a whole warp: the lanes share its bins; the sum of the
// contributions comes back in every lane.
__device__ __noinline__ double prepass_slow_warp(double A, double fs, double fds, const Grid g,
                                                 const Tables tb, unsigned long long* acc,
                                                 unsigned* err) {
  const int lane = threadIdx.x & 31;
  Sweep sw = make_sweep(fs, fds, g.T, g.T2);
  long long k0, k1;
  sweep_bins(sw, g, &k0, &k1);
  double r = sweep_deposit(sw, g, tb, __dmul_rn(A, A), k0, k1, lane, 32, acc, err);
  for (int o = 16; o > 0; o >>= 1) r = __dadd_rn(r, __shfl_xor_sync(0xFFFFFFFFu, r, o));
  return r;
}

// Record of a kept candidate (rare; out of line).
__device__ __noinline__ void emit_candidate(Cands cd, long long c, long long s, double A,
                                            double fs, double fds, const Grid g,
                                            unsigned long long* nwide) {
  Sweep sw = make_sweep(fs, fds, g.T, g.T2);
  const double a2 = __dmul_rn(A, A);
  cd.src[c] = s;
  cd.pk[c] = make_int4((int)(sw.ka - g.k_lo), (int)(sw.kb - sw.ka + 1),
                       __float_as_int(dbl_to_f32_scaled(a2, 160)),
                       __float_as_int((float)(sw.lo - (double)sw.ka)));
  cd.len[c] = (float)(sw.hi - sw.lo);
  cd.a2[c] = a2;
  cd.amp[c] = A;
  cd.lo[c] = sw.lo;
  cd.hi[c] = sw.hi;
  cd.res[c] = 0;
  if (sw.kb - sw.ka + 1 > kSnrLaneBins) cd.wide[atomicAdd(nwide, 1ull)] = c;
}

// The decision for one source once r (its rho_0^2 / 4 in units of 2^-96) is known: count
// it among the paper's candidates, and keep it when it can still be resolved.
__device__ __forceinline__ void prepass_decide(double r, u64 tk_bits, u64 tl_bits, bool valid,
                                               long long s, double A, double fs, double fds,
                                               const Grid& g, Cands& cd, RunState* rs,
                                               unsigned long long& nkappa) {
  const int lane = threadIdx.x & 31;
  u64 rb = (u64)__double_as_longlong(r);
  bool live = false;
  if (valid) {
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
      emit_candidate(cd, c, s, A, fs, fds, g, &rs->nwide);
    }
  }
}

// ---------------------------------------------------------------- TMA staging
// The catalog streams through shared memory: one thread issues bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier) of whole tiles of A, f and
// fdot a few tiles ahead, so no thread waits on HBM for its sources.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Wait for phase `parity` of the barrier; false after about a second of polling.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const uint32_t a = smem_addr(bar);
  for (int i = 0; i < (1 << 20); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(1000);
  }
  return false;
}

// Sources whose sweep the FP32 bound cannot keep in one bin go through the FP64 path.  They
// are rare (well under 1%), but one such lane would hold its whole warp on the slow FP64
// pipe, so each warp queues them in shared memory and runs them 32 at a time.
//
// Layout of a CTA: kPreConsumers consumer warps and one producer warp.  The producer takes
// tiles of kPreTile sources from a global counter (CTAs that run faster take more tiles) and
// streams each into one of kPreStages shared-memory stages with bulk asynchronous copies of
// A, f and fdot (cp.async.bulk, completion counted in bytes on the stage's "full" mbarrier).
// Each consumer warp takes its own kPreTile / kPreConsumers sources of the stage and, done,
// arrives on the stage's "empty" mbarrier; the producer refills a stage once every consumer
// warp has arrived.  No CTA-wide barrier runs in the steady state, so a warp that meets a
// slow source delays no other warp.
constexpr int kPreConsumers = 8;
constexpr int kPrepassThreads = (kPreConsumers + 1) * 32;
constexpr int kPreTile = 512;                                 // sources per staged tile
constexpr int kPreStages = 4;                                 // tiles in flight per CTA
constexpr int kPreWarpSrc = kPreTile / kPreConsumers;         // sources per consumer warp
constexpr int kPrePer = kPreWarpSrc / 32;                     // sources per lane per tile
constexpr int kSlowWarpCap = 64;                              // queue of a warp (drained at 32)
constexpr size_t kPrepassSmem = (size_t)kPreStages * kPreTile * 3 * sizeof(double);

// Sweeps longer than this many bins are walked by a whole warp (loud high-frequency sources
// sweep up to hundreds of bins; one lane walking them in FP64 would hold its warp, and the
// launch, long after every other warp is done).
constexpr long long kSlowLaneBins = 4;

// Source s of a generated catalog.
__device__ __forceinline__ double3 gen_source_at(const CatalogRef* __restrict__ cat, long long s) {
  const GenParams g = cat->gen;
  double3 r;
  gen_source(g, s, &r.x, &r.y, &r.z);
  return r;
}

// f T + 1/2 split into its integer part k and the top 24 bits of its fraction, from the
// exact product when T's mantissa has at most 32 significant bits (T = tq 2^etq; whole
// seconds of observation time qualify).  The mantissa of f is split in 21 + 32 bits, so the
// product is two 32 x 32 -> 64-bit multiplies.  Exact f T, not its FP64 rounding: the two
// differ by less than 2^-33 bins in the band, and the caller keeps a source on this path
// only when the fraction is at least 2^-20 from a cell edge, where both give the same bin.
// False for f not positive normal, or f T outside the range handled here.
__device__ __forceinline__ bool ft_bin_short(double f, unsigned tq, int etq, long long* k,
                                             unsigned* frac24) {
  const u64 b = (u64)__double_as_longlong(f);
  const int e = (int)(b >> 52);  // sign bit included: a negative f fails the range test
  if (e <= 0 || e >= 0x7FF) return false;
  const u64 mf = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const u64 p0 = (u64)(unsigned)mf * tq;           // low 32 bits of mf times tq
  const u64 p1 = (u64)(unsigned)(mf >> 32) * tq;   // high 21 bits of mf times tq
  const u64 hi = p1 + (p0 >> 32);                  // f T = (hi 2^32 + lo) 2^(e - 1075 + etq)
  const int G = 1075 - etq - e - 32;               // fraction bits of f T within hi
  if (G < 24 || G > 62) return false;
  const u64 x = hi + (1ull << (G - 1));            // + 1/2
  *k = (long long)(x >> G);
  *frac24 = (unsigned)(x >> (G - 24)) & 0xFFFFFFu;
  return true;
}

// The common case of one source without any FP64 arithmetic beyond A^2: its bin k0 and the
// FP32 certificate that the whole sweep [f T, f T + fdot T^2] stays inside cell k0 (else the
// FP64 path takes it).
__device__ __forceinline__ bool single_bin(double fs, double fds, const Grid& g, long long* k0) {
  unsigned fr24 = 0;
  bool ok;
  if (g.short_t) {
    ok = ft_bin_short(fs, g.tq, g.etq, k0, &fr24);
  } else {
    int fb;
    ok = ft_bin(fs, g.mT, g.eT, k0, &fr24, &fb);
  }
  if (!ok) return false;
  const float du = __fmul_rn(dbl_to_f32_signed(fds), g.T2f);
  const float phi = __fmul_rn((float)fr24, 5.9604644775390625e-8f);             // 2^-24
  const float m = __fadd_rn(9.5367431640625e-7f, __fmul_rn(4e-7f, fabsf(du)));  // 2^-20 + ...
  const float x = __fadd_rn(phi, du);
  return (x >= m) && (x < __fsub_rn(1.0f, m));
}

// The FP64 path of up to 32 queued sources q[0 .. cnt) of one warp (lane i takes entry i;
// sweeps longer than kSlowLaneBins by the whole warp).
template <bool kGen>
__device__ __forceinline__ void prepass_drain_warp(const CatalogRef* __restrict__ cat,
                                                   const double* __restrict__ A,
                                                   const double* __restrict__ f,
                                                   const double* __restrict__ fdot,
                                                   const Grid& g, const Tables& tb, u64 tk_bits,
                                                   u64 tl_bits, unsigned long long* __restrict__ acc,
                                                   Cands& cd, RunState* rs, const long long* q,
                                                   int cnt, unsigned long long& nkappa) {
  const int lane = threadIdx.x & 31;
  const bool valid = lane < cnt;
  long long s = valid ? q[lane] : 0;
  double a = 0.0, fs = 0.0, fds = 0.0, r = 0.0;
  bool wide = false;
  if (valid) {
    if (kGen) {
      const double3 gsrc = gen_source_at(cat, s);
      a = gsrc.x;
      fs = gsrc.y;
      fds = gsrc.z;
    } else {
      a = A[s];
      fs = f[s];
      fds = fdot[s];
    }
    wide = slow_span(fs, fds, g) > kSlowLaneBins;
    if (!wide) r = prepass_slow(a, fs, fds, g, tb, acc, &rs->err);
  }
  prepass_decide(r, tk_bits, tl_bits, valid && !wide, s, a, fs, fds, g, cd, rs, nkappa);
  unsigned pending = __ballot_sync(0xFFFFFFFFu, wide);
  while (pending) {
    const int src = __ffs(pending) - 1;
    pending &= pending - 1;
    const long long sw_s = __shfl_sync(0xFFFFFFFFu, s, src);
    const double sw_a = __shfl_sync(0xFFFFFFFFu, a, src);
    const double sw_f = __shfl_sync(0xFFFFFFFFu, fs, src);
    const double sw_fd = __shfl_sync(0xFFFFFFFFu, fds, src);
    const double rw = prepass_slow_warp(sw_a, sw_f, sw_fd, g, tb, acc, &rs->err);
    prepass_decide(rw, tk_bits, tl_bits, lane == 0, sw_s, sw_a, sw_f, sw_fd, g, cd, rs,
                   nkappa);
  }
}

// One source of the catalog pass (s < N; every lane of the warp calls it together): the
// common case deposited here, a source the FP64 path must take appended to the warp's queue
// q (qn entries, the same in every lane), which is drained 32 at a time.
template <bool kGen>
__device__ __forceinline__ void prepass_source(
    long long s, long long N, double a, double fs, double fds, const CatalogRef* __restrict__ cat,
    const double* __restrict__ A, const double* __restrict__ f, const double* __restrict__ fdot,
    const Grid& g, const Tables& tb, u64 tk_bits, u64 tl_bits, unsigned long long* __restrict__ acc,
    const AccReplicas& rep, Cands& cd, RunState* rs, long long* q, int& qn,
    unsigned long long& nkappa) {
  const int lane = threadIdx.x & 31;
  bool valid = false, slow = false;
  double r = 0.0;
  if (s < N) {
    // finite inputs, and A^2 finite (|A| < 2^512): else the source is refused below
    const bool fin = finite3(a, fs, fds) && (((u64)__double_as_longlong(a) >> 52) & 0x7FF) < 1535;
    long long k0 = 0;
    const bool single = fin && single_bin(fs, fds, g, &k0);
    if (single) {
      valid = true;
      const long long j = k0 - g.k_lo;
      if (j >= 0 && j < g.nb) {
        u64 c0, c1, c2, qb;
        if (q_single(a, tb.gq[j], &c0, &c1, &c2, &qb)) {
          if (j < rep.nbins)
            add_parts_rep(rep, acc, j, (int)(s & (kAccReplicas - 1)), c0, c1, c2);
          else
            add_parts(acc, j, c0, c1, c2);
          r = __longlong_as_double((long long)qb);
        } else {
          atomicOr(&rs->err, ERR_RANGE);
        }
      }
    } else if (fin) {
      slow = true;
    } else {
      atomicOr(&rs->err, ERR_INPUT);  // the source is skipped; the run reports it
    }
  }
  // append the warp's slow sources to its queue
  const unsigned sm = __ballot_sync(0xFFFFFFFFu, slow);
  if (slow) q[qn + __popc(sm & ((1u << lane) - 1u))] = s;
  qn += __popc(sm);
  prepass_decide(r, tk_bits, tl_bits, valid, s, a, fs, fds, g, cd, rs, nkappa);
  if (qn >= 32) {
    __syncwarp();
    prepass_drain_warp<kGen>(cat, A, f, fdot, g, tb, tk_bits, tl_bits, acc, cd, rs, q, 32,
                             nkappa);
    __syncwarp();
    if (lane < qn - 32) q[lane] = q[32 + lane];
    qn -= 32;
    __syncwarp();
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Wait for phase `parity` of the barrier; false once *abort is set by another warp of the CTA,
// or after about a second (2^31 clocks), or after 2^24 polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, unsigned parity,
                                                const int* abort) {
  const uint32_t a = smem_addr(bar);
  const long long t0 = clock64();
  for (int i = 0; i < (1 << 24); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 63) == 63) {
      if (*(volatile const int*)abort) return false;
      if (clock64() - t0 > (2LL << 30)) return false;
      __nanosleep(256);
    }
  }
  return false;
}

__global__ void __launch_bounds__(kPrepassThreads, 3) k_prepass(
    const CatalogRef* cat, Grid g, Tables tb, double thr_kappa, double thr_live,
    unsigned long long* __restrict__ acc, AccReplicas rep, Cands cd, RunState* rs,
    int test_flags) {
  extern __shared__ __align__(128) double pre_tiles[];  // [stage][A | f | fdot][kPreTile]
  __shared__ __align__(8) uint64_t full[kPreStages], empty[kPreStages];
  __shared__ long long stage_tile[kPreStages];  // tile held by each stage
  __shared__ long long slow_q[kPreConsumers][kSlowWarpCap];
  __shared__ int abort_flag;
  // the catalog record (and a generated catalog's constants), read once per CTA: every
  // thread of the grid loading it would queue on one L2 line
  __shared__ CatalogRef scat;
  const int tid = threadIdx.x;
  if (tid == 0) {
    scat = *cat;
    for (int k = 0; k < kPreStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kPreConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();
  cat = &scat;
  const double* __restrict__ A = scat.A;
  const double* __restrict__ f = scat.f;
  const double* __restrict__ fdot = scat.fdot;
  const long long N = scat.n;
  const bool use_tma = scat.staged == kCatDevice;
  if (scat.staged == kCatGenerated) return;  // k_prepass_gen's catalog
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const long long ntiles = (N + kPreTile - 1) / kPreTile;
  // full tiles of device memory come through TMA; the ragged one, and every tile of a catalog
  // in host memory, through plain loads
  const long long nfull = use_tma ? N / kPreTile : 0;

  if (warp == kPreConsumers) {
    // ------------------------------------------------ producer (one lane)
    if (lane != 0) return;
    // bit k of copying: the copies of stage k's latest tile were started, in its use of
    // parity bit k of copy_par (they complete that phase of full[k])
    unsigned copying = 0, copy_par = 0;  // bit k: stage k
    for (long long i = 0;; ++i) {
      const int stage = (int)(i % kPreStages);
      const unsigned use = (unsigned)(i / kPreStages);
      if (use > 0) {
        // every consumer warp has let go of the stage's previous tile
        if (!mbar_wait_abort(&empty[stage], (use - 1) & 1, &abort_flag)) {
          atomicOr(&rs->err, ERR_TIMEOUT);
          *(volatile int*)&abort_flag = 1;
          break;
        }
        copying &= ~(1u << stage);  // the consumers waited for those copies
      }
      const long long t = (long long)atomicAdd(&rs->next_tile, 1ull);
      stage_tile[stage] = t;
      if (t < nfull && !(test_flags & 1)) {
        copying |= 1u << stage;
        copy_par = (copy_par & ~(1u << stage)) | ((use & 1u) << stage);
        double* d = pre_tiles + (size_t)stage * 3 * kPreTile;
        const size_t off = (size_t)t * kPreTile;
        mbar_expect_tx(&full[stage], 3u * kPreTile * (unsigned)sizeof(double));
        bulk_g2s(d, A + off, kPreTile * sizeof(double), &full[stage]);
        bulk_g2s(d + kPreTile, f + off, kPreTile * sizeof(double), &full[stage]);
        bulk_g2s(d + 2 * kPreTile, fdot + off, kPreTile * sizeof(double), &full[stage]);
      } else if (t >= nfull) {
        mbar_arrive(&full[stage]);  // a ragged or mapped tile, or the end
      }
      // (with the test hook a full tile gets no copy and no arrival: its waits run out)
      if (t >= ntiles) break;
    }
    if (*(volatile int*)&abort_flag) {
      // the consumers gave up: wait (bounded) for every copy this CTA started before its
      // shared memory goes away
      for (int k = 0; k < kPreStages; ++k)
        if ((copying >> k) & 1u) mbar_wait(&full[k], (copy_par >> k) & 1u);
    }
    return;
  }

  // -------------------------------------------------- consumers
  // thresholds on r >= 0 compared as the integer bits of non-negative doubles
  const u64 tk_bits = (u64)__double_as_longlong(thr_kappa);
  const u64 tl_bits = (u64)__double_as_longlong(thr_live);
  unsigned long long nkappa = 0;
  long long* myq = slow_q[warp];
  int qn = 0;  // entries of the warp's queue (the same in every lane)
  for (long long i = 0;; ++i) {
    const int stage = (int)(i % kPreStages);
    const unsigned use = (unsigned)(i / kPreStages);
    const bool ok = mbar_wait_abort(&full[stage], use & 1, &abort_flag);
    if (!__all_sync(0xFFFFFFFFu, ok)) {
      if (lane == 0) {
        atomicOr(&rs->err, ERR_TIMEOUT);
        *(volatile int*)&abort_flag = 1;
      }
      return;
    }
    const long long t = stage_tile[stage];
    if (t >= ntiles) break;
    const bool staged = t < nfull;
    const double* sA = pre_tiles + (size_t)stage * 3 * kPreTile;
    const double* sF = sA + kPreTile;
    const double* sD = sF + kPreTile;
    const int base = warp * kPreWarpSrc + lane;
    // every load of the lane's sources first: from host memory each one takes a
    // microsecond or more
    double av[kPrePer], fv[kPrePer], dv[kPrePer];
#pragma unroll
    for (int k = 0; k < kPrePer; ++k) {
      const int idx = base + 32 * k;
      const long long s = t * kPreTile + idx;
      av[k] = fv[k] = dv[k] = 0.0;
      if (staged) {
        av[k] = sA[idx];
        fv[k] = sF[idx];
        dv[k] = sD[idx];
      } else if (s < N) {
        av[k] = A[s];
        fv[k] = f[s];
        dv[k] = fdot[s];
      }
    }
    // the stage may be refilled once every warp has its values in registers
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[stage]);
#pragma unroll
    for (int k = 0; k < kPrePer; ++k)
      prepass_source<false>(t * kPreTile + base + 32 * k, N, av[k], fv[k], dv[k], cat, A, f,
                            fdot, g, tb, tk_bits, tl_bits, acc, rep, cd, rs, myq, qn, nkappa);
  }
  __syncwarp();
  if (qn > 0)
    prepass_drain_warp<false>(cat, A, f, fdot, g, tb, tk_bits, tl_bits, acc, cd, rs, myq, qn,
                              nkappa);
  for (int o = 16; o > 0; o >>= 1) nkappa += __shfl_xor_sync(0xFFFFFFFFu, nkappa, o);
  if (lane == 0 && nkappa) atomicAdd(&rs->ncand, nkappa);
}

// The catalog pass over a generated catalog: every source computed from (seed, index) where
// the pass over a stored catalog loads it, then the same per-source step.  Generation is
// ~300 FP32 and integer instructions per source, so there is nothing to stage: each warp takes
// runs of 32 kGenPer sources from the tile counter.  The other pass leaves a generated catalog
// to this one, and this one leaves every other catalog to it.
constexpr int kGenThreads = 256;
constexpr int kGenPer = 8;  // sources per lane per run

__global__ void __launch_bounds__(kGenThreads, 4) k_prepass_gen(
    const CatalogRef* cat, Grid g, Tables tb, double thr_kappa, double thr_live,
    unsigned long long* __restrict__ acc, AccReplicas rep, Cands cd, RunState* rs) {
  __shared__ CatalogRef scat;
  __shared__ long long slow_q[kGenThreads / 32][kSlowWarpCap];
  if (threadIdx.x == 0) scat = *cat;
  __syncthreads();
  if (scat.staged != kCatGenerated) return;
  cat = &scat;
  const long long N = scat.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u64 tk_bits = (u64)__double_as_longlong(thr_kappa);
  const u64 tl_bits = (u64)__double_as_longlong(thr_live);
  unsigned long long nkappa = 0;
  long long* myq = slow_q[warp];
  int qn = 0;
  constexpr long long kRun = 32LL * kGenPer;
  for (;;) {
    unsigned long long r0 = 0;
    if (lane == 0) r0 = atomicAdd(&rs->next_tile, 1ull);
    const long long base = (long long)__shfl_sync(0xFFFFFFFFu, r0, 0) * kRun;
    if (base >= N) break;
#pragma unroll 1
    for (int k = 0; k < kGenPer; ++k) {
      const long long s = base + 32 * k + lane;
      double3 src = make_double3(0.0, 0.0, 0.0);
      if (s < N) src = gen_source_at(cat, s);
      prepass_source<true>(s, N, src.x, src.y, src.z, cat, nullptr, nullptr, nullptr, g, tb,
                           tk_bits, tl_bits, acc, rep, cd, rs, myq, qn, nkappa);
    }
  }
  __syncwarp();
  if (qn > 0)
    prepass_drain_warp<true>(cat, nullptr, nullptr, nullptr, g, tb, tk_bits, tl_bits, acc, cd,
                             rs, myq, qn, nkappa);
  for (int o = 16; o > 0; o >>= 1) nkappa += __shfl_xor_sync(0xFFFFFFFFu, nkappa, o);
  if (lane == 0 && nkappa) atomicAdd(&rs->ncand, nkappa);
}

void launch_prepass(const CatalogRef* cat, long long cap, const Grid& g, const Tables& tb,
                    double thr_kappa, double thr_live, unsigned long long* acc, AccReplicas rep,
                    Cands cd, RunState* rs, int nsm, int test_flags, cudaStream_t st) {
  long long tiles = (cap + kPreTile - 1) / kPreTile;
  long long lim = (long long)nsm * 3;  // resident CTAs (launch bounds, shared memory)
  int bl = (int)(tiles < lim ? (tiles < 1 ? 1 : tiles) : lim);
  k_prepass<<<bl, kPrepassThreads, kPrepassSmem, st>>>(cat, g, tb, thr_kappa, thr_live, acc,
                                                       rep, cd, rs, test_flags);
  // the generated-catalog pass: resident CTAs, at most one per run of sources
  const long long runs = (cap + 32LL * kGenPer - 1) / (32LL * kGenPer);
  const long long glim = (long long)nsm * 4 * (kGenThreads / 32);
  const long long gwarps = runs < glim ? (runs < 1 ? 1 : runs) : glim;
  k_prepass_gen<<<(unsigned)((gwarps + kGenThreads / 32 - 1) / (kGenThreads / 32)), kGenThreads, 0,
                  st>>>(cat, g, tb, thr_kappa, thr_live, acc, rep, cd, rs);
  if (rep.nbins > 0)
    k_fold_replicas<<<(unsigned)((rep.nbins + 255) / 256), 256, 0, st>>>(acc, rep);
}

__global__ void k_set_catalog(CatalogRef* p, CatalogRef v) { *p = v; }

void launch_set_catalog(CatalogRef* p, const CatalogRef& v, cudaStream_t st) {
  k_set_catalog<<<1, 1, 0, st>>>(p, v);
}

// ---------------------------------------------------------------- generated catalogs
// The recipe's constants for the power law f^-gamma and Gamma(shape, 1), computed on the device
// (so that no host compiler contracts them into fused multiply-adds).
__device__ GenParams gen_setup(unsigned long long seed, double gamma, double shape) {
  GenParams g;
  g.k0 = (unsigned)seed;
  g.k1 = (unsigned)(seed >> 32);
  const float e = __double2float_rn(__dsub_rn(1.0, gamma));
  const float lmin = gen_log(__double2float_rn(1e-4)), lmax = gen_log(__double2float_rn(1e-2));
  g.power = fabs(__dsub_rn(gamma, 1.0)) >= 1e-3 ? 1 : 0;
  const float lf0 = e < 0.0f ? lmin : lmax, lf1 = e < 0.0f ? lmax : lmin;
  g.lf0 = lf0;
  g.rho = g.power ? gen_exp(__fmul_rn(e, __fsub_rn(lf1, lf0))) : 0.0f;
  g.omr = __fsub_rn(1.0f, g.rho);
  g.inv_e = g.power ? __fdiv_rn(1.0f, e) : 0.0f;
  g.lmin = lmin;
  g.span = __fsub_rn(lmax, lmin);
  g.d = __fsub_rn(__double2float_rn(shape), (float)(1.0 / 3.0));
  g.c = __fdiv_rn(1.0f, __fsqrt_rn(__fmul_rn(9.0f, g.d)));
  g.pref = __fmul_rn((float)19.2, gen_exp(__fmul_rn((float)(8.0 / 3.0),
                                                    gen_log((float)3.141592653589793))));
  g.log1e3 = gen_log((float)1e-3);
  g.kind = 0;
  g.beta = g.alpha = g.gln = g.mu_g = g.mu = g.sigma = g.rho_cop = g.rho_c = 0.0f;
  return g;
}

__device__ void gen_publish(CatalogRef* ref, long long n, const GenParams& g, const double* A,
                            const double* f, const double* fdot) {
  CatalogRef r;
  r.A = A;
  r.f = f;
  r.fdot = fdot;
  r.n = n;
  r.staged = A ? kCatDevice : kCatGenerated;
  r.pad = 0;
  r.gen = g;
  *ref = r;
}

__global__ void k_gen_setup(CatalogRef* ref, long long n, unsigned long long seed, double gamma,
                            double shape, const double* A, const double* f, const double* fdot) {
  gen_publish(ref, n, gen_setup(seed, gamma, shape), A, f, fdot);
}

// The paper's population: the power law p(f) ~ f^alpha_pl (gamma = -alpha_pl), Gamma of shape
// alpha_g, and the copula, amplitude and rate constants.
__global__ void k_gen_setup_paper(CatalogRef* ref, long long n, unsigned long long seed,
                                  PaperPop pp, const double* A, const double* f,
                                  const double* fdot) {
  GenParams g = gen_setup(seed, -pp.alpha_pl, pp.alpha_g);
  g.kind = 1;
  g.beta = __double2float_rn(pp.beta_g);
  g.alpha = __double2float_rn(pp.alpha_g);
  g.gln = gen_lgamma(g.alpha);
  g.mu_g = __double2float_rn(pp.mu_g);
  g.mu = __double2float_rn(pp.mu);
  g.sigma = __double2float_rn(pp.sigma);
  g.rho_cop = __double2float_rn(pp.rho);
  g.rho_c = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(g.rho_cop, g.rho_cop)));
  gen_publish(ref, n, g, A, f, fdot);
}

void launch_gen_setup(CatalogRef* ref, long long n, unsigned long long seed, double gamma,
                      double shape, const double* A, const double* f, const double* fdot,
                      cudaStream_t st) {
  k_gen_setup<<<1, 1, 0, st>>>(ref, n, seed, gamma, shape, A, f, fdot);
}

void launch_gen_setup_paper(CatalogRef* ref, long long n, unsigned long long seed,
                            const PaperPop& pp, const double* A, const double* f,
                            const double* fdot, cudaStream_t st) {
  k_gen_setup_paper<<<1, 1, 0, st>>>(ref, n, seed, pp, A, f, fdot);
}

__global__ void __launch_bounds__(256) k_generate(const CatalogRef* __restrict__ ref,
                                                  long long start, long long n,
                                                  double* __restrict__ A, double* __restrict__ f,
                                                  double* __restrict__ fdot) {
  const GenParams g = ref->gen;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double a, fs, fd;
    gen_source(g, start + i, &a, &fs, &fd);
    A[i] = a;
    f[i] = fs;
    fdot[i] = fd;
  }
}

void launch_generate(const CatalogRef* ref, long long start, long long n, double* A, double* f,
                     double* fdot, cudaStream_t st) {
  if (n <= 0) return;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  long long want = (n + 255) / 256, cap = (long long)(nsm > 0 ? nsm : 1) * 8;
  k_generate<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(ref, start, n, A, f, fdot);
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

// Sum over the CTA of every thread's count c (0 <= c <= cmax, cmax the same in every thread),
// by barrier reductions of its bits: a barrier, and no shared memory.
__device__ __forceinline__ int cta_count(int c, int cmax) {
  int total = 0;
  for (int bit = 0; (1 << bit) <= cmax; ++bit) total += __syncthreads_count((c >> bit) & 1) << bit;
  return total;
}

// ============================================================================ chunk sort
// Chunks of Kc >= W consecutive bins: any window of at most W bins lies in at most two
// consecutive chunks.  Each chunk is sorted once (keys: the bits of the non-negative
// doubles, whose integer order is their value order; ties broken by position); srank
// maps a position to its sorted index.

// Sort key of a value x >= 0 (a negative value or -0.0 sorts as zero): the bits of the
// double (FP64 path), or of the float nearest to x * scale (mixed precision; scale is a
// power of two that brings the powers, ~1e-50 .. 1e-30, into the FP32 range).  For
// non-negative numbers the integer order of the bits is their value order.
template <typename K>
__device__ __forceinline__ K sort_key(double x, double scale);
template <>
__device__ __forceinline__ u64 sort_key<u64>(double x, double) {
  u64 k = (u64)__double_as_longlong(x);
  return (k >> 63) ? 0ull : k;
}
template <>
__device__ __forceinline__ uint32_t sort_key<uint32_t>(double x, double scale) {
  uint32_t k = __float_as_uint(__double2float_rn(__dmul_rn(x, scale)));
  return (k >> 31) ? 0u : k;
}
// The value a key stands for (inv_scale = 1 / scale, exact).
template <typename K>
__device__ __forceinline__ double key_value(K k, double inv_scale);
template <>
__device__ __forceinline__ double key_value<u64>(u64 k, double) {
  return __longlong_as_double((i64)k);
}
template <>
__device__ __forceinline__ double key_value<uint32_t>(uint32_t k, double inv_scale) {
  return __dmul_rn((double)__uint_as_float(k), inv_scale);
}

// Bitonic sort of (key, position) with E consecutive elements per thread: stages whose
// partners are less than E apart run in registers, less than 32 E apart through warp
// shuffles, and only the longest ones through shared memory (a barrier per stage).
template <typename K>
__device__ __forceinline__ void cmp_keep(K& k, int& x, K ko, int xo, bool keep_min) {
  const bool gt = (k > ko) || (k == ko && x > xo);  // this element after the other one
  if (gt == keep_min) {
    k = ko;
    x = xo;
  }
}

// Re-sort of a chunk whose values changed at few positions since it was last sorted (the
// iterations after the first remove a few sources each).  The unchanged elements keep their
// relative order.  An unchanged element's new index is its old index, less the changed
// elements before it in the old order, plus the changed elements whose new (key, position)
// precede it; a changed element's new index is its rank among the changed elements plus the
// unchanged elements that precede it, found by a binary search of the old order.  This is
// the (key, position) order the full sort produces, so the two paths write the same arrays.
// Returns false, having written nothing, when more than kResortMax positions changed.
constexpr int kResortMax = 128;

template <typename K>
__device__ __forceinline__ bool key_pos_less(K ka, int pa, K kb, int pb) {
  return ka < kb || (ka == kb && pa < pb);
}

template <int E, typename K>
__device__ bool resort_few_changes(const K (&knew)[E], const K (&kold)[E], const int (&rold)[E],
                                   int len, int kpad, K* __restrict__ skey_c,
                                   uint16_t* __restrict__ srank_c, unsigned char* raw) {
  K* old_k = (K*)raw;                                // [kpad] old keys, in old sorted order
  K* ch_k = old_k + kpad;                            // [kResortMax] changed: new keys
  K* cs_k = ch_k + kResortMax;                       // [kResortMax] the same, sorted
  uint16_t* old_p = (uint16_t*)(cs_k + kResortMax);  // [kpad] position of each old index
  uint16_t* csum = old_p + kpad;                     // [kpad + 2] changed before an old index
  uint16_t* ch_p = csum + kpad + 2;                  // [kResortMax] changed: positions
  uint16_t* cs_p = ch_p + kResortMax;                // [kResortMax] the same, sorted
  unsigned char* chg = (unsigned char*)(cs_p + kResortMax);  // [kpad] changed, by position
  __shared__ int n_changed;
  __shared__ int bad_state;
  __shared__ int warp_sum[32];
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, wid = tid >> 5;
  // 1. the old sorted state of the chunk (an index out of range, which a consistent state
  // never holds, sends the chunk to the full sort)
  if (tid == 0) {
    n_changed = 0;
    bad_state = 0;
  }
  // (the caller loaded this thread's old keys kold and sorted indices rold, of indices and
  // positions tid E + a, beside the new values)
  int r[E];
#pragma unroll
  for (int a = 0; a < E; ++a) {
    const int p = tid * E + a;
    if (p < len) old_k[p] = kold[a];
    r[a] = p < len ? rold[a] : 0;
    if (r[a] >= len) {
      bad_state = 1;
      r[a] = 0;
    }
  }
  __syncthreads();
  if (bad_state) {
    __syncthreads();  // every thread has read the flag
    return false;
  }
#pragma unroll
  for (int a = 0; a < E; ++a) {
    const int p = tid * E + a;
    if (p < len) old_p[r[a]] = (uint16_t)p;
  }
  __syncthreads();
  // 2. positions whose key changed, gathered in any order
#pragma unroll
  for (int a = 0; a < E; ++a) {
    const int p = tid * E + a;
    const bool c = p < len && knew[a] != old_k[r[a]];
    chg[p] = c ? 1 : 0;
    if (c) {
      const int slot = atomicAdd(&n_changed, 1);
      if (slot < kResortMax) {
        ch_k[slot] = knew[a];
        ch_p[slot] = (uint16_t)p;
      }
    }
  }
  __syncthreads();
  const int C = n_changed;
  __syncthreads();  // every thread has read the count before the caller reuses shared memory
  if (C > kResortMax) return false;
  if (C == 0) return true;
  // 3. csum[i] = changed elements among old indices < i (exclusive scan in old order)
  int f[E], run = 0;
#pragma unroll
  for (int a = 0; a < E; ++a) {
    const int i = tid * E + a;
    f[a] = i < len ? chg[old_p[i] & (kpad - 1)] : 0;
    run += f[a];
  }
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = T >> 5;
    int v = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) warp_sum[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  int ex = incl - run + (wid > 0 ? warp_sum[wid - 1] : 0);
#pragma unroll
  for (int a = 0; a < E; ++a) {
    const int i = tid * E + a;
    if (i < len) csum[i] = (uint16_t)ex;
    ex += f[a];
  }
  if (tid == 0) csum[len] = (uint16_t)C;
  __syncthreads();
  // 4. changed elements: rank among themselves, plus the unchanged ones before them
  for (int t = tid; t < C; t += T) {
    const K ke = ch_k[t];
    const int pe = ch_p[t];
    int crank = 0;
    for (int u = 0; u < C; ++u) crank += key_pos_less<K>(ch_k[u], ch_p[u], ke, pe) ? 1 : 0;
    int lo = 0, hi = len;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (key_pos_less<K>(old_k[mid], old_p[mid], ke, pe))
        lo = mid + 1;
      else
        hi = mid;
    }
    const int ni = crank + lo - (int)csum[lo];
    cs_k[crank] = ke;
    cs_p[crank] = (uint16_t)pe;
    if (ni < len) {  // always, for a consistent old state
      skey_c[ni] = ke;
      srank_c[pe] = (uint16_t)ni;
    }
  }
  __syncthreads();
  // 5. unchanged elements: old index, less the changed before, plus the changed below them
#pragma unroll
  for (int a = 0; a < E; ++a) {
    const int i = tid * E + a;
    if (i < len && !f[a]) {
      const K ki = old_k[i];
      const int pi = old_p[i];
      int lo = 0, hi = C;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_pos_less<K>(cs_k[mid], cs_p[mid], ki, pi))
          lo = mid + 1;
        else
          hi = mid;
      }
      const int ni = i - (int)csum[i] + lo;
      if (ni < len && pi < len) {  // always, for a consistent old state
        skey_c[ni] = ki;
        srank_c[pi] = (uint16_t)ni;
      }
    }
  }
  return true;
}

template <int E, typename K>
__global__ void __launch_bounds__(1024) k_chunk_sort(SpecIn in, long long n, SmoothPlan pl,
                                                     K* __restrict__ skey,
                                                     uint16_t* __restrict__ srank, Dirty d) {
  extern __shared__ __align__(16) unsigned char sort_raw[];
  K* sm_keys = (K*)sort_raw;
  uint16_t* sm_idx = (uint16_t*)(sm_keys + pl.kpad);
  const int T = blockDim.x, tid = threadIdx.x;
  const int kpad = pl.kpad;  // = T * E
  const ListHead head = list_head(d, kListR0, pl.nch);
  const int nitem = head.count;
  // after the first iteration of a tracked run every chunk holds the sorted state of its
  // previous values
  const bool resort = d.base != nullptr && head.iter > 0;
  int b_next = head.first;
  for (int item = blockIdx.x; item < nitem; item += gridDim.x) {
    const int b = b_next;  // a chunk whose input changed
    if (item + (int)gridDim.x < nitem) b_next = d.item(kListR0, item + gridDim.x);
    const long long base = (long long)b * pl.Kc;
    const int len = (int)((n - base) < pl.Kc ? (n - base) : pl.Kc);
    K k[E], kold[E];
    int x[E], rold[E];
    // the previous sorted state, loaded beside the new values
#pragma unroll
    for (int a = 0; a < E; ++a) {
      const int i = tid * E + a;
      kold[a] = (resort && i < len) ? skey[base + i] : (K)0;
      rold[a] = (resort && i < len) ? (int)srank[base + i] : 0;
    }
#pragma unroll
    for (int a = 0; a < E; ++a) {
      const int i = tid * E + a;
      K kv = (K)~(K)0;
      if (i < len) kv = sort_key<K>(spec_value(in, base + i), pl.key_scale);
      k[a] = kv;
      x[a] = i;
    }
    if (resort &&
        resort_few_changes<E, K>(k, kold, rold, len, kpad, skey + base, srank + base, sort_raw)) {
      __syncthreads();  // before the next chunk overwrites shared memory
      continue;
    }
    // a chunk of zeros (no power in it: much of the band's high-frequency end before any
    // removal) is sorted already: every key 0, ties in position order; a chunk with few
    // nonzero bins is that order with the few merged in (the re-sort from an all-zero state)
    {
      int nzc = 0;
#pragma unroll
      for (int a = 0; a < E; ++a) nzc += ((tid * E + a < len) && k[a] != (K)0) ? 1 : 0;
      const int nzt = cta_count(nzc, E);
      if (nzt == 0) {
#pragma unroll
        for (int a = 0; a < E; ++a) {
          const int i = tid * E + a;
          if (i < len) {
            skey[base + i] = (K)0;
            srank[base + i] = (uint16_t)i;
          }
        }
        continue;
      }
      if (nzt <= kResortMax) {
        K kz[E];
        int rid[E];
#pragma unroll
        for (int a = 0; a < E; ++a) {
          kz[a] = (K)0;
          rid[a] = tid * E + a < len ? tid * E + a : 0;
        }
        if (resort_few_changes<E, K>(k, kz, rid, len, kpad, skey + base, srank + base,
                                     sort_raw)) {
          __syncthreads();  // before the next chunk overwrites shared memory
          continue;
        }
      }
    }
    bool first_smem = true;
    for (int kk = 2; kk <= kpad; kk <<= 1) {
      int jj = kk >> 1;
      if (jj >= 32 * E) {
        if (!first_smem) __syncthreads();  // everyone has read the previous round back
        first_smem = false;
#pragma unroll
        for (int a = 0; a < E; ++a) {
          sm_keys[tid * E + a] = k[a];
          sm_idx[tid * E + a] = (uint16_t)x[a];
        }
        __syncthreads();
        for (; jj >= 32 * E; jj >>= 1) {
          for (int q = tid; q < kpad / 2; q += T) {
            const int i = ((q & ~(jj - 1)) << 1) | (q & (jj - 1));
            const int ixj = i | jj;
            K ki = sm_keys[i], kj = sm_keys[ixj];
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
          __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < E; ++a) {
          k[a] = sm_keys[tid * E + a];
          x[a] = sm_idx[tid * E + a];
        }
      }
      for (; jj >= E; jj >>= 1) {
        const int lm = jj / E;  // partner lane offset (< 32)
#pragma unroll
        for (int a = 0; a < E; ++a) {
          const int i = tid * E + a;
          const K ko = __shfl_xor_sync(0xFFFFFFFFu, k[a], lm);
          const int xo = __shfl_xor_sync(0xFFFFFFFFu, x[a], lm);
          const bool lower = (i & jj) == 0, asc = (i & kk) == 0;
          cmp_keep<K>(k[a], x[a], ko, xo, lower == asc);
        }
      }
      // in-thread stages: distances E/2 .. 1 (those below kk), unrolled so that the
      // element arrays stay in registers
#pragma unroll
      for (int jl = E / 2; jl >= 1; jl >>= 1) {
        if (jl > (kk >> 1)) continue;
#pragma unroll
        for (int a = 0; a < E; ++a) {
          if ((a & jl) == 0) {
            const int c = a | jl;
            const int i = tid * E + a;
            const bool asc = (i & kk) == 0;
            const K ka = k[a], kc = k[c];
            const int xa = x[a], xc = x[c];
            const bool gt = (ka > kc) || (ka == kc && xa > xc);
            if (gt == asc) {
              k[a] = kc;
              k[c] = ka;
              x[a] = xc;
              x[c] = xa;
            }
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < E; ++a) {
      const int sidx = tid * E + a;
      if (sidx < len) {
        skey[base + sidx] = k[a];
        srank[base + x[a]] = (uint16_t)sidx;
      }
    }
    if (!first_smem) __syncthreads();  // before the next chunk overwrites shared memory
  }
}

// Persistent grid: as many CTAs as fit on the GPU at once (items are dealt out statically,
// so a CTA that had to wait for a free slot would serialise its share), never more than
// the work items.
template <typename K>
static int resident_ctas(const SmoothPlan& pl, K kernel, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return pl.nsm * per_sm;
}
static int persistent_grid(const SmoothPlan& pl, int items, int resident) {
  if (pl.nsm <= 0 || resident <= 0) return items;
  return items < resident ? items : resident;
}

// Launch one k_chunk_sort instantiation with the key buffer cast to its key type.
template <typename K>
static void launch_sort_as(void (*kern)(SpecIn, long long, SmoothPlan, K*, uint16_t*, Dirty),
                           int bl, int th, size_t smem, cudaStream_t st, SpecIn in, long long n,
                           const SmoothPlan& pl, unsigned long long* skey, uint16_t* srank,
                           Dirty d) {
  kern<<<bl, th, smem, st>>>(in, n, pl, (K*)skey, srank, d);
}

static int sort_per_thread(const SmoothPlan& pl) {
  if (pl.sort_e) return pl.sort_e;
  return pl.kpad <= 2048 ? 2 : pl.kpad / 1024;
}
static int sort_threads(const SmoothPlan& pl) { return pl.kpad / sort_per_thread(pl); }
static size_t sort_smem(const SmoothPlan& pl) {
  const size_t kb = pl.fp32_keys ? 4 : 8;
  const size_t full = (size_t)pl.kpad * (kb + sizeof(uint16_t));
  const size_t few = (size_t)pl.kpad * (kb + 2 + 1) + (size_t)(pl.kpad + 2) * 2 +
                     (size_t)kResortMax * 2 * (kb + 2);
  return full > few ? full : few;
}
template <typename K, typename F>
static void with_sort_kernel_k(const SmoothPlan& pl, F fn) {
  switch (sort_per_thread(pl)) {
    case 2: fn(k_chunk_sort<2, K>); break;
    case 4: fn(k_chunk_sort<4, K>); break;
    default: fn(k_chunk_sort<8, K>); break;
  }
}
template <typename F>
static void with_sort_kernel(const SmoothPlan& pl, F fn) {
  if (pl.fp32_keys)
    with_sort_kernel_k<uint32_t>(pl, fn);
  else
    with_sort_kernel_k<u64>(pl, fn);
}

void launch_chunk_sort(SpecIn in, long long n, const SmoothPlan& pl, unsigned long long* skey,
                       uint16_t* srank, Dirty d, cudaStream_t st) {
  const size_t smem = sort_smem(pl);
  const int th = sort_threads(pl);
  const int bl = persistent_grid(pl, pl.nch, pl.res_sort);
  with_sort_kernel(pl, [&](auto kern) {
    launch_sort_as(kern, bl, th, smem, st, in, n, pl, skey, srank, d);
  });
}

// ============================================================================ running median
// Tile u (u = 0 .. nch) produces the outputs j in [(u-1) Kc + h, u Kc + h), h = W/2.
// Their windows [s(j), e(j)] = [max(0, j - h), min(n-1, j - h + W - 1)] lie in the 2 Kc
// bins of chunks u-1 and u (W <= Kc): the tile's span.  One CTA per tile
//  1. merges the two sorted chunks, so that every position p of the span gets its rank
//     v(p) in the merged order (key, then position): a permutation of 0 .. 2Kc-1, bins
//     outside the band taking the top ranks (they are never inside a window);
//  2. builds a wavelet matrix of v over the positions: level l (l = 0 .. LV-1) stores bit
//     LV-1-l of the ranks in the order the stable partitions (zeros first) of the levels
//     above left them, as bitset words with exclusive prefix counts of their ones;
//  3. answers, one thread per output, "k-th smallest rank among positions [s, e]" by LV
//     descents of two rank lookups each, for k = c/2 (the upper median of c bins) and
//     k = c/2 - 1 (the lower one, used when c is even).
// Both results are elements of the window, so the median (App. D, Eq. running median)
// is a selection, exact whatever the order of the arithmetic; the ranks only say which
// element is selected.  Every output costs O(log Kc) independent of its neighbours, so
// a tile's latency is a few thousand cycles even when a single chunk has changed.

__device__ __forceinline__ int wm_levels(int M) { return 32 - __clz(M - 1); }
// Ones of the warps before this one (run) and of all of them (total), from the per-warp
// counts c (lane i holds warp i's, zero beyond the warps).
__device__ __forceinline__ void wm_warp_offsets(int c, int warp, int* run, int* total) {
  const int lane = threadIdx.x & 31;
  *total = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)c);
  *run = (int)__reduce_add_sync(0xFFFFFFFFu, lane < warp ? (unsigned)c : 0u);
}

__device__ __forceinline__ unsigned lds_u16(uint32_t addr) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_u16(uint32_t addr, unsigned v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"((unsigned short)v) : "memory");
}

// Wavelet matrix of the permutation seq0 (M elements) when every warp owns exactly WPW words
// of a level: each level loads the warp's elements once, all of them before the first ballot,
// and the ballots serve both the count and the stable partition into the other buffer.
// Level l stores its words in rk[l ws ..] (bits in the low half, ones of the earlier words
// in the high half) and its number of zeros in zeros[l].  seq0 and seq1 are both
// overwritten.
template <int WPW>
__device__ __forceinline__ void wm_build_fixed(uint16_t* seq0, uint16_t* seq1, u64* rk, int ws,
                                               int* zeros, int* warp_ones, int M, int LV,
                                               int nwm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int w0 = warp * WPW;
  const unsigned below = (1u << lane) - 1u;
  uint32_t cur = (uint32_t)__cvta_generic_to_shared(seq0);
  uint32_t nxt = (uint32_t)__cvta_generic_to_shared(seq1);
  for (int l = 0; l < LV; ++l) {
    const int sh = LV - 1 - l;
    u64* rkl = rk + (size_t)l * ws;
    uint32_t xv[WPW];
    unsigned bal[WPW];
    int mine = 0;
#pragma unroll
    for (int q = 0; q < WPW; ++q) xv[q] = lds_u16(cur + 2u * (uint32_t)((w0 + q) * 32 + lane));
#pragma unroll
    for (int q = 0; q < WPW; ++q) {
      bal[q] = __ballot_sync(0xFFFFFFFFu, (xv[q] >> sh) & 1u);
      mine += __popc(bal[q]);
    }
    if (lane == 0) warp_ones[warp] = mine;
    __syncthreads();
    int run, total;
    wm_warp_offsets(lane < nwarp ? warp_ones[lane] : 0, warp, &run, &total);
    const int Z = M - total;
#pragma unroll
    for (int q = 0; q < WPW; ++q) {
      const int k = w0 + q;
      if (lane == 0) rkl[k] = ((u64)run << 32) | bal[q];
      if (l + 1 < LV) {
        const int ob = run + __popc(bal[q] & below);
        const int dst = ((xv[q] >> sh) & 1u) ? Z + ob : k * 32 + lane - ob;
        sts_u16(nxt + 2u * (uint32_t)dst, xv[q]);
      }
      run += __popc(bal[q]);
    }
    if (tid == 0) {
      rkl[nwm] = (u64)total << 32;
      zeros[l] = Z;
    }
    __syncthreads();
    const uint32_t t = cur;
    cur = nxt;
    nxt = t;
  }
}

// The same for any number of words per warp (the last warps may own fewer, or none).
__device__ __forceinline__ void wm_build_any(uint16_t* seq0, uint16_t* seq1, u64* rk, int ws,
                                             int* zeros, int* warp_ones, int M, int LV,
                                             int nwm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int wpw = (nwm + nwarp - 1) / nwarp;
  const int w0 = warp * wpw, w1 = min(w0 + wpw, nwm);
  uint16_t* cur = seq0;
  uint16_t* nxt = seq1;
  for (int l = 0; l < LV; ++l) {
    const int sh = LV - 1 - l;
    u64* rkl = rk + (size_t)l * ws;
    int mine = 0;
    for (int k = w0; k < w1; ++k)
      mine += __popc(__ballot_sync(0xFFFFFFFFu, (cur[k * 32 + lane] >> sh) & 1));
    if (lane == 0) warp_ones[warp] = mine;
    __syncthreads();
    int run, total;
    wm_warp_offsets(lane < nwarp ? warp_ones[lane] : 0, warp, &run, &total);
    const int Z = M - total;
    for (int k = w0; k < w1; ++k) {
      const int i = k * 32 + lane;
      const int x = cur[i];
      const int b = (x >> sh) & 1;
      const unsigned bits = __ballot_sync(0xFFFFFFFFu, b);
      if (lane == 0) rkl[k] = ((u64)run << 32) | bits;
      if (l + 1 < LV) {
        const int ob = run + __popc(bits & ((1u << lane) - 1u));
        nxt[b ? Z + ob : i - ob] = (uint16_t)x;
      }
      run += __popc(bits);
    }
    if (tid == 0) {
      rkl[nwm] = (u64)total << 32;
      zeros[l] = Z;
    }
    __syncthreads();
    uint16_t* t = cur;
    cur = nxt;
    nxt = t;
  }
}

// Ones of a level's bitset before position i (the word holds its bits in the low half and
// the ones of all earlier words in the high half).
__device__ __forceinline__ int wm_rank1(const u64* rkl, int i) {
  const u64 e = rkl[i >> 5];
  return (int)(e >> 32) + __popc((uint32_t)e & ((1u << (i & 31)) - 1u));
}

// One tile; returns the largest relative change of S_n among its outputs (conv_rtol).
template <typename K>
__device__ __forceinline__ double median_tile(const K* __restrict__ skey,
                                              const uint16_t* __restrict__ srank, long long n,
                                              const SmoothPlan& pl, const SgOut& o, long long u,
                                              unsigned char* sm_raw, int* zeros) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int Kc = pl.Kc, M = 2 * Kc, LV = wm_levels(M);
  const int nwm = M >> 5, ws = nwm + 1;  // words per level (one zero word of padding)
  const int h = pl.W / 2;
  long long j_lo = (u - 1) * Kc + h, j_hi = u * Kc + h;
  if (j_lo < 0) j_lo = 0;
  if (j_hi > n) j_hi = n;
  if (j_lo >= j_hi) return 0.0;
  const double inv_scale = 1.0 / pl.key_scale;  // exact: a power of two
  const long long span = (u - 1) * (long long)Kc;
  int len0 = 0, len1 = 0;
  if (u >= 1) len0 = (n - span) < Kc ? (int)(n - span) : Kc;
  if (u < pl.nch) len1 = (n - span - Kc) < Kc ? (int)(n - span - Kc) : Kc;
  double relmax = 0.0;
  K* sk = (K*)sm_raw;                                        // [M] sorted keys (step 1)
  uint16_t* seq1 = (uint16_t*)sm_raw;                        // [M] (steps 2-3, over sk)
  uint16_t* src = seq1 + M;                                  // [M] rank -> element
  uint16_t* seq0 = (uint16_t*)(sm_raw + sizeof(K) * (size_t)M);  // [M]
  // [LV][ws]: per bitset word, its 32 bits (low half) and the ones before it (high half),
  // so that a rank is one 64-bit load
  u64* rk = (u64*)(seq0 + M);
  uint16_t* mr = (uint16_t*)rk;  // [M] merged index of (chunk, sorted index) (step 1, over rk)
  __shared__ int warp_ones[32];

  // 1. merged ranks.  Chunk u-1 precedes chunk u on equal keys (its positions are lower).
  int nzc = 0;  // this thread's nonzero keys of the span
  for (int i = tid; i < len0; i += T) {
    const K v = skey[span + i];
    sk[i] = v;
    nzc += v != (K)0 ? 1 : 0;
  }
  for (int i = tid; i < len1; i += T) {
    const K v = skey[span + Kc + i];
    sk[Kc + i] = v;
    nzc += v != (K)0 ? 1 : 0;
  }
  // Every window lies in the span; a window of c bins with fewer than ceil(c / 2) nonzero
  // values has a zero median (both middle elements are zeros).  The smallest window of
  // the tile is at one of its ends.
  auto win = [&](long long j) {
    const long long s0 = j - h > 0 ? j - h : 0;
    const long long e0 = j - h + pl.W - 1 < n - 1 ? j - h + pl.W - 1 : n - 1;
    return (int)(e0 - s0 + 1);
  };
  const int cmin = min(win(j_lo), win(j_hi - 1));
  const int nzt = cta_count(nzc, 2 * ((Kc + T - 1) / T));  // a thread loads at most that many
  if (nzt < (cmin + 1) / 2) {
    // every window's median is 0
    const int nz_out = (int)(j_hi - j_lo);
    for (int t = tid; t < nz_out; t += T) {
      const double rel = sg_store(o, j_lo + t, __dmul_rn(kMedianBias, 0.0));
      relmax = rel > relmax ? rel : relmax;
    }
    return relmax;
  }
  {
    // merge path: thread t emits the merged indices [d0, d1) of the two sorted chunks,
    // starting where a binary search on the diagonal d0 puts it
    const int L = len0 + len1, per = (L + T - 1) / T;
    const int d0 = min(tid * per, L), d1 = min(d0 + per, L);
    if (d0 < d1) {
      const K* A = sk;
      const K* B = sk + Kc;
      int lo = max(0, d0 - len1), hi = min(d0, len0);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] <= B[d0 - 1 - mid])
          lo = mid + 1;
        else
          hi = mid;
      }
      int i = lo, j = d0 - lo;
      for (int m = d0; m < d1; ++m) {
        if (i < len0 && (j >= len1 || A[i] <= B[j]))
          mr[i++] = (uint16_t)m;
        else
          mr[Kc + j++] = (uint16_t)m;
      }
    }
  }
  __syncthreads();
  for (int p = tid; p < M; p += T) {
    const int X = p >= Kc, q = p - X * Kc;
    int v;
    if (q < (X ? len1 : len0)) {
      const int si = srank[span + p];
      v = mr[X * Kc + si];
      src[v] = (uint16_t)((X << 15) | si);
    } else {
      v = len0 + len1 + (X ? (Kc - len0) + (q - len1) : (q - len0));
    }
    seq0[p] = (uint16_t)v;
  }
  __syncthreads();

  // 2. wavelet matrix.  Warp w owns the words [w wpw, (w + 1) wpw) of every level (M is a
  // multiple of 64: whole words).  A level takes two barriers: one after the warps have
  // counted their ones, one after the stable partition.
  {
    const int nwarp = T >> 5;
    const int wpw = (nwm + nwarp - 1) / nwarp;
    const bool full = wpw * nwarp == nwm;
    if (full && wpw == 4)
      wm_build_fixed<4>(seq0, seq1, rk, ws, zeros, warp_ones, M, LV, nwm);
    else if (full && wpw == 2)
      wm_build_fixed<2>(seq0, seq1, rk, ws, zeros, warp_ones, M, LV, nwm);
    else if (full && wpw == 8)
      wm_build_fixed<8>(seq0, seq1, rk, ws, zeros, warp_ones, M, LV, nwm);
    else if (full && wpw == 1)
      wm_build_fixed<1>(seq0, seq1, rk, ws, zeros, warp_ones, M, LV, nwm);
    else
      wm_build_any(seq0, seq1, rk, ws, zeros, warp_ones, M, LV, nwm);
  }

  // 3. selections
  const int nout = (int)(j_hi - j_lo);
  for (int t = tid; t < nout; t += T) {
    const long long j = j_lo + t;
    const long long s = j - h > 0 ? j - h : 0;
    const long long e = j - h + pl.W - 1 < n - 1 ? j - h + pl.W - 1 : n - 1;
    const int cnt = (int)(e - s + 1);
    // two descents side by side: a = upper median (k = c/2), b = lower (k = c/2 - 1)
    int la = (int)(s - span), ra = (int)(e + 1 - span), ka = cnt >> 1, va = 0;
    int lb = la, rb = ra, kb = ka > 0 ? ka - 1 : 0, vb = 0;
    for (int l = 0; l < LV; ++l) {
      const u64* rkl = rk + (size_t)l * ws;
      const int Z = zeros[l];
      const int oal = wm_rank1(rkl, la);
      const int oar = wm_rank1(rkl, ra);
      // the two order statistics are neighbours: their descents share a node at most
      // levels, and then share its ranks
      int obl = oal, obr = oar;
      if (__any_sync(__activemask(), la != lb || ra != rb)) {  // lanes still in the loop
        obl = wm_rank1(rkl, lb);
        obr = wm_rank1(rkl, rb);
      }
      const int za = (ra - oar) - (la - oal), zb = (rb - obr) - (lb - obl);
      const int bit = 1 << (LV - 1 - l);
      if (ka < za) {
        la -= oal;
        ra -= oar;
      } else {
        ka -= za;
        la = Z + oal;
        ra = Z + oar;
        va |= bit;
      }
      if (kb < zb) {
        lb -= obl;
        rb -= obr;
      } else {
        kb -= zb;
        lb = Z + obl;
        rb = Z + obr;
        vb |= bit;
      }
    }
    const int ea = src[va];
    const K khi = skey[span + (ea >> 15) * Kc + (ea & 0x7FFF)];
    double med;
    if (cnt & 1) {
      med = key_value<K>(khi, inv_scale);
    } else {
      const int eb = src[vb];
      const K klo = skey[span + (eb >> 15) * Kc + (eb & 0x7FFF)];
      med = __dmul_rn(__dadd_rn(key_value<K>(klo, inv_scale), key_value<K>(khi, inv_scale)),
                      0.5);
    }
    double v = __dmul_rn(kMedianBias, med);
    double rel = sg_store(o, j, v);
    relmax = rel > relmax ? rel : relmax;
  }
  return relmax;
}

template <typename K>
__global__ void __launch_bounds__(512, 2) k_median_wm(
    const K* __restrict__ skey, const uint16_t* __restrict__ srank,
    long long n, SmoothPlan pl, SgOut o, Dirty d) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int zeros[16];
  double relmax = 0.0;
  const ListHead head = list_head(d, kListTile, pl.nch + 1);
  const int nitem = head.count;
  int u_next = head.first;
  for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
    // a tile whose windows changed
    const int u = u_next;
    if (it + (int)gridDim.x < nitem) u_next = d.item(kListTile, it + gridDim.x);
    double r = median_tile<K>(skey, srank, n, pl, o, u, sm_raw, zeros);
    relmax = r > relmax ? r : relmax;
    __syncthreads();  // before the next tile overwrites shared memory
  }
  if (o.rtol_on) warp_max_atomic((u64)__double_as_longlong(relmax), &o.rs->relchg_bits);
}

static int median_threads(const SmoothPlan& pl) {
  if (pl.median_th) return pl.median_th;
  int t = ((pl.Kc / 2 + 31) / 32) * 32;
  if (t < 32) t = 32;
  if (t > 512) t = 512;
  return t;
}

size_t median_smem_bytes(int Kc, int key_bytes) {
  int M = 2 * Kc, LV = 0;
  while ((1 << LV) < M) ++LV;
  size_t ws = (size_t)M / 32 + 1;
  size_t rk = (size_t)LV * ws * 8, mr = (size_t)2 * M;  // the merged indices sit over rk
  return (size_t)key_bytes * M + (size_t)2 * M + (rk > mr ? rk : mr);
}

void launch_running_median(const unsigned long long* skey, const uint16_t* srank, long long n,
                           const SmoothPlan& pl, SgOut o, Dirty d, cudaStream_t st) {
  int th = median_threads(pl);
  size_t smem = median_smem_bytes(pl.Kc, pl.fp32_keys ? 4 : 8);
  int bl = persistent_grid(pl, pl.nch + 1, pl.res_median);
  if (pl.fp32_keys)
    k_median_wm<uint32_t><<<bl, th, smem, st>>>((const uint32_t*)skey, srank, n, pl, o, d);
  else
    k_median_wm<u64><<<bl, th, smem, st>>>(skey, srank, n, pl, o, d);
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

// Prefix sums of chunk b.
__device__ __forceinline__ void chunk_prefix(const SpecIn& in, long long n, const SmoothPlan& pl,
                                             unsigned long long* __restrict__ pre_lo,
                                             unsigned long long* __restrict__ pre_hi,
                                             int* __restrict__ sig, unsigned* __restrict__ uflow,
                                             double* __restrict__ x_out, int b, U128* warp_tot,
                                             u64* warp_max, int& any_uf) {
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
  if (warp_max[0] == 0ull) {
    // a chunk of zeros: every prefix is 0 and nothing fell below one unit
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < per && p0 + i < len) {
        pre_lo[base + p0 + i] = 0ull;
        pre_hi[base + p0 + i] = 0ull;
      }
    }
    if (threadIdx.x == 0) {
      uflow[b] = 0u;
      sig[b] = sigma;
    }
    return;
  }
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

__global__ void k_chunk_prefix(SpecIn in, long long n, SmoothPlan pl,
                               unsigned long long* __restrict__ pre_lo,
                               unsigned long long* __restrict__ pre_hi, int* __restrict__ sig,
                               unsigned* __restrict__ uflow, double* __restrict__ x_out, Dirty d,
                               int in_radius) {
  __shared__ U128 warp_tot[32];
  __shared__ u64 warp_max[32];
  __shared__ int any_uf;
  // chunks whose input changed (a chunk within in_radius of them is dirty)
  const int list = kListR0 + in_radius;
  const ListHead head = list_head(d, list, pl.nch);
  const int nitem = head.count;
  int b_next = head.first;
  for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
    const int b = b_next;
    if (it + (int)gridDim.x < nitem) b_next = d.item(list, it + gridDim.x);
    chunk_prefix(in, n, pl, pre_lo, pre_hi, sig, uflow, x_out, b, warp_tot,
                 warp_max, any_uf);
    __syncthreads();
  }
}

void launch_chunk_prefix(SpecIn in, long long n, const SmoothPlan& pl, unsigned long long* pre_lo,
                         unsigned long long* pre_hi, int* sig, unsigned* uflow, double* x_out,
                         Dirty d, int in_radius, cudaStream_t st) {
  int th = pl.Kc < 1024 ? pl.Kc : 1024;  // at most 8 values per thread
  int bl = persistent_grid(pl, pl.nch, pl.res_prefix);
  k_chunk_prefix<<<bl, th, 0, st>>>(in, n, pl, pre_lo, pre_hi, sig, uflow, x_out, d, in_radius);
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
  double relmax = 0.0;
  const int h = pl.W / 2;
  const double inv_w = 1.0 / (double)pl.W;
  // output chunks with a dirty chunk within out_radius
  const int list = kListR0 + out_radius;
  const ListHead head = list_head(d, list, pl.nch);
  const int nitem = head.count;
  int b_next = head.first;
  for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
    const long long b = b_next;
    if (it + (int)gridDim.x < nitem) b_next = d.item(list, it + gridDim.x);
    const long long b0 = b * pl.Kc;
    const long long jend = b0 + pl.Kc < n ? b0 + pl.Kc : n;
    for (long long j = b0 + threadIdx.x; j < jend; j += blockDim.x) {
      long long s = j - h > 0 ? j - h : 0;
      long long e = j - h + pl.W - 1 < n - 1 ? j - h + pl.W - 1 : n - 1;
      // s and e lie within one chunk of chunk b (h < W <= Kc): no 64-bit division
      const long long ds = s - b0, de = e - b0;
      const long long cs = b + (ds < 0 ? -1 : (ds >= pl.Kc ? 1 : 0));
      const long long ce = b + (de < 0 ? -1 : (de >= pl.Kc ? 1 : 0));
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
      double v = (cnt == pl.W) ? __dmul_rn(sum, inv_w) : __ddiv_rn(sum, (double)cnt);
      double rel = sg_store(o, j, v);
      relmax = rel > relmax ? rel : relmax;
    }
  }
  if (o.rtol_on) warp_max_atomic((u64)__double_as_longlong(relmax), &o.rs->relchg_bits);
}

// One output of the chunk per thread.
static int mean_threads(const SmoothPlan& pl) { return pl.Kc < 1024 ? pl.Kc : 1024; }

void launch_window_mean(const double* x, long long n, const SmoothPlan& pl,
                        const unsigned long long* pre_lo, const unsigned long long* pre_hi,
                        const int* sig, const unsigned* uflow, SgOut o, Dirty d, int out_radius,
                        cudaStream_t st) {
  int th = mean_threads(pl);
  int bl = persistent_grid(pl, pl.nch, pl.res_mean);
  k_window_mean<<<bl, th, 0, st>>>(x, n, pl, pre_lo, pre_hi, sig, uflow, o, d, out_radius);
}

// ============================================================================ SNR + resolve
// rho^2 = 4 (T/5) A^2 sum_k w_k R_k / (S_k + S_gal,k) = sum_k rho0_k / (1 + S_gal,k / S_k).
// The screen evaluates it in FP32 as sum_k a2f w_k Gf_k inv_f_k; its relative error is
// below 2.2e-6 (FP32 roundings of the inputs, the ratio, the reciprocal and the products of
// each term) + 2e-7 per rounding of the sum that a term passes through: per bin for a sum
// on one lane, and for a sweep summed by a warp the longest lane's count plus the five
// levels of the butterfly (a sum of positive terms loses at most one rounding per step of
// its longest chain).  Outside twice that, 1e-5 + 4e-7 per step, around rho_th^2 the FP64
// decision is known.  Inside it, and always when the caller asks for the strict path,
// rho^2 is recomputed in FP64 with the oracle's terms: on one lane in the oracle's order
// for a sweep of a few bins, by the warp for a longer one.  In the mixed-precision mode the
// FP32 value decides alone.

__device__ __forceinline__ bool rtol_stop(const RunState* rs, double rtol) {
  if (!(rtol > 0.0) || rs->iter < 1) return false;
  double r = __longlong_as_double((i64)rs->relchg_bits);
  return r <= rtol;
}

// rho^2 of a sweep of many bins in FP64 by a whole warp: the same terms as rho2_exact, lane i
// summing the bins k0 + i, k0 + i + 32, ..., then a butterfly (a fixed order; every lane ends
// with the same value).  Its rounding differs from the sequential sum's by a few parts in
// 10^16; a decision that could differ lies within the near-threshold band.
__device__ double rho2_exact_warp(const Grid& g, const Tables& tb, const double* __restrict__ Sg,
                                  double a2, double lo, double hi) {
  const int lane = threadIdx.x & 31;
  Sweep sw;
  sw.lo = lo;
  sw.hi = hi;
  sw.ka = (i64)floor(__dadd_rn(lo, 0.5));
  sw.kb = (i64)floor(__dadd_rn(hi, 0.5));
  const bool single = (sw.ka == sw.kb);
  const long long k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
  const long long k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
  double acc = 0.0;
  for (long long k = k0 + lane; k <= k1; k += 32) {
    const double w = single ? 1.0 : sweep_weight(sw, k);
    if (w > 0.0) {
      const long long j = k - g.k_lo;
      const double sn = __dadd_rn(tb.S[j], Sg[j]);
      const double psk = __dmul_rn(__dmul_rn(__dmul_rn(g.t5, tb.R[j]), a2), w);
      acc = __dadd_rn(acc, __ddiv_rn(psk, sn));
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, o));
  return __dmul_rn(4.0, acc);
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

// FP32 screen sum of candidate c over the bins t0 + off, t0 + off + step, ... < t1 of its
// sweep (t relative to its first bin ka); kcount counts the terms.
__device__ __forceinline__ float screen_part(const Cands& cd, long long c, const int4 pk,
                                             const Grid& g, const Tables& tb,
                                             const float* __restrict__ inv_f, int off, int step,
                                             int& kcount) {
  const int ka = pk.x;
  const int nbin = pk.y;
  const float a2f = __int_as_float(pk.z);
  float r2 = 0.0f;
  kcount = 0;
  if (nbin == 1) {
    if (off == 0 && ka >= 0 && ka < g.nb) {
      r2 = __fmul_rn(__fmul_rn(a2f, tb.Gf[ka]), inv_f[ka]);
      kcount = 1;
    }
    return r2;
  }
  const float flo = __int_as_float(pk.w), len = cd.len[c];
  const float fhi = __fadd_rn(flo, len), invlen = 1.0f / len;
  const int t0 = ka < 0 ? -ka : 0;
  const int t1 = (long long)ka + nbin > g.nb ? (int)(g.nb - ka) : nbin;
  for (int t = t0 + off; t < t1; t += step) {
    float a = fmaxf(flo, (float)t - 0.5f);
    float b = fminf(fhi, (float)t + 0.5f);
    if (b > a) {
      float w = __fmul_rn(__fsub_rn(b, a), invlen);
      int k = ka + t;
      r2 = __fadd_rn(r2, __fmul_rn(__fmul_rn(__fmul_rn(a2f, w), tb.Gf[k]), inv_f[k]));
      ++kcount;
    }
  }
  return r2;
}

// Margin of the screen: the FP32 value is within this relative distance of the FP64 one
// (the bound above, doubled, for kcount bins).
__device__ __forceinline__ float screen_margin(int kcount) {
  return 1e-5f + 4e-7f * (float)kcount;
}

// Decision from the FP32 value: 1 resolve, 0 keep, -1 too close to rho_th to tell (the
// caller then computes rho^2 exactly).
__device__ __forceinline__ int screen_decide(float r2, int kcount, float th2f, int mode) {
  if (mode == 1) return r2 > th2f ? 1 : 0;
  float m = screen_margin(kcount);
  if (mode == 0 && r2 > th2f * (1.0f + m)) return 1;
  if (mode == 0 && r2 < th2f * (1.0f - m)) return 0;
  return -1;
}

// An FP32 decision (mixed precision) that the FP64 value could take the other way.
__device__ __forceinline__ bool screen_uncertain(float r2, int kcount, float th2f) {
  const float m = screen_margin(kcount);
  return r2 <= th2f * (1.0f + m) && r2 >= th2f * (1.0f - m);
}

// An FP64 value of rho^2 with |rho - rho_th| / rho_th < 1e-9, i.e. |rho^2 / rho_th^2 - 1|
// below 2e-9 (to first order): a decision that the order of the FP64 roundings could flip.
__device__ __forceinline__ bool near_threshold(double r2, double th2) {
  return fabs(__dsub_rn(r2, th2)) < __dmul_rn(2e-9, th2);
}

// Remove the parts of candidate c that the catalog pass deposited: bins k0 + off,
// k0 + off + step, ... of its sweep.
__device__ __forceinline__ void remove_part(const Cands& cd, long long c, const Grid& g,
                                            const Tables& tb, unsigned long long* acc,
                                            const DirtyIter& d, int Kc, int off, int step) {
  Sweep sw;
  sw.lo = cd.lo[c];
  sw.hi = cd.hi[c];
  sw.ka = (i64)floor(__dadd_rn(sw.lo, 0.5));
  sw.kb = (i64)floor(__dadd_rn(sw.hi, 0.5));
  const double a2 = cd.a2[c];
  if (sw.ka == sw.kb) {
    long long j = sw.ka - g.k_lo;
    if (off == 0 && j >= 0 && j < g.nb) {
      u64 c0, c1, c2, qb;
      if (q_single(cd.amp[c], tb.gq[j], &c0, &c1, &c2, &qb)) sub_parts(acc, j, c0, c1, c2);
      d.mark_next(j / Kc);
    }
    return;
  }
  long long k0 = sw.ka > g.k_lo ? sw.ka : g.k_lo;
  long long k1 = sw.kb < g.k_lo + g.nb - 1 ? sw.kb : g.k_lo + g.nb - 1;
  const double inv = sweep_inv_len(sw);
  for (long long k = k0 + off; k <= k1; k += step) {
    double w = sweep_weight_inv(sw, k, inv);
    if (w > 0.0) {
      long long j = k - g.k_lo;
      remove_q(acc, j, __dmul_rn(__dmul_rn(a2, w), tb.gq[j]));
      d.mark_next(j / Kc);
    }
  }
}

// Every lane screens one candidate of a group of 32: still unresolved, and S_n changed on
// a bin of its sweep (else rho is the value already found below rho_th).  Candidates of a
// few bins are done by their own lane.  Longer sweeps (loud high-frequency sources cover up
// to hundreds of bins, and more) come from their own list, one per warp in turn over the
// grid, the lanes sharing the bins: no launch waits on one thread walking a long sweep, nor
// on one warp walking many.

__global__ void __launch_bounds__(256) k_snr_resolve(
    Cands cd, Grid g, Tables tb, const double* __restrict__ Sg, const float* __restrict__ inv_f,
    double th2, double rtol, int mode, unsigned char* __restrict__ resolved,
    unsigned long long* __restrict__ acc, RunState* rs, Dirty d, int Kc, int sg_radius) {
  // the loop state, read by one thread per CTA (every thread of the grid loading the same
  // words would queue on one L2 line)
  __shared__ long long snr_head[4];  // stop, iteration, live candidates, long sweeps
  if (threadIdx.x == 0) {
    snr_head[0] = (rs->final_pass || rtol_stop(rs, rtol)) ? 1 : 0;
    snr_head[1] = rs->iter;
    snr_head[2] = (long long)rs->nlive;
    snr_head[3] = (long long)rs->nwide;
  }
  __syncthreads();
  if (snr_head[0]) return;
  const long long nlive = snr_head[2];
  const DirtyIter di(d, (int)snr_head[1]);
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const float th2f = (float)th2;
  unsigned local_new = 0, local_exact = 0, local_near = 0, local_unc = 0;
  // group grp holds candidates grp, grp + ngroups, grp + 2 ngroups, ...: candidates that
  // sit together in the list (the catalog pass emits the long sweeps of its FP64 path in
  // runs) are spread over many warps
  const long long ngroups = (nlive + 31) / 32;
  for (long long grp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; grp < ngroups;
       grp += nwarps) {
    bool todo = false;
    const long long c = grp + (long long)lane * ngroups;
    int4 pk = make_int4(0, 0, 0, 0);
    unsigned char done = 1;
    if (c < nlive) {  // both loads at once
      done = cd.res[c];
      pk = cd.pk[c];
    }
    if (!done && pk.y <= kSnrLaneBins) {  // the long sweeps are taken below
      const int ka = pk.x;
      const int nbin = pk.y;
      long long c0 = ka < 0 ? 0 : ka / Kc;
      long long kl = (long long)ka + nbin - 1;
      if (kl > g.nb - 1) kl = g.nb - 1;
      if (kl >= 0) {
        long long c1 = kl / Kc;
        for (long long cc = c0; cc <= c1 && !todo; ++cc) todo = di.any(cc, sg_radius);
      }
    }
    if (todo) {
      int kcount;
      const float r2 = screen_part(cd, c, pk, g, tb, inv_f, 0, 1, kcount);
      int dec = screen_decide(r2, kcount, th2f, mode);
      if (mode == 1 && screen_uncertain(r2, kcount, th2f)) ++local_unc;
      if (dec < 0) {
        ++local_exact;
        const double ex = rho2_exact(g, tb, Sg, cd.a2[c], cd.lo[c], cd.hi[c]);
        if (near_threshold(ex, th2)) ++local_near;
        dec = ex > th2;
      }
      if (dec) {
        cd.res[c] = 1;
        resolved[cd.src[c]] = 1;
        ++local_new;
        remove_part(cd, c, g, tb, acc, di, Kc, 0, 1);
      }
    }
  }
  // the long sweeps, one per warp at a time
  const long long nwide = snr_head[3];
  for (long long wi = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; wi < nwide;
       wi += nwarps) {
    const long long cw = cd.wide[wi];
    if (cd.res[cw]) continue;  // the same in every lane
    const int4 pkw = cd.pk[cw];
    const long long c0 = pkw.x < 0 ? 0 : pkw.x / Kc;
    long long kl = (long long)pkw.x + pkw.y - 1;
    if (kl > g.nb - 1) kl = g.nb - 1;
    bool t = false;
    if (kl >= 0)
      for (long long cc = c0 + lane; cc <= kl / Kc; cc += 32) t = t || di.any(cc, sg_radius);
    if (!__any_sync(0xFFFFFFFFu, t)) continue;
    {
      int kcount;
      float r2 = screen_part(cd, cw, pkw, g, tb, inv_f, lane, 32, kcount);
      // butterfly sums: every lane ends with the same values.  The sum's longest sequential
      // chain is the largest lane count, and the butterfly adds five roundings: the screen's
      // bound takes that many terms, not every bin of the sweep
      int kchain = kcount;
      for (int o = 16; o > 0; o >>= 1) {
        r2 = __fadd_rn(r2, __shfl_xor_sync(0xFFFFFFFFu, r2, o));
        kchain = max(kchain, __shfl_xor_sync(0xFFFFFFFFu, kchain, o));
      }
      const int keff = kchain + 5;
      int dec = screen_decide(r2, keff, th2f, mode);
      if (mode == 1 && lane == 0 && screen_uncertain(r2, keff, th2f)) ++local_unc;
      if (dec < 0) {
        // FP64, the lanes sharing the bins
        if (lane == 0) ++local_exact;
        const double v = rho2_exact_warp(g, tb, Sg, cd.a2[cw], cd.lo[cw], cd.hi[cw]);
        if (lane == 0 && near_threshold(v, th2)) ++local_near;
        dec = v > th2 ? 1 : 0;
      }
      if (dec) {
        if (lane == 0) {
          cd.res[cw] = 1;
          resolved[cd.src[cw]] = 1;
          ++local_new;
        }
        remove_part(cd, cw, g, tb, acc, di, Kc, lane, 32);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    local_new += __shfl_xor_sync(0xFFFFFFFFu, local_new, o);
    local_exact += __shfl_xor_sync(0xFFFFFFFFu, local_exact, o);
    local_near += __shfl_xor_sync(0xFFFFFFFFu, local_near, o);
    local_unc += __shfl_xor_sync(0xFFFFFFFFu, local_unc, o);
  }
  if (lane == 0) {
    if (local_new) atomicAdd(&rs->count_new, (unsigned long long)local_new);
    if (local_exact) atomicAdd(&rs->nexact, (unsigned long long)local_exact);
    if (local_near) atomicAdd(&rs->nnear, (unsigned long long)local_near);
    if (local_unc) atomicAdd(&rs->nuncertain, (unsigned long long)local_unc);
  }
}

// Both evaluations of rho^2 for every kept candidate against the current S_gal: the FP32
// screen (what the loop decides on first) and the FP64 value in the oracle's order of
// summation, with the bins the screen summed.  A measurement of the screen's error.
__global__ void __launch_bounds__(256) k_snr_check(Cands cd, Grid g, Tables tb,
                                                   const double* __restrict__ Sg,
                                                   const float* __restrict__ inv_f,
                                                   const RunState* rs,
                                                   long long* __restrict__ src,
                                                   float* __restrict__ screen,
                                                   double* __restrict__ exact,
                                                   int* __restrict__ kcount_out) {
  const long long nlive = (long long)rs->nlive;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nlive;
       c += (long long)gridDim.x * blockDim.x) {
    const int4 pk = cd.pk[c];
    int kcount = 0;
    screen[c] = screen_part(cd, c, pk, g, tb, inv_f, 0, 1, kcount);
    exact[c] = rho2_exact(g, tb, Sg, cd.a2[c], cd.lo[c], cd.hi[c]);
    src[c] = cd.src[c];
    kcount_out[c] = kcount;
  }
}

void launch_snr_check(Cands cd, long long ncap, const Grid& g, const Tables& tb, const double* Sg,
                      const float* inv_f, const RunState* rs, long long* src, float* screen,
                      double* exact, int* kcount, cudaStream_t st) {
  long long want = (ncap + 255) / 256;
  int bl = (int)(want < 4096 ? (want < 1 ? 1 : want) : 4096);
  k_snr_check<<<bl, 256, 0, st>>>(cd, g, tb, Sg, inv_f, rs, src, screen, exact, kcount);
}

void launch_snr_resolve(Cands cd, long long ncap, const Grid& g, const Tables& tb,
                        const double* Sg, const float* inv_f, double th2, double rtol, int mode,
                        unsigned char* resolved, unsigned long long* acc, RunState* rs,
                        Dirty d, int Kc, int sg_radius, int nsm, cudaStream_t st) {
  int th = 256;  // 8 warps, each screening 32 candidates at a time
  long long want = (ncap + th - 1) / th;
  long long cap = (long long)nsm * 8;
  int bl = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  k_snr_resolve<<<bl, th, 0, st>>>(cd, g, tb, Sg, inv_f, th2, rtol, mode, resolved, acc, rs, d, Kc,
                                   sg_radius);
}

// ============================================================================ coarse graining
// Bin averages of a per-bin series over log-spaced frequency bins (the coarse-grained
// spectrum and frequencies).  Bin k covers the grid indices [edge[k], edge[k+1]); one CTA
// per bin sums its values in a fixed order (no atomics), so the result is reproducible.
// The mean frequency of indices a .. b-1 is (2 k_lo + a + b - 1) / (2 T) exactly.
__global__ void __launch_bounds__(256) k_coarse_grain(const double* __restrict__ x,
                                                      const double* __restrict__ S,
                                                      const long long* __restrict__ edge,
                                                      long long k_lo, double T,
                                                      double* __restrict__ S_out,
                                                      double* __restrict__ f_out,
                                                      long long* __restrict__ cnt_out) {
  __shared__ double part[8];
  const int k = blockIdx.x;
  const long long a = edge[k], b = edge[k + 1];
  double s = 0.0;
  for (long long i = a + threadIdx.x; i < b; i += blockDim.x)
    s = __dadd_rn(s, S ? __dadd_rn(S[i], x[i]) : x[i]);
  for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xFFFFFFFFu, s, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = __dadd_rn(t, part[w]);
    const long long c = b - a;
    cnt_out[k] = c;
    S_out[k] = c > 0 ? __ddiv_rn(t, (double)c) : __longlong_as_double(0x7FF8000000000000ll);
    f_out[k] = c > 0 ? __ddiv_rn((double)(2 * k_lo + a + b - 1), __dmul_rn(2.0, T))
                     : __longlong_as_double(0x7FF8000000000000ll);
  }
}

void launch_coarse_grain(const double* x, const double* S, const long long* edge, int nbins,
                         long long k_lo, double T, double* S_out, double* f_out,
                         long long* cnt_out, cudaStream_t st) {
  k_coarse_grain<<<nbins, 256, 0, st>>>(x, S, edge, k_lo, T, S_out, f_out, cnt_out);
}

// ============================================================================ loop control

// Work lists from the dirty set `cur` (one CTA).  Their order depends on the atomics,
// which is harmless: every item is computed on its own.
__device__ void build_lists_cta(const unsigned char* __restrict__ cur, int nch,
                                int* __restrict__ lists, int* __restrict__ counts) {
  __shared__ int cnt[kNumLists];
  if (threadIdx.x < kNumLists) cnt[threadIdx.x] = 0;
  __syncthreads();
  const size_t stride = (size_t)nch + 1;
  for (int b = threadIdx.x; b <= nch; b += blockDim.x) {
    auto at = [&](int i) { return i >= 0 && i < nch && cur[i] != 0; };
    const bool d0 = at(b), dm1 = at(b - 1);
    if (b < nch) {
      const bool r0 = d0, r1 = r0 || dm1 || at(b + 1), r2 = r1 || at(b - 2) || at(b + 2);
      if (r0) lists[kListR0 * stride + atomicAdd(&cnt[kListR0], 1)] = b;
      if (r1) lists[kListR1 * stride + atomicAdd(&cnt[kListR1], 1)] = b;
      if (r2) lists[kListR2 * stride + atomicAdd(&cnt[kListR2], 1)] = b;
    }
    if (d0 || dm1) lists[kListTile * stride + atomicAdd(&cnt[kListTile], 1)] = b;
  }
  __syncthreads();
  if (threadIdx.x < kNumLists) counts[threadIdx.x] = cnt[threadIdx.x];
}

__global__ void k_build_lists(Dirty d, int* lists, int* counts, RunState* rs) {
  build_lists_cta(d.base + (size_t)(d.rs->iter & 1) * d.nch, d.nch, lists, counts);
  __syncthreads();
  if (threadIdx.x < kNumLists) rs->work[threadIdx.x] += (unsigned long long)counts[threadIdx.x];
}

void launch_build_lists(Dirty d, int* lists, int* counts, RunState* rs, cudaStream_t st) {
  k_build_lists<<<1, 1024, 0, st>>>(d, lists, counts, rs);
}

__global__ void k_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                          unsigned long long cond_handle, int use_cond, unsigned char* dirty,
                          int nch, int* lists, int* counts) {
  // every thread reads the count before thread 0 advances it (after the barriers below)
  const int it0 = rs->iter;
  // thread 0 loads the rest of the loop state now, so that its latency overlaps the lists
  int final_pass = 0;
  unsigned err = 0u;
  unsigned long long nn = 0ull, nres = 0ull;
  bool rstop = false;
  unsigned long long work[kNumLists] = {};
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < kNumLists; ++i) work[i] = rs->work[i];
    final_pass = rs->final_pass;
    err = rs->err;
    nn = rs->count_new;
    nres = rs->nres;
    rstop = rtol_stop(rs, rtol);
  }
  if (dirty) {
    // clear the set this iteration read; the removals of this iteration marked the other
    // one, which the next iteration reads through its work lists
    unsigned char* cur = dirty + (size_t)(it0 & 1) * nch;
    for (int i = threadIdx.x; i < nch; i += blockDim.x) cur[i] = 0;
    build_lists_cta(dirty + (size_t)((it0 + 1) & 1) * nch, nch, lists, counts);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned go = 1u;
  if (final_pass || (err & ERR_TIMEOUT)) {
    go = 0u;  // the last pass is done, or the catalog pass gave up
  } else {
    int it = it0 + 1;
    rs->iter = it;
    if (new_hist && it <= max_iter) new_hist[it - 1] = (int)nn;
    rs->nres = nres + nn;
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
  if (go && dirty)  // the lists just built go to the next iteration's kernels
    for (int i = 0; i < kNumLists; ++i) rs->work[i] = work[i] + (unsigned long long)counts[i];
  if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, go);
}

void launch_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                    unsigned long long cond_handle, int use_cond, unsigned char* dirty, int nch,
                    int* lists, int* counts, cudaStream_t st) {
  k_control<<<1, 1024, 0, st>>>(rs, max_iter, rtol, new_hist, cond_handle, use_cond, dirty, nch,
                                lists, counts);
}

void plan_grids(SmoothPlan& pl) {
  pl.res_sort = pl.res_median = pl.res_prefix = pl.res_mean = 0;
  if (pl.nsm <= 0) return;
  with_sort_kernel(pl, [&](auto kern) {
    pl.res_sort = resident_ctas(pl, kern, sort_threads(pl), sort_smem(pl));
  });
  if (pl.fp32_keys)
    pl.res_median = resident_ctas(pl, k_median_wm<uint32_t>, median_threads(pl),
                                  median_smem_bytes(pl.Kc, 4));
  else
    pl.res_median = resident_ctas(pl, k_median_wm<u64>, median_threads(pl),
                                  median_smem_bytes(pl.Kc, 8));
  pl.res_prefix = resident_ctas(pl, k_chunk_prefix, pl.Kc < 1024 ? pl.Kc : 1024, 0);
  pl.res_mean = resident_ctas(pl, k_window_mean, mean_threads(pl), 0);
}

void configure_kernels() {
  cudaFuncSetAttribute(k_prepass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepassSmem);
  SmoothPlan p64 = {}, p32 = {};
  p32.fp32_keys = 1;
  for (int kp : {64, 4096, 8192}) {  // one of each instantiation; 8192: the widest sort
    p64.kpad = p32.kpad = kp;
    auto set = [](auto kern) {
      SmoothPlan widest = {};
      widest.kpad = 8192;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sort_smem(widest));
    };
    with_sort_kernel(p64, set);
    with_sort_kernel(p32, set);
  }
  cudaFuncSetAttribute(k_median_wm<u64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)median_smem_bytes(kMaxWindow, 8));
  cudaFuncSetAttribute(k_median_wm<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)median_smem_bytes(kMaxWindow, 4));
}

}  // namespace gbsub
