// Launch interface of the subtraction kernels (arXiv 2602.18560, App. D).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "generate.cuh"

namespace gbsub {

// Candidates that can still be resolved (rho_0 > rho_th), structure of arrays.
struct Cands {
  long long* src;     // index in the catalog
  int4* pk;           // the screen's 16-byte record, read in one load:
                      //   x = ka, first bin of the sweep relative to k_lo (may be < 0)
                      //   y = nbin, bins touched by the sweep (kb - ka + 1)
                      //   z = bits of A^2 * 2^160 (FP32), w = bits of lo - ka (FP32)
  float* len;         // hi - lo (FP32 screen of sweeps over more than one bin)
  double* a2;         // A^2 (exact path)
  double* amp;        // A (removal of a single-bin source: the same units it deposited)
  double* lo;         // sweep endpoints in bin units (exact path)
  double* hi;
  unsigned char* res; // 1 once resolved
  long long* wide;    // the candidates whose sweeps cross more than kSnrLaneBins bins
};
// Sweeps of at most this many bins are screened by one lane; longer ones by a whole warp.
constexpr int kSnrLaneBins = 4;

// Loop state kept on the device for one run.
struct RunState {
  int iter;              // iterations completed
  int final_pass;        // 1: max_iter reached, one more estimate of S_gal without SNR
  int converged;         // 1: stopped because nothing crossed rho_th (or rtol met)
  int stopped;           // 1: the loop is over
  unsigned long long ncand;     // sources with rho_0 >= kappa rho_th (paper's candidates)
  unsigned long long nlive;     // candidates kept (rho_0 > rho_th, and >= kappa rho_th)
  unsigned long long nres;
  unsigned long long count_new;
  unsigned long long nexact;    // SNR decisions that needed the exact FP64 recomputation
  unsigned long long max_p_bits;    // scratch maximum (estimate on a given spectrum)
  unsigned long long relchg_bits;   // max relative change of S_n (conv_rtol)
  unsigned long long next_tile;  // catalog tiles handed out so far (catalog pass)
  unsigned long long work[4];    // work-list items the loop kernels were handed (by list)
  unsigned long long nnear;      // FP64 decisions with |rho^2 / rho_th^2 - 1| < 2e-9
  unsigned long long nuncertain; // FP32 decisions (mixed precision) inside the screen's bound
  unsigned long long nwide;      // entries of Cands::wide
  unsigned err;
  unsigned pad;
};

// Grid and per-bin tables.
struct Grid {
  double T, T2, t5;      // T_obs, T_obs^2, T_obs / 5
  long long k_lo;        // first DFT index in band
  long long nb;          // bins in band
  unsigned long long mT; // T_obs = mT 2^eT, mT the 53-bit integer mantissa
  int eT;
  float T2f;             // T_obs^2 in FP32
  unsigned tq;           // T_obs = tq 2^etq with tq odd, when it fits in 32 bits (short_t)
  int etq;
  int short_t;
};

// Per-bin tables, built once per context.
struct Tables {
  const double* S;       // S_instr
  const double* R;       // R
  const double* gq;      // 2^96 (T/5) R / S: fixed-point units per unit of A^2 w
  const float* Gf;       // 4 (T/5) R / S * 2^-160: rho_0^2 per unit of A^2 w * 2^160
  const float* invSf;    // 1 / (S * 2^150)
};

struct SmoothPlan {
  int W;        // window (bins)
  int Kc;       // chunk length: multiple of 32, >= W
  int nw;       // 32-bit words per chunk bitset (Kc / 32)
  int nch;      // chunks
  int kpad;     // power of two >= Kc (sort width)
  int nsm;      // SMs for persistent grids (0: one CTA per work item)
  int fp32_keys;  // median on the FP32-rounded values (mixed precision): 4-byte keys
  double key_scale;  // power of two the values are scaled by before rounding to FP32
  int res_sort, res_median, res_prefix, res_mean;  // CTAs resident at once (plan_grids)
  int sort_e;     // elements per sorting thread (2, 4, 8), 0: chosen from kpad
  int median_th;  // threads per median tile (multiple of 32, <= 512), 0: chosen from Kc
};

// Source of an estimator's input: the run's fixed-point spectrum (P_k = S_k Q_k 2^-96) or
// a plain array of doubles.
struct SpecIn {
  const unsigned long long* acc;  // 4 words per bin (three used), or null
  const double* S;                // S_instr when acc is set
  const double* x;                // input doubles when acc is null
};

// Chunks whose input changed since the previous iteration.  Two byte arrays of nch
// entries alternate: iteration i reads set (i-1) & 1 and the removals of iteration i mark
// set i & 1 (rs->iter = i - 1 while iteration i runs).  A null base means every chunk
// has changed (first estimate, or an estimate of a given spectrum).
//
// From the set an iteration reads, the loop control builds work lists (ascending order is
// not kept): the chunks with a changed chunk within 0, 1 or 2 of them, and the median
// tiles u whose chunks u-1 or u changed.  The chunk kernels run persistent grids over
// them, so an iteration that changed a few chunks launches a few busy CTAs.
enum { kListR0 = 0, kListR1 = 1, kListR2 = 2, kListTile = 3, kNumLists = 4 };

struct Dirty {
  unsigned char* base;
  int nch;
  const RunState* rs;
  const int* lists;   // [kNumLists][nch + 1], null when base is null
  const int* counts;  // [kNumLists]
  __device__ __forceinline__ bool any(long long c, int radius) const {
    return any_between(c - radius, c + radius);
  }
  // any chunk of [a, b] (clipped to the chunks that exist)
  __device__ __forceinline__ bool any_between(long long a, long long b) const {
    if (!base) return true;
    const unsigned char* cur = base + (size_t)(rs->iter & 1) * nch;
    if (a < 0) a = 0;
    if (b > nch - 1) b = nch - 1;
    for (long long i = a; i <= b; ++i)
      if (cur[i]) return true;
    return false;
  }
  __device__ __forceinline__ void mark_next(long long c) const {
    if (base) base[(size_t)((rs->iter + 1) & 1) * nch + c] = 1;
  }
  // items of work list `which` (all `all` of them when nothing is tracked)
  __device__ __forceinline__ int count(int which, int all) const {
    return lists ? counts[which] : all;
  }
  __device__ __forceinline__ int item(int which, int i) const {
    return lists ? lists[(size_t)which * (nch + 1) + i] : i;
  }
};

// The dirty sets of one iteration, the iteration fixed: the set read (cur) and the set
// written for the next one (nxt); both null when nothing is tracked.
struct DirtyIter {
  const unsigned char* cur;
  unsigned char* nxt;
  int nch;
  __device__ __forceinline__ DirtyIter(const Dirty& d, int iter) : nch(d.nch) {
    cur = d.base ? d.base + (size_t)(iter & 1) * d.nch : nullptr;
    nxt = d.base ? d.base + (size_t)((iter + 1) & 1) * d.nch : nullptr;
  }
  // any chunk of [c - radius, c + radius] (clipped to the chunks that exist)
  __device__ __forceinline__ bool any(long long c, int radius) const {
    if (!cur) return true;
    long long a = c - radius, b = c + radius;
    if (a < 0) a = 0;
    if (b > nch - 1) b = nch - 1;
    bool r = false;
    for (long long i = a; i <= b; ++i) r |= cur[i] != 0;  // independent loads
    return r;
  }
  __device__ __forceinline__ void mark_next(long long c) const {
    if (nxt) nxt[c] = 1;
  }
};

// A work list's length, the CTA's first item and the iteration, read by one thread and
// shared with the CTA: when every thread of hundreds of CTAs loads the same words, the
// requests queue on one L2 line and a late iteration's few working CTAs wait behind them.
struct ListHead {
  int count, first, iter;
};
__device__ __forceinline__ ListHead list_head(const Dirty& d, int which, int all) {
  __shared__ ListHead sh;
  if (threadIdx.x == 0) {
    ListHead h;
    h.count = d.count(which, all);
    h.first = d.item(which, blockIdx.x);  // the grid is never longer than the list
    h.iter = d.base ? d.rs->iter : 0;
    sh = h;
  }
  __syncthreads();
  const ListHead r = sh;
  return r;
}

// Output epilogue of the kernel that writes S_gal.
struct SgOut {
  double* out;           // S_gal (or the median of median-then-mean)
  float* inv_f;          // 1 / (1 + S_gal / S_instr) in FP32, or null
  const double* S;       // S_instr (for inv_f and the rtol test)
  const float* invSf;
  int rtol_on;
  RunState* rs;
};

// Raise the dynamic shared-memory limits of the kernels that need more than 48 KB.
void configure_kernels();

// Persistent-grid sizes of the chunk kernels for pl (after configure_kernels; pl.nsm set).
void plan_grids(SmoothPlan& pl);

void launch_tables(const Grid& g, int tdi2, double* S, double* R, double* gq, float* Gf,
                   float* invSf, cudaStream_t st);

// Private copies of words 1 and 2 of the first nbins bins, kAccReplicas of them, zeroed
// before the catalog pass; the pass folds them into the spectrum.
constexpr int kAccReplicas = 16;
constexpr long long kAccReplicaBins = 65536;
struct AccReplicas {
  unsigned long long* w;  // [kAccReplicas][nbins][2]
  long long nbins;
};

// Where the catalog pass finds the catalog.  Each load writes it on the stream, so that one
// captured launch serves every catalog of up to the capacity it was built for.
struct CatalogRef {
  const double* A;
  const double* f;
  const double* fdot;
  long long n;
  int staged;  // 1: device memory, staged in tiles by bulk copies
               // 0: page-locked host memory, read in place with plain loads
               // 2: generated: every source is computed from gen inside the pass
  int pad;
  GenParams gen;  // the recipe's constants (generated catalogs)
};
enum { kCatHostMapped = 0, kCatDevice = 1, kCatGenerated = 2 };

// The catalog pass over the cat->n sources.  test_flags & 1: issue no catalog copies, so
// that the bounded waits run out (tests of the timeout path).
void launch_prepass(const CatalogRef* cat, long long cap, const Grid& g, const Tables& tb,
                    double thr_kappa, double thr_live, unsigned long long* acc, AccReplicas rep,
                    Cands cd, RunState* rs, int nsm, int test_flags, cudaStream_t st);

// *p = v on the stream.
void launch_set_catalog(CatalogRef* p, const CatalogRef& v, cudaStream_t st);

// A generated catalog of n sources (seed, power-law index gamma, Gamma shape >= 1): its
// constants are computed on the device into ref->gen.  With A null the catalog pass generates
// every source itself (ref->staged = kCatGenerated); otherwise A, f, fdot receive the
// catalog (launch_generate) and the pass reads them like a loaded one.
void launch_gen_setup(CatalogRef* ref, long long n, unsigned long long seed, double gamma,
                      double shape, const double* A, const double* f, const double* fdot,
                      cudaStream_t st);
// The same for the paper's population model (Sec. II.B, Table I; App. A).
void launch_gen_setup_paper(CatalogRef* ref, long long n, unsigned long long seed,
                            const PaperPop& pp, const double* A, const double* f,
                            const double* fdot, cudaStream_t st);
// Sources start .. start+n-1 of the generated catalog described by ref->gen into A, f, fdot.
void launch_generate(const CatalogRef* ref, long long start, long long n, double* A, double* f,
                     double* fdot, cudaStream_t st);

// Coarse graining: for every bin k of [edge[k], edge[k+1]) (nbins + 1 edges on the device),
// the mean of x (of S + x when S is given), the mean frequency (k_lo + i) / T and the count.
void launch_coarse_grain(const double* x, const double* S, const long long* edge, int nbins,
                         long long k_lo, double T, double* S_out, double* f_out,
                         long long* cnt_out, cudaStream_t st);

// P[j] = S_j Q_j 2^-96 for every bin.
void launch_power_out(const unsigned long long* acc, const double* S, long long n, double* P,
                      cudaStream_t st);

// *max_bits = max(*max_bits, bits of max x) over x[0 .. n) (x >= 0).
void launch_max_bits(const double* x, long long n, unsigned long long* max_bits, cudaStream_t st);

// Sort every chunk of the input whose values changed (sorted keys, position -> rank).
void launch_chunk_sort(SpecIn in, long long n, const SmoothPlan& pl, unsigned long long* skey,
                       uint16_t* srank, Dirty d, cudaStream_t st);

// out = C * running median from the sorted chunks, recomputed in the tiles whose windows
// changed.
void launch_running_median(const unsigned long long* skey, const uint16_t* srank, long long n,
                           const SmoothPlan& pl, SgOut o, Dirty d, cudaStream_t st);
size_t median_smem_bytes(int Kc, int key_bytes);

// Exact 128-bit prefix sums of the input inside each chunk at a per-chunk scale sig[b];
// uflow[b] = 1 when an input > 0 of chunk b is below one unit.  x_out (may be null)
// receives the input values.
// (in_radius: the input of chunk b changed when a chunk within in_radius of b is dirty.)
void launch_chunk_prefix(SpecIn in, long long n, const SmoothPlan& pl, unsigned long long* pre_lo,
                         unsigned long long* pre_hi, int* sig, unsigned* uflow, double* x_out,
                         Dirty d, int in_radius, cudaStream_t st);

void launch_window_mean(const double* x, long long n, const SmoothPlan& pl,
                        const unsigned long long* pre_lo, const unsigned long long* pre_hi,
                        const int* sig, const unsigned* uflow, SgOut o, Dirty d, int out_radius,
                        cudaStream_t st);

// sg_radius: S_gal of chunk c changed when a chunk within sg_radius of c is dirty; only
// candidates with a bin in such a chunk are tested again.
void launch_snr_resolve(Cands cd, long long ncap, const Grid& g, const Tables& tb,
                        const double* Sg, const float* inv_f, double th2, double rtol, int mixed,
                        unsigned char* resolved, unsigned long long* acc, RunState* rs,
                        Dirty d, int Kc, int sg_radius, int nsm, cudaStream_t st);

// For each kept candidate c < rs->nlive (ncap: capacity): its catalog index, its rho^2 as the
// FP32 screen evaluates it against the current S_gal (through inv_f) with the count of bins
// summed, and its rho^2 in FP64 in the oracle's order of summation.
void launch_snr_check(Cands cd, long long ncap, const Grid& g, const Tables& tb, const double* Sg,
                      const float* inv_f, const RunState* rs, long long* src, float* screen,
                      double* exact, int* kcount, cudaStream_t st);

// Work lists of the set the next iteration reads (set rs->iter & 1).
void launch_build_lists(Dirty d, int* lists, int* counts, RunState* rs, cudaStream_t st);

// Loop control; it also clears the dirty set the finished iteration read and builds the
// work lists of the next one.
void launch_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                    unsigned long long cond_handle, int use_cond, unsigned char* dirty, int nch,
                    int* lists, int* counts, cudaStream_t st);

}  // namespace gbsub
