// Launch interface of the subtraction kernels (arXiv 2602.18560, App. D).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbsub {

// One candidate source: everything the SNR step needs, 32 bytes (two 16-byte loads).
struct Cand {
  long long src;  // index in the catalog
  double a2;      // A^2
  double lo, hi;  // sweep endpoints in bin units (sorted)
};

// Loop state kept on the device for one run.
struct RunState {
  int iter;              // iterations completed
  int final_pass;        // 1: max_iter reached, one more estimate of S_gal without SNR
  int converged;         // 1: stopped because nothing crossed rho_th (or rtol met)
  int stopped;           // 1: the loop is over
  unsigned long long ncand;
  unsigned long long nres;
  unsigned long long count_new;
  unsigned long long max_p_bits;    // max of the estimator input, as bits of a double >= 0
  unsigned long long max_m_bits;    // max of the median output (median-then-mean)
  unsigned long long relchg_bits;   // max relative change of S_n (conv_rtol)
  unsigned err;
  unsigned pad;
};

// Grid and per-bin tables.
struct Grid {
  double T, T2, t5;      // T_obs, T_obs^2, T_obs / 5
  long long k_lo;        // first DFT index in band
  long long nb;          // bins in band
};

struct SmoothPlan {
  int W;        // window (bins)
  int Kc;       // chunk length: multiple of 32, >= W
  int nw;       // 32-bit words per chunk bitset (Kc / 32)
  int nch;      // chunks
  int nsnap;    // snapshots per chunk (Kc / kSnapStride + 1)
  int kpad;     // power of two >= Kc (sort width)
  int L;        // outputs per thread in the median slide
  int slide_threads;
};

// Raise the dynamic shared-memory limits of the kernels that need more than 48 KB.
void configure_kernels();

void launch_tables(const Grid& g, int tdi2, double* S, double* R, double* gq, cudaStream_t st);

void launch_prepass(const double* A, const double* f, const double* fdot, long long N,
                    const Grid& g, const double* gq, double thr_q, unsigned long long* acc_lo,
                    unsigned long long* acc_hi, Cand* cand, RunState* rs, int nsm,
                    cudaStream_t st);

void launch_q2p(const unsigned long long* acc_lo, const unsigned long long* acc_hi,
                const double* S, long long nb, double* P, RunState* rs, int final_only,
                cudaStream_t st);

// *max_bits = max(*max_bits, bits of max x) over x[0 .. n) (x >= 0).
void launch_max_bits(const double* x, long long n, unsigned long long* max_bits, cudaStream_t st);

void launch_chunk_sort(const double* x, long long n, const SmoothPlan& pl, unsigned long long* skey,
                       uint16_t* srank, uint32_t* snap, const RunState* rs, cudaStream_t st);

// out = C * running median of x.  max_bits_out (may be null) receives the max of out.
// When rtol_on, relative change of S_instr + out against its previous content is
// folded into rs->relchg_bits before out is overwritten.
void launch_median_slide(const unsigned long long* skey, const uint16_t* srank,
                         const uint32_t* snap, long long n, const SmoothPlan& pl, double* out,
                         unsigned long long* max_bits_out, const double* S, int rtol_on,
                         RunState* rs, cudaStream_t st);

// Exact 128-bit prefix sums of x inside each chunk; uflow[b] = 1 when an input > 0 of
// chunk b is below one fixed-point unit.
void launch_chunk_prefix(const double* x, long long n, const SmoothPlan& pl,
                         const unsigned long long* max_bits, unsigned long long* pre_lo,
                         unsigned long long* pre_hi, unsigned* uflow, const RunState* rs,
                         cudaStream_t st);

void launch_window_mean(const double* x, long long n, const SmoothPlan& pl,
                        const unsigned long long* max_bits, const unsigned long long* pre_lo,
                        const unsigned long long* pre_hi, const unsigned* uflow, double* out,
                        const double* S, int rtol_on, RunState* rs, cudaStream_t st);

void launch_snr_resolve(const Cand* cand, long long ncand_cap, const Grid& g, const double* S,
                        const double* R, const double* gq, const double* Sg, double th2,
                        double rtol, unsigned char* cres, unsigned char* resolved,
                        unsigned long long* acc_lo, unsigned long long* acc_hi, RunState* rs,
                        int nsm, cudaStream_t st);

void launch_control(RunState* rs, int max_iter, double rtol, int* new_hist,
                    unsigned long long cond_handle, int use_cond, cudaStream_t st);

}  // namespace gbsub
