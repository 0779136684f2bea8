// Running mean of a caller's spectrum with no device allocation at all.
//
// Some callers cannot call cudaMalloc: a plug-in that only receives device
// buffers from a host framework which owns every byte of device memory and does
// not allow allocations behind its back, or a latency-critical loop that must not
// enter the allocator (cudaMalloc may synchronise the device and may fail at run
// time).  For them, sub_running_mean_noalloc computes the same running mean as the
// context path (exact 128-bit window sums over chunks, App. D Eq. running mean)
// with its scratch in one file-scope device array below.
//
// The array is part of the library image: every GPU that loads the library holds
// it (about 21 MB) until the process exits.  Every call shares it and it keeps the
// last call's contents, so calls whose work overlaps on the GPU (different streams,
// or different host threads) race with each other and must be serialised by the
// caller.  Nothing in it has to start at zero: every call rewrites the prefix sums,
// the per-chunk scales and the underflow flags of all the bins and chunks it reads.

#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/gbsub.h"
#include "common.cuh"
#include "kernels.cuh"

namespace gbsub {
void set_global_error(const char* msg);
}

using namespace gbsub;

namespace {

constexpr long long kNoAllocMaxBins = SUB_NOALLOC_MAX_BINS;
constexpr long long kNoAllocMaxWindow = SUB_NOALLOC_MAX_WINDOW;
// chunk cells: at most one chunk beyond the bins, chunks of >= 32 and <= max window
constexpr long long kCells = kNoAllocMaxBins + kNoAllocMaxWindow + 32;
constexpr long long kChunks = kNoAllocMaxBins / 32 + 2;
// layout in 8-byte words: pre_lo[kCells] | pre_hi[kCells] | scale (i32)[kChunks] |
// underflow flag (u32)[kChunks]
constexpr long long kWords = 2 * kCells + kChunks;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kWords];


}  // namespace

extern "C" int sub_running_mean_noalloc(const double* x, double* out, int64_t n, int32_t window,
                                        void* stream) {
  char msg[256];
  if (!x || !out) {
    set_global_error("sub_running_mean_noalloc: x and out must be device pointers");
    return SUB_EINVAL;
  }
  if (n < 1 || n > kNoAllocMaxBins) {
    snprintf(msg, sizeof(msg),
             "sub_running_mean_noalloc: n = %lld bins is outside 1 .. %lld (the size of its "
             "static scratch)", (long long)n, kNoAllocMaxBins);
    set_global_error(msg);
    return SUB_EINVAL;
  }
  if (window < 1 || window > kNoAllocMaxWindow) {
    snprintf(msg, sizeof(msg), "sub_running_mean_noalloc: window %d is outside 1 .. %lld",
             window, kNoAllocMaxWindow);
    set_global_error(msg);
    return SUB_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "sub_running_mean_noalloc: cudaGetDevice failed: %s",
             cudaGetErrorString(e));
    set_global_error(msg);
    return SUB_ECUDA;
  }
  // The host-side name of the array is only a stand-in: the runtime gives its device
  // address on the current device.  Asked on every call (it allocates nothing once the
  // module is loaded), so that no address outlives a reset of the device's context.
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    snprintf(msg, sizeof(msg), "sub_running_mean_noalloc: cudaGetSymbolAddress failed: %s",
             cudaGetErrorString(e));
    set_global_error(msg);
    return SUB_ECUDA;
  }
  unsigned long long* base = (unsigned long long*)p;
  SmoothPlan pl = {};
  pl.W = window;
  pl.Kc = ((window + 31) / 32) * 32;
  if (pl.Kc < 32) pl.Kc = 32;
  pl.nw = pl.Kc / 32;
  pl.nch = (int)((n + pl.Kc - 1) / pl.Kc);
  pl.kpad = 0;
  pl.nsm = 0;  // one CTA per chunk
  pl.fp32_keys = 0;
  pl.key_scale = 1.0;
  pl.res_sort = pl.res_median = pl.res_prefix = pl.res_mean = 0;
  unsigned long long* pre_lo = base;
  unsigned long long* pre_hi = base + kCells;
  int* sig = (int*)(base + 2 * kCells);
  unsigned* uflow = (unsigned*)(sig + kChunks);
  cudaStream_t st = (cudaStream_t)stream;
  SpecIn in;
  in.acc = nullptr;
  in.S = nullptr;
  in.x = x;
  SgOut o;
  o.out = out;
  o.inv_f = nullptr;
  o.S = nullptr;
  o.invSf = nullptr;
  o.rtol_on = 0;
  o.rs = nullptr;
  Dirty all;  // every chunk is computed
  all.base = nullptr;
  all.nch = pl.nch;
  all.rs = nullptr;
  all.lists = nullptr;
  all.counts = nullptr;
  launch_chunk_prefix(in, n, pl, pre_lo, pre_hi, sig, uflow, nullptr, all, 0, st);
  launch_window_mean(x, n, pl, pre_lo, pre_hi, sig, uflow, o, all, 0, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "sub_running_mean_noalloc: launch failed: %s",
             cudaGetErrorString(e));
    set_global_error(msg);
    return SUB_ECUDA;
  }
  return SUB_OK;
}
