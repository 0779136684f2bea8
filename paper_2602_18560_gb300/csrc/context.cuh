// Internal layout of a subtraction context, shared by the C ABI (api.cu) and the batch
// and serving runtime (runtime.cu).  Not part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gbsub.h"
#include "kernels.cuh"

using gbsub::AccReplicas;
using gbsub::CatalogRef;
using gbsub::Cands;
using gbsub::Grid;
using gbsub::RunState;
using gbsub::SmoothPlan;

struct sub_ctx {
  sub_params p;
  Grid grid;
  SmoothPlan plan;
  cudaStream_t stream = nullptr;   // where work is issued
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  int nsm = 0;
  int device = 0;
  int grid_div = 1;      // the persistent kernels use 1/grid_div of the GPU (batches)
  int nsm_run = 0;       // SMs the catalog pass and the SNR size their grids for
  // bookkeeping
  std::vector<std::pair<void*, int64_t>> allocs;
  int64_t bytes = 0;
  std::string err;
  // tables
  double *S = nullptr, *R = nullptr, *gq = nullptr;
  float *Gf = nullptr, *invSf = nullptr;
  // spectrum and smoothing buffers
  unsigned long long* acc = nullptr;  // 4 words per bin
  AccReplicas rep = {nullptr, 0};     // private copies of the first bins (catalog pass)
  double *P = nullptr, *M = nullptr, *Sg = nullptr;
  double* estimate_in = nullptr;  // input copy of sub_estimate
  double* cg = nullptr;           // coarse graining: [S | f | counts | edges] of cg_cap bins
  int cg_cap = 0;
  float* inv_f = nullptr;
  int* sig = nullptr;
  unsigned char* dirty = nullptr;  // two sets of one byte per chunk
  int* lists = nullptr;            // work lists of the chunk kernels [kNumLists][nch + 1]
  int* list_counts = nullptr;      // [kNumLists]
  unsigned long long* skey = nullptr;
  uint16_t* srank = nullptr;
  unsigned long long *pre_lo = nullptr, *pre_hi = nullptr;
  unsigned* uflow = nullptr;
  // catalog and per-source buffers
  int64_t N = -1;        // sources loaded (-1: none)
  int64_t cap_N = 0;     // capacity of the per-source buffers
  double *A = nullptr, *f = nullptr, *fdot = nullptr;
  CatalogRef* dcat = nullptr;  // where the catalog pass reads the catalog (on the device)
  int cat_kind = 1;            // kCatDevice (copied or materialised), kCatHostMapped, kCatGenerated
  const double* cat_host[3] = {nullptr, nullptr, nullptr};  // the mapped arrays (kCatHostMapped)
  int test_flags = 0;       // sub_test_hooks
  Cands cd = {};
  unsigned char* resolved = nullptr;
  // run state
  RunState* rs = nullptr;
  int* new_hist = nullptr;
  RunState* h_rs = nullptr;  // pinned copy
  bool ran = false;
  // graph
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t graph_cap = -1;  // catalog capacity the graph was built for
  int64_t graph_gen = 0;   // bumped whenever launch settings change (batches rebuild)
  bool use_graph = true;
  // timing
  cudaEvent_t ev_start = nullptr, ev_pre = nullptr, ev_end = nullptr;
  cudaEvent_t ev_k[2] = {nullptr, nullptr};
  float prof_ms[SUB_K_COUNT];
  int prof_n[SUB_K_COUNT];
  std::vector<float> prof_iter_ms;  // per profiled iteration, per kernel (SUB_K_*)
  int prof_iter = -1;               // iteration being profiled (-1: the catalog pass)
  bool profiling = false;
};

namespace gbsub {
// Message of a failure that has no context.
void set_global_error(const char* msg);
// Message of the last failure of a call on c (or of a call without a context).
void ctx_set_err(sub_ctx* c, const char* fmt, ...);
// Copy the run state back (synchronises the context's stream) and fill st (may be null);
// returns the run's status.
int ctx_fill_stats(sub_ctx* c, sub_stats* st);
// Add the nodes of one whole run of c (catalog pass, device loop, timing events) to g with
// no dependencies; *last receives the final node.  The conditional handle of the loop is
// created on g.
cudaError_t ctx_add_run_nodes(sub_ctx* c, cudaGraph_t g, cudaGraphNode_t* last);
// Grid divisor of the persistent kernels (1 = the whole GPU).
void ctx_set_grid_div(sub_ctx* c, int div);
int ctx_set_tuning(sub_ctx* c, int knob, int value);  // SUB_OK or SUB_EINVAL
// Buffers for catalogs of up to cap sources and the run's graph, ahead of the first catalog.
int ctx_prepare(sub_ctx* c, int64_t cap);
// Test hooks (SUB_TEST_*) baked into the next graph.
void ctx_set_test_flags(sub_ctx* c, int flags);
}  // namespace gbsub
