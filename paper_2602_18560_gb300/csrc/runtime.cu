// Batches and serving on top of the subtraction contexts.
//
// A batch runs many catalogs at once: one CUDA graph holds every context's catalog pass and
// device loop as independent branches and is launched once.  The per-iteration kernels of
// one catalog leave most of the GPU idle (a few chunks change per iteration), so catalogs
// run side by side overlap on the SMs.
//
// A server accepts subtraction jobs as they arrive (host catalogs and host result buffers),
// admits them in arrival order while a device-memory budget and an in-flight limit allow
// (a job that an idle pooled context can take starts past a head that has to wait),
// runs each on a pooled context with its own stream (jobs overlap on the GPU: continuous
// batching), and hands back each job's statistics with its latency from submission to
// results in the caller's buffers.  Completion is observed by a host function enqueued
// behind the result copies, so the latency is not quantised by polling.

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "context.cuh"

using namespace gbsub;
using Clock = std::chrono::steady_clock;

// ============================================================================ batch

struct sub_batch {
  std::vector<sub_ctx*> ctxs;
  std::vector<int64_t> sizes;  // catalog capacities the graph was built for
  std::vector<int64_t> gens;   // and the contexts' launch-setting generations
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  float last_ms = 0.0f;
  std::string err;
};

static void batch_err(sub_batch* b, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
}

static void batch_drop_graph(sub_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->sizes.clear();
  b->gens.clear();
}

static int batch_build(sub_batch* b) {
  batch_drop_graph(b);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  for (size_t i = 0; !e && i < b->ctxs.size(); ++i) {
    cudaGraphNode_t last = nullptr;
    e = ctx_add_run_nodes(b->ctxs[i], g, &last);
  }
  if (!e) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    b->exec = nullptr;
    batch_err(b, "batch graph build failed: %s", cudaGetErrorString(e));
    return SUB_ECUDA;
  }
  b->graph = g;
  for (sub_ctx* c : b->ctxs) {
    b->sizes.push_back(c->cap_N);
    b->gens.push_back(c->graph_gen);
  }
  return SUB_OK;
}

extern "C" int sub_batch_create(sub_ctx* const* ctxs, int32_t n, sub_batch** out) {
  if (!out) return SUB_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1) {
    set_global_error("sub_batch_create: need at least one context");
    return SUB_EINVAL;
  }
  for (int32_t i = 0; i < n; ++i) {
    if (!ctxs[i]) {
      set_global_error("sub_batch_create: null context");
      return SUB_EINVAL;
    }
    for (int32_t k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) {
        set_global_error("sub_batch_create: a context appears twice");
        return SUB_EINVAL;
      }
    if (ctxs[i]->device != ctxs[0]->device) {
      set_global_error("sub_batch_create: contexts on different devices");
      return SUB_EINVAL;
    }
  }
  sub_batch* b = new (std::nothrow) sub_batch;
  if (!b) return SUB_ENOMEM;
  b->ctxs.assign(ctxs, ctxs + n);
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreate(&b->ev0);
  if (!e) e = cudaEventCreate(&b->ev1);
  if (e) {
    set_global_error("sub_batch_create: stream or event creation failed");
    sub_batch_destroy(b);
    return SUB_ECUDA;
  }
  *out = b;
  return SUB_OK;
}

extern "C" int sub_batch_run(sub_batch* b, sub_stats* stats) {
  if (!b) return SUB_EINVAL;
  for (sub_ctx* c : b->ctxs)
    if (c->N < 0) {
      batch_err(b, "a context of the batch has no catalog");
      return SUB_ESTATE;
    }
  bool stale = b->exec == nullptr || b->sizes.size() != b->ctxs.size();
  for (size_t i = 0; !stale && i < b->ctxs.size(); ++i)
    stale = b->sizes[i] != b->ctxs[i]->cap_N || b->gens[i] != b->ctxs[i]->graph_gen;
  if (stale) {
    int rc = batch_build(b);
    if (rc) return rc;
  }
  // each context's own work (catalog copies) is ordered before the batch
  for (sub_ctx* c : b->ctxs) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) {
      batch_err(b, "context stream: %s", cudaGetErrorString(e));
      return SUB_ECUDA;
    }
  }
  cudaError_t e = cudaEventRecord(b->ev0, b->stream);
  if (!e) e = cudaGraphLaunch(b->exec, b->stream);
  if (!e) e = cudaEventRecord(b->ev1, b->stream);
  if (!e) e = cudaStreamSynchronize(b->stream);
  if (!e) e = cudaEventElapsedTime(&b->last_ms, b->ev0, b->ev1);
  if (e) {
    batch_err(b, "batch launch: %s", cudaGetErrorString(e));
    return SUB_ECUDA;
  }
  int status = SUB_OK;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    b->ctxs[i]->ran = true;
    int rc = ctx_fill_stats(b->ctxs[i], stats ? &stats[i] : nullptr);
    if (rc != SUB_OK && (status == SUB_OK || status == SUB_ENOTCONVERGED)) status = rc;
  }
  return status;
}

extern "C" float sub_batch_last_ms(const sub_batch* b) { return b ? b->last_ms : 0.0f; }

extern "C" const char* sub_batch_last_error(const sub_batch* b) {
  return b ? b->err.c_str() : "null batch";
}

extern "C" void sub_batch_destroy(sub_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

extern "C" int sub_test_hooks(sub_ctx* c, int32_t flags) {
  if (!c) return SUB_EINVAL;
  if (flags & ~SUB_TEST_SKIP_CATALOG_COPIES) {
    ctx_set_err(c, "unknown test hook flags 0x%x", (unsigned)flags);
    return SUB_EINVAL;
  }
  ctx_set_test_flags(c, flags);
  return SUB_OK;
}

extern "C" int sub_set_grid_div(sub_ctx* c, int32_t div) {
  if (!c) return SUB_EINVAL;
  if (div < 1 || div > 64) {
    ctx_set_err(c, "grid divisor %d is outside 1 .. 64", div);
    return SUB_EINVAL;
  }
  ctx_set_grid_div(c, div);
  return SUB_OK;
}

extern "C" int sub_set_tuning(sub_ctx* c, int32_t knob, int32_t value) {
  if (!c) return SUB_EINVAL;
  const int rc = ctx_set_tuning(c, knob, value);
  if (rc) ctx_set_err(c, "launch setting %d = %d is not allowed for this context", knob, value);
  return rc;
}

// ============================================================================ server

namespace {

struct Job {
  int64_t id = 0;
  double T_obs = 0.0;
  const double *A = nullptr, *f = nullptr, *fdot = nullptr;
  int64_t n = 0;
  double* sg_out = nullptr;
  int64_t cap = 0;
  uint8_t* mask_out = nullptr;
  bool generated = false;  // the catalog is drawn on the device from (seed, gamma, shape)
  bool paper = false;      // ... or from (seed, pop): the paper's population model
  uint64_t seed = 0;
  double gamma = 0.0, shape = 0.0;
  sub_population pop = {};
  Clock::time_point t_submit, t_admit, t_done;
};

struct Slot {
  sub_server* srv = nullptr;
  sub_ctx* ctx = nullptr;
  bool busy = false;
  Job job;
  uint64_t last_use = 0;
  // Page-locked staging of the results, for callers whose buffers are pageable: a copy from
  // the device into pageable memory returns only once it is done, which would hold the
  // worker (and every other job's admission) until this job's whole run had finished.
  double* h_sg = nullptr;
  uint8_t* h_mask = nullptr;
  int64_t h_sg_cap = 0, h_mask_cap = 0;
  bool stage_sg = false, stage_mask = false;  // this job's results go through the staging
};

void free_staging(Slot* sl) {
  if (sl->h_sg) cudaFreeHost(sl->h_sg);
  if (sl->h_mask) cudaFreeHost(sl->h_mask);
  sl->h_sg = nullptr;
  sl->h_mask = nullptr;
  sl->h_sg_cap = sl->h_mask_cap = 0;
}

// True for host memory the GPU can copy into asynchronously (page-locked or registered).
bool page_locked(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

}  // namespace

struct sub_server {
  sub_server_params p;
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::vector<Slot*> slots;
  std::vector<Slot*> finished;
  std::vector<sub_job_result> results;
  bool stop = false;
  int inflight = 0;
  int64_t pool_bytes = 0, peak_bytes = 0;
  uint64_t tick = 0;
  int64_t contexts_created = 0;
  std::string err;
};

static int64_t bins_of(double T_obs, double f_min, double f_max) {
  int64_t lo = (int64_t)std::ceil(f_min * T_obs), hi = (int64_t)std::floor(f_max * T_obs);
  return hi >= lo ? hi - lo + 1 : 0;
}

// Device bytes of a context before it exists: the per-bin buffers (about 130 B/bin), the
// 16 MB of hot-bin replicas and the per-source buffers (94 B/source), rounded up.
static int64_t predicted_bytes(const sub_server* s, double T_obs, int64_t n) {
  const int64_t nb = bins_of(T_obs, s->p.f_min, s->p.f_max);
  return nb * 136 + ((int64_t)24 << 20) + n * 96;
}

static void CUDART_CB job_done(void* arg) {
  Slot* sl = static_cast<Slot*>(arg);
  sub_server* s = sl->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    sl->job.t_done = Clock::now();
    s->finished.push_back(sl);
  }
  s->cv_work.notify_one();
}

static double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

static void push_result(sub_server* s, const Job& j, int status, const sub_stats* st,
                        float gpu_ms) {
  sub_job_result r;
  std::memset(&r, 0, sizeof(r));
  r.job_id = j.id;
  r.status = status;
  if (st) r.stats = *st;
  r.latency_ms = ms_between(j.t_submit, j.t_done);
  r.queue_ms = ms_between(j.t_submit, j.t_admit);
  r.gpu_ms = gpu_ms;
  std::lock_guard<std::mutex> lk(s->mu);
  s->results.push_back(r);
  s->cv_done.notify_all();
}

static Slot* make_slot(sub_server* s, double T_obs, int64_t cap, int* status);

// A context for job j: an idle one with the same T_obs and room for the catalog, else a new
// one if the budget allows (idle contexts are destroyed, least recently used first, to make
// room).  Returns null when the job must wait for running jobs to finish.
// With idle_only, only an idle pooled context is taken (no context is created or replaced):
// the rule for jobs admitted past a queue head that has to wait.
static Slot* acquire_slot(sub_server* s, const Job& j, int* fail_status, bool idle_only) {
  *fail_status = SUB_OK;
  Slot* best = nullptr;
  for (Slot* sl : s->slots) {
    if (sl->busy || sl->ctx->p.T_obs != j.T_obs || sl->ctx->cap_N < j.n) continue;
    if (!best || sl->ctx->cap_N < best->ctx->cap_N) best = sl;
  }
  if (best || idle_only) return best;
  if (s->p.max_contexts > 0 && (int)s->slots.size() >= s->p.max_contexts) {
    // At the pool limit a job that a busy context could take waits for it: replacing an
    // idle context of another observation time would only move the shortage there, and
    // building a context costs far more than one job.
    for (Slot* sl : s->slots)
      if (sl->busy && sl->ctx->p.T_obs == j.T_obs && sl->ctx->cap_N >= j.n) return nullptr;
    // Otherwise an idle context that cannot take this job is replaced; with none idle the
    // job waits.
    Slot* victim = nullptr;
    for (Slot* sl : s->slots)
      if (!sl->busy && (!victim || sl->last_use < victim->last_use)) victim = sl;
    if (!victim) return nullptr;
    s->pool_bytes -= sub_device_bytes(victim->ctx);
    sub_destroy(victim->ctx);
    free_staging(victim);
    s->slots.erase(std::find(s->slots.begin(), s->slots.end(), victim));
    delete victim;
  }
  const int64_t need = predicted_bytes(s, j.T_obs, j.n);
  const uint64_t budget = s->p.hbm_budget;
  if (budget && (uint64_t)need > budget) {
    *fail_status = SUB_EBUDGET;
    return nullptr;
  }
  while (budget && (uint64_t)(s->pool_bytes + need) > budget) {
    Slot* victim = nullptr;
    for (Slot* sl : s->slots)
      if (!sl->busy && (!victim || sl->last_use < victim->last_use)) victim = sl;
    if (!victim) return nullptr;
    s->pool_bytes -= sub_device_bytes(victim->ctx);
    sub_destroy(victim->ctx);
    free_staging(victim);
    s->slots.erase(std::find(s->slots.begin(), s->slots.end(), victim));
    delete victim;
  }
  int st = SUB_OK;
  Slot* sl = make_slot(s, j.T_obs, j.n, &st);
  if (!sl) *fail_status = st;
  return sl;
}

// Enqueue job j on slot sl: catalog in, run, results out, then the completion callback.
static int launch_job(sub_server* s, Slot* sl, Job& j) {
  sub_ctx* c = sl->ctx;
  const int64_t before = sub_device_bytes(c);
  int rc = j.paper       ? sub_load_population(c, j.n, j.seed, &j.pop, 1)
           : j.generated ? sub_load_generated(c, j.n, j.seed, j.gamma, j.shape, 1)
                         : sub_load_catalog(c, j.A, j.f, j.fdot, j.n, SUB_HOST);
  s->pool_bytes += sub_device_bytes(c) - before;
  if (rc) return rc;
  rc = sub_run(c, nullptr);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  // results go straight into page-locked caller buffers, else through the slot's staging
  // (finalize copies them on): either way this thread only enqueues
  sl->stage_sg = j.sg_out && !page_locked(j.sg_out);
  sl->stage_mask = j.mask_out && j.n > 0 && !page_locked(j.mask_out);
  const int64_t nb = c->grid.nb;
  if (sl->stage_sg && sl->h_sg_cap < nb) {
    if (sl->h_sg) cudaFreeHost(sl->h_sg);
    sl->h_sg = nullptr;
    sl->h_sg_cap = 0;
    e = cudaHostAlloc((void**)&sl->h_sg, (size_t)nb * 8, cudaHostAllocDefault);
    if (!e) sl->h_sg_cap = nb;
  }
  if (!e && sl->stage_mask && sl->h_mask_cap < j.n) {
    if (sl->h_mask) cudaFreeHost(sl->h_mask);
    sl->h_mask = nullptr;
    sl->h_mask_cap = 0;
    e = cudaHostAlloc((void**)&sl->h_mask, (size_t)j.n, cudaHostAllocDefault);
    if (!e) sl->h_mask_cap = j.n;
  }
  if (!e && j.sg_out)
    e = cudaMemcpyAsync(sl->stage_sg ? sl->h_sg : j.sg_out, c->Sg, (size_t)nb * 8,
                        cudaMemcpyDeviceToHost, c->stream);
  if (!e && j.mask_out && j.n > 0)
    e = cudaMemcpyAsync(sl->stage_mask ? sl->h_mask : j.mask_out, c->resolved, (size_t)j.n,
                        cudaMemcpyDeviceToHost, c->stream);
  sl->busy = true;
  sl->job = j;
  sl->last_use = ++s->tick;
  if (!e) e = cudaLaunchHostFunc(c->stream, job_done, sl);
  if (e) {
    sl->busy = false;
    return SUB_ECUDA;
  }
  return SUB_OK;
}

static void finalize(sub_server* s, Slot* sl) {
  sub_stats st;
  std::memset(&st, 0, sizeof(st));
  int status = ctx_fill_stats(sl->ctx, &st);
  if (sl->stage_sg) {
    std::memcpy(sl->job.sg_out, sl->h_sg, (size_t)sl->ctx->grid.nb * 8);
    sl->job.t_done = Clock::now();
  }
  if (sl->stage_mask) {
    std::memcpy(sl->job.mask_out, sl->h_mask, (size_t)sl->job.n);
    sl->job.t_done = Clock::now();
  }
  float gpu_ms = 0.0f;
  float pre = 0.0f, loop = 0.0f;
  if (sub_get_timing(sl->ctx, &pre, &loop, &gpu_ms) != SUB_OK) gpu_ms = 0.0f;
  Job j = sl->job;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    sl->busy = false;
    s->inflight -= 1;
  }
  push_result(s, j, status, &st, gpu_ms);
}

static void worker_main(sub_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Slot*> fin;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::microseconds(200), [&] {
        return s->stop || !s->finished.empty() ||
               (!s->queue.empty() && s->inflight < s->p.max_inflight);
      });
      fin.swap(s->finished);
      if (s->stop && s->inflight == 0 && fin.empty()) break;
    }
    for (Slot* sl : fin) finalize(s, sl);
    // Admission in arrival order.  When the job at the head has to wait (for memory, or
    // for a busy context it alone fits), later jobs that an idle pooled context can take
    // start past it: they use no memory or context the head could have had (an idle context
    // that fits the head would have gone to the head), so it is not delayed by them.
    size_t pos = 0;  // queue position to try next (jobs before it wait)
    for (;;) {
      Job j;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop || pos >= s->queue.size() || s->inflight >= s->p.max_inflight) break;
        j = s->queue[pos];
      }
      int fail = SUB_OK;
      Slot* sl = acquire_slot(s, j, &fail, pos > 0);
      if (!sl && fail == SUB_OK) {
        ++pos;  // this job waits; a later one may fit an idle context
        if (pos > 256) break;
        continue;
      }
      {
        // only this thread removes jobs, and submissions only append: j is still at pos
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.erase(s->queue.begin() + (std::ptrdiff_t)pos);
        if (sl) s->inflight += 1;
      }
      j.t_admit = Clock::now();
      if (!sl) {
        j.t_done = j.t_admit;
        push_result(s, j, fail, nullptr, 0.0f);
        continue;
      }
      int rc = launch_job(s, sl, j);
      if (s->pool_bytes > s->peak_bytes) s->peak_bytes = s->pool_bytes;
      if (rc) {
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->inflight -= 1;
        }
        cudaStreamSynchronize(sl->ctx->stream);
        j.t_done = Clock::now();
        push_result(s, j, rc, nullptr, 0.0f);
      }
    }
  }
}

extern "C" int sub_server_params_default(sub_server_params* p) {
  if (!p) return SUB_EINVAL;
  std::memset(p, 0, sizeof(*p));
  sub_params d;
  sub_params_default(&d);
  p->hbm_budget = 0;
  p->max_inflight = 16;
  p->window = d.window;
  p->estimator = d.estimator;
  p->precision = d.precision;
  p->max_iter = d.max_iter;
  p->tdi2 = d.tdi2;
  p->grid_div = 1;
  p->f_min = d.f_min;
  p->f_max = d.f_max;
  p->rho_th = d.rho_th;
  p->kappa = d.kappa;
  return SUB_OK;
}

extern "C" int sub_server_create(const sub_server_params* p, sub_server** out) {
  if (!out || !p) return SUB_EINVAL;
  *out = nullptr;
  if (p->max_inflight < 1 || p->max_inflight > 256 || p->grid_div < 1 || p->grid_div > 64 ||
      p->max_contexts < 0) {
    set_global_error("sub_server_create: max_inflight must be 1 .. 256, grid_div 1 .. 64, "
                     "max_contexts >= 0");
    return SUB_EINVAL;
  }
  sub_server* s = new (std::nothrow) sub_server;
  if (!s) return SUB_ENOMEM;
  s->p = *p;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    set_global_error("sub_server_create: no CUDA device");
    return SUB_ECUDA;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return SUB_OK;
}

extern "C" int sub_server_submit(sub_server* s, int64_t job_id, double T_obs, const double* A,
                                 const double* f, const double* fdot, int64_t n, double* S_gal,
                                 int64_t cap, uint8_t* mask) {
  if (!s) return SUB_EINVAL;
  if (n < 0 || (n > 0 && (!A || !f || !fdot)) || !(T_obs > 0.0)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "sub_server_submit: bad catalog or T_obs";
    return SUB_EINVAL;
  }
  if (S_gal && cap < bins_of(T_obs, s->p.f_min, s->p.f_max)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "sub_server_submit: S_gal buffer smaller than the number of bins";
    return SUB_EINVAL;
  }
  Job j;
  j.id = job_id;
  j.T_obs = T_obs;
  j.A = A;
  j.f = f;
  j.fdot = fdot;
  j.n = n;
  j.sg_out = S_gal;
  j.cap = cap;
  j.mask_out = mask;
  j.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return SUB_ESTATE;
    s->queue.push_back(j);
  }
  s->cv_work.notify_one();
  return SUB_OK;
}

extern "C" int sub_server_submit_generated(sub_server* s, int64_t job_id, double T_obs,
                                           int64_t n, uint64_t seed, double gamma,
                                           double shape, double* S_gal, int64_t cap,
                                           uint8_t* mask) {
  if (!s) return SUB_EINVAL;
  if (n < 0 || n > ((int64_t)1 << 40) || !(T_obs > 0.0) || !(gamma >= -8.0 && gamma <= 10.0) ||
      !(shape >= 1.0 && shape <= 1e6)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "sub_server_submit_generated: bad size, T_obs or population";
    return SUB_EINVAL;
  }
  if (S_gal && cap < bins_of(T_obs, s->p.f_min, s->p.f_max)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "sub_server_submit_generated: S_gal buffer smaller than the number of bins";
    return SUB_EINVAL;
  }
  Job j;
  j.id = job_id;
  j.T_obs = T_obs;
  j.n = n;
  j.sg_out = S_gal;
  j.cap = cap;
  j.mask_out = mask;
  j.generated = true;
  j.seed = seed;
  j.gamma = gamma;
  j.shape = shape;
  j.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return SUB_ESTATE;
    s->queue.push_back(j);
  }
  s->cv_work.notify_one();
  return SUB_OK;
}

extern "C" int sub_server_submit_population(sub_server* s, int64_t job_id, double T_obs,
                                            int64_t n, uint64_t seed, const sub_population* pop,
                                            double* S_gal, int64_t cap, uint8_t* mask) {
  if (!s) return SUB_EINVAL;
  if (!pop || n < 0 || n > ((int64_t)1 << 40) || !(T_obs > 0.0) ||
      !(pop->alpha_g >= 1.0 && pop->alpha_g <= 1e3) || !(pop->rho >= 0.0 && pop->rho < 1.0) ||
      !(pop->beta_g > 0.0) || !(pop->sigma > 0.0) ||
      !(pop->alpha_pl >= -10.0 && pop->alpha_pl <= 8.0)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "sub_server_submit_population: bad size, T_obs or population";
    return SUB_EINVAL;
  }
  if (S_gal && cap < bins_of(T_obs, s->p.f_min, s->p.f_max)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "sub_server_submit_population: S_gal buffer smaller than the number of bins";
    return SUB_EINVAL;
  }
  Job j;
  j.id = job_id;
  j.T_obs = T_obs;
  j.n = n;
  j.sg_out = S_gal;
  j.cap = cap;
  j.mask_out = mask;
  j.generated = true;
  j.paper = true;
  j.seed = seed;
  j.pop = *pop;
  j.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return SUB_ESTATE;
    s->queue.push_back(j);
  }
  s->cv_work.notify_one();
  return SUB_OK;
}

extern "C" int32_t sub_server_poll(sub_server* s, sub_job_result* out, int32_t cap,
                                   int32_t timeout_ms) {
  if (!s || !out || cap < 1) return 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->results.empty() && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                        [&] { return !s->results.empty(); });
  int32_t k = 0;
  while (k < cap && !s->results.empty()) {
    out[k++] = s->results.front();
    s->results.erase(s->results.begin());
  }
  return k;
}

extern "C" int sub_server_info(sub_server* s, sub_server_stats* st) {
  if (!s || !st) return SUB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  st->queued = (int64_t)s->queue.size();
  st->inflight = s->inflight;
  st->contexts = (int32_t)s->slots.size();
  st->device_bytes = s->pool_bytes;
  st->peak_device_bytes = s->peak_bytes;
  st->contexts_created = s->contexts_created;
  return SUB_OK;
}

// A context for T_obs with room for `cap` sources and its graph built, ready for jobs.
static Slot* make_slot(sub_server* s, double T_obs, int64_t cap, int* status) {
  sub_params prm;
  sub_params_default(&prm);
  prm.T_obs = T_obs;
  prm.f_min = s->p.f_min;
  prm.f_max = s->p.f_max;
  prm.window = s->p.window;
  prm.estimator = s->p.estimator;
  prm.rho_th = s->p.rho_th;
  prm.kappa = s->p.kappa;
  prm.max_iter = s->p.max_iter;
  prm.tdi2 = s->p.tdi2;
  prm.precision = s->p.precision;
  sub_ctx* c = nullptr;
  *status = sub_create(&prm, nullptr, &c);
  if (*status) return nullptr;
  if (s->p.grid_div > 1) sub_set_grid_div(c, s->p.grid_div);
  if (cap > 0) *status = ctx_prepare(c, cap);
  if (*status) {
    sub_destroy(c);
    return nullptr;
  }
  Slot* sl = new Slot;
  sl->srv = s;
  sl->ctx = c;
  s->slots.push_back(sl);
  s->pool_bytes += sub_device_bytes(c);
  if (s->pool_bytes > s->peak_bytes) s->peak_bytes = s->pool_bytes;
  s->contexts_created += 1;
  return sl;
}

extern "C" int sub_server_prewarm(sub_server* s, double T_obs, int64_t n_sources,
                                  int32_t count) {
  if (!s || !(T_obs > 0.0) || n_sources < 0 || count < 0) return SUB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);  // the worker touches the pool only for jobs
  if (!s->queue.empty() || s->inflight > 0) {
    s->err = "sub_server_prewarm: jobs are queued or running";
    return SUB_ESTATE;
  }
  for (int32_t i = 0; i < count; ++i) {
    const int64_t need = predicted_bytes(s, T_obs, n_sources);
    if (s->p.hbm_budget && (uint64_t)(s->pool_bytes + need) > s->p.hbm_budget) {
      s->err = "sub_server_prewarm: the budget is full";
      return SUB_EBUDGET;
    }
    int st = SUB_OK;
    if (!make_slot(s, T_obs, n_sources, &st)) {
      s->err = "sub_server_prewarm: context creation failed";
      return st;
    }
  }
  return SUB_OK;
}

extern "C" const char* sub_server_last_error(sub_server* s) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  return s->err.empty() ? "no error" : s->err.c_str();
}

extern "C" void sub_server_destroy(sub_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();  // jobs not admitted yet are dropped
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Slot* sl : s->slots) {
    sub_destroy(sl->ctx);
    free_staging(sl);
    delete sl;
  }
  delete s;
}
