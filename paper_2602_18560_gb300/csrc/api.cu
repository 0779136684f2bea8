// C ABI of the GB300 subtraction library (declarations and contracts in include/gbsub.h).
//
// A context owns the grid, the per-bin tables, the catalog copy and every work buffer of a
// run.  sub_run launches one CUDA graph: a pre-loop part (clear the spectrum, one pass over
// the catalog) followed by a conditional WHILE node whose body is one iteration of App. D
// (estimate S_gal, SNR of the candidates, remove the resolved ones, loop control).  The
// loop condition is set on the device, so a run crosses the host/device boundary only when
// the caller asks for results.

#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdarg>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gbsub.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace gbsub;

#include "context.cuh"

static std::string g_create_err = "no error";

namespace gbsub {
// Message of a failure that has no context (sub_create, sub_running_mean_noalloc).
void set_global_error(const char* msg) { g_create_err = msg; }
}  // namespace gbsub

static void set_err(sub_ctx* c, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_err = buf;
}

#define CU(call, ctx)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_err(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return SUB_ECUDA;                                                            \
    }                                                                              \
  } while (0)

static int dalloc(sub_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (c->p.hbm_budget && (uint64_t)(c->bytes + (int64_t)bytes) > c->p.hbm_budget) {
    set_err(c, "device memory budget exceeded: need %lld more bytes, hold %lld of %llu",
            (long long)bytes, (long long)c->bytes, (unsigned long long)c->p.hbm_budget);
    return SUB_EBUDGET;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_err(c, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return SUB_ENOMEM;
  }
  c->allocs.push_back(std::make_pair(*p, (int64_t)bytes));
  c->bytes += (int64_t)bytes;
  return SUB_OK;
}

static void dfree(sub_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i) {
    if (c->allocs[i].first == p) {
      c->bytes -= c->allocs[i].second;
      c->allocs.erase(c->allocs.begin() + i);
      break;
    }
  }
  cudaFree(p);
}

static void drop_graph(sub_ctx* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->exec = nullptr;
  c->graph = nullptr;
  c->graph_cap = -1;
  c->graph_gen += 1;
}

extern "C" int sub_params_default(sub_params* p) {
  if (!p) return SUB_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->T_obs = 4.0 * 365.25 * 86400.0;
  p->f_min = 1e-4;
  p->f_max = 1e-2;
  p->window = 2000;
  p->estimator = SUB_MEAN;
  p->rho_th = 7.0;
  p->kappa = 1.0 / 7.0;
  p->max_iter = 100;
  p->tdi2 = 1;
  p->precision = SUB_FP64;
  p->conv_rtol = 0.0;
  p->hbm_budget = 0;
  return SUB_OK;
}

static int validate(const sub_params* p, int64_t* k_lo, int64_t* n) {
  if (!p) { set_err(nullptr, "params is null"); return SUB_EINVAL; }
  if (!(p->T_obs > 0.0) || !std::isfinite(p->T_obs)) { set_err(nullptr, "T_obs must be > 0"); return SUB_EINVAL; }
  if (!(p->f_min > 0.0) || !(p->f_max > p->f_min) || !std::isfinite(p->f_max)) {
    set_err(nullptr, "band must satisfy 0 < f_min < f_max");
    return SUB_EINVAL;
  }
  if (p->window < 1 || p->window > kMaxWindow) { set_err(nullptr, "window must be in 1..%d", kMaxWindow); return SUB_EINVAL; }
  if (p->estimator < SUB_MEAN || p->estimator > SUB_MEDIAN_MEAN) { set_err(nullptr, "unknown estimator %d", p->estimator); return SUB_EINVAL; }
  if (!(p->rho_th > 0.0) || !(p->kappa >= 0.0)) { set_err(nullptr, "rho_th must be > 0 and kappa >= 0"); return SUB_EINVAL; }
  if (p->max_iter < 1) { set_err(nullptr, "max_iter must be >= 1"); return SUB_EINVAL; }
  if (p->precision < SUB_FP64 || p->precision > SUB_FP64_STRICT) { set_err(nullptr, "unknown precision %d", p->precision); return SUB_EINVAL; }
  if (!(p->conv_rtol >= 0.0)) { set_err(nullptr, "conv_rtol must be >= 0"); return SUB_EINVAL; }
  double a = std::ceil(p->f_min * p->T_obs);
  double b = std::floor(p->f_max * p->T_obs);
  if (!(b >= a) || b - a + 1 > 16.0e6) { set_err(nullptr, "band holds %g bins (1 .. 16e6 allowed)", b - a + 1); return SUB_EINVAL; }
  *k_lo = (int64_t)a;
  *n = (int64_t)(b - a + 1);
  return SUB_OK;
}

static SmoothPlan make_plan(int W, int64_t n) {
  SmoothPlan pl = {};
  pl.W = W;
  int kc = ((W + 31) / 32) * 32;
  if (kc < 32) kc = 32;
  pl.Kc = kc;
  pl.nw = kc / 32;
  pl.nch = (int)((n + kc - 1) / kc);
  int kp = 64;  // sort width: a power of two >= Kc, and two elements for each of >= 32 threads
  while (kp < kc) kp <<= 1;
  pl.kpad = kp;
  pl.nsm = 0;
  pl.fp32_keys = 0;
  pl.key_scale = 1.0;
  return pl;
}

extern "C" int sub_create(const sub_params* p, void* stream, sub_ctx** out) {
  if (!out) { set_err(nullptr, "out is null"); return SUB_EINVAL; }
  *out = nullptr;
  int64_t k_lo, n;
  int rc = validate(p, &k_lo, &n);
  if (rc) return rc;
  sub_ctx* c = new (std::nothrow) sub_ctx();
  if (!c) { set_err(nullptr, "host allocation failed"); return SUB_ENOMEM; }
  c->p = *p;
  c->grid.T = p->T_obs;
  c->grid.T2 = p->T_obs * p->T_obs;
  c->grid.t5 = p->T_obs / 5.0;
  c->grid.k_lo = k_lo;
  c->grid.nb = n;
  {
    // T_obs = mT 2^eT with mT the 53-bit integer mantissa (for the exact f T in the prepass)
    int ex = 0;
    double m = std::frexp(p->T_obs, &ex);  // T = m 2^ex, m in [0.5, 1)
    c->grid.mT = (unsigned long long)std::ldexp(m, 53);
    c->grid.eT = ex - 53;
    c->grid.T2f = (float)(p->T_obs * p->T_obs);
    // the same with the trailing zero bits of the mantissa dropped: whole seconds of
    // observation time leave at most 32 bits, and f T then takes two 32-bit products
    unsigned long long tq = c->grid.mT;
    int etq = c->grid.eT;
    while (tq && !(tq & 1ull)) {
      tq >>= 1;
      ++etq;
    }
    c->grid.short_t = (tq > 0 && tq < (1ull << 32)) ? 1 : 0;
    c->grid.tq = c->grid.short_t ? (unsigned)tq : 0u;
    c->grid.etq = etq;
  }
  c->plan = make_plan(p->window, n);
  c->plan.fp32_keys = p->precision == SUB_MIXED ? 1 : 0;  // FP32 median selection
  auto fail = [&](int code) {
    g_create_err = c->err;
    sub_destroy(c);
    return code;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { c->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return fail(SUB_ECUDA); }
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (c->nsm <= 0) c->nsm = 1;
  c->plan.nsm = c->nsm;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    // a blocking stream orders itself after work on the legacy default stream
    e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) { c->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e); return fail(SUB_ECUDA); }
    c->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { c->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e); return fail(SUB_ECUDA); }
  configure_kernels();
  plan_grids(c->plan);
  c->nsm_run = c->nsm;
  {
    cudaEvent_t* evs[] = {&c->ev_start, &c->ev_pre, &c->ev_end, &c->ev_k[0], &c->ev_k[1]};
    for (cudaEvent_t* ev : evs) {
      e = cudaEventCreate(ev);
      if (e != cudaSuccess) { c->err = std::string("cudaEventCreate: ") + cudaGetErrorString(e); return fail(SUB_ECUDA); }
    }
  }
  const SmoothPlan& pl = c->plan;
  int64_t ncell = (int64_t)pl.nch * pl.Kc;
  struct { void** p; size_t b; } want[] = {
      {(void**)&c->S, (size_t)n * 8}, {(void**)&c->R, (size_t)n * 8}, {(void**)&c->gq, (size_t)n * 8},
      {(void**)&c->Gf, (size_t)n * 4}, {(void**)&c->invSf, (size_t)n * 4},
      {(void**)&c->acc, (size_t)n * 32}, {(void**)&c->inv_f, (size_t)n * 4},
      {(void**)&c->rep.w, (size_t)kAccReplicas * (n < kAccReplicaBins ? n : kAccReplicaBins) * 16},
      {(void**)&c->P, (size_t)n * 8}, {(void**)&c->Sg, (size_t)n * 8},
      {(void**)&c->sig, (size_t)pl.nch * 4}, {(void**)&c->estimate_in, (size_t)n * 8},
      {(void**)&c->dirty, (size_t)pl.nch * 2},
      {(void**)&c->lists, (size_t)kNumLists * (pl.nch + 1) * 4},
      {(void**)&c->list_counts, (size_t)kNumLists * 4},
      {(void**)&c->pre_lo, (size_t)ncell * 8}, {(void**)&c->pre_hi, (size_t)ncell * 8},
      {(void**)&c->uflow, (size_t)pl.nch * 4},
      {(void**)&c->rs, sizeof(RunState)}, {(void**)&c->new_hist, (size_t)p->max_iter * 4},
      {(void**)&c->dcat, sizeof(CatalogRef)},
  };
  for (auto& w : want) {
    rc = dalloc(c, w.p, w.b);
    if (rc) return fail(rc);
  }
  c->rep.nbins = n < kAccReplicaBins ? n : kAccReplicaBins;
  if (p->estimator != SUB_MEAN) {
    rc = dalloc(c, (void**)&c->skey, (size_t)ncell * 8);
    if (!rc) rc = dalloc(c, (void**)&c->srank, (size_t)ncell * 2);
    if (!rc && p->estimator == SUB_MEDIAN_MEAN) rc = dalloc(c, (void**)&c->M, (size_t)n * 8);
    if (rc) return fail(rc);
  }
  e = cudaMallocHost((void**)&c->h_rs, sizeof(RunState));
  if (e != cudaSuccess) { c->err = "cudaMallocHost failed"; return fail(SUB_ENOMEM); }
  std::memset(c->h_rs, 0, sizeof(RunState));
  launch_tables(c->grid, p->tdi2, c->S, c->R, c->gq, c->Gf, c->invSf, c->stream);
  e = cudaMemsetAsync(c->Sg, 0, (size_t)n * 8, c->stream);
  // The FP32 keys of the mixed-precision median are the powers times 2^e: the spectrum
  // holds less than 2^63 S_instr per bin, so with e = 59 - ilogb(max S_instr) every power
  // is below 2^123, and the smallest non-zero power (2^-64 S_instr) stays far above the
  // FP32 normal range over any band whose S_instr spans less than 2^60.
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->rs->max_p_bits, 0, 8, c->stream);
  if (e == cudaSuccess) launch_max_bits(c->S, n, &c->rs->max_p_bits, c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_rs, c->rs, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) { c->err = std::string("table build: ") + cudaGetErrorString(e); return fail(SUB_ECUDA); }
  {
    double smax;
    unsigned long long b = c->h_rs->max_p_bits;
    std::memcpy(&smax, &b, 8);
    int ex = smax > 0.0 ? std::ilogb(smax) : 0;
    c->plan.key_scale = std::ldexp(1.0, 59 - ex);
  }
  *out = c;
  return SUB_OK;
}

// Per-source buffers for catalogs of up to n sources (kept when they already fit).
static int reserve_sources(sub_ctx* c, int64_t n) {
  if (n > c->cap_N || c->A == nullptr) {
    drop_graph(c);
    dfree(c, c->A); dfree(c, c->f); dfree(c, c->fdot); dfree(c, c->resolved);
    void* cds[] = {c->cd.src, c->cd.pk, c->cd.len, c->cd.a2, c->cd.amp, c->cd.lo, c->cd.hi,
                   c->cd.res, c->cd.wide};
    for (void* q : cds) dfree(c, q);
    c->A = c->f = c->fdot = nullptr;
    c->resolved = nullptr;
    c->cd = Cands{};
    c->cap_N = 0;
    c->N = -1;
    int rc;
    size_t m = (size_t)(n > 0 ? n : 1);
    // Candidate arrays hold every source in the worst case (a catalog of bright sources).
    if ((rc = dalloc(c, (void**)&c->A, m * 8)) || (rc = dalloc(c, (void**)&c->f, m * 8)) ||
        (rc = dalloc(c, (void**)&c->fdot, m * 8)) || (rc = dalloc(c, (void**)&c->resolved, m)) ||
        (rc = dalloc(c, (void**)&c->cd.src, m * 8)) || (rc = dalloc(c, (void**)&c->cd.pk, m * 16)) ||
        (rc = dalloc(c, (void**)&c->cd.len, m * 4)) ||
        (rc = dalloc(c, (void**)&c->cd.a2, m * 8)) || (rc = dalloc(c, (void**)&c->cd.amp, m * 8)) ||
        (rc = dalloc(c, (void**)&c->cd.lo, m * 8)) ||
        (rc = dalloc(c, (void**)&c->cd.hi, m * 8)) || (rc = dalloc(c, (void**)&c->cd.res, m)) ||
        (rc = dalloc(c, (void**)&c->cd.wide, m * 8))) {
      return rc;
    }
    c->cap_N = (int64_t)m;
  }
  return SUB_OK;
}

// Device address of page-locked host memory, or nullptr when p is not such memory.
static const double* mapped_address(const double* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer leaves a (non-sticky) error behind
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
  return static_cast<const double*>(at.devicePointer);
}

extern "C" int sub_load_catalog(sub_ctx* c, const double* A, const double* f, const double* fdot,
                                int64_t n, int where) {
  if (!c) return SUB_EINVAL;
  if (n < 0 || (n > 0 && (!A || !f || !fdot)) ||
      (where != SUB_HOST && where != SUB_DEVICE && where != SUB_HOST_MAPPED)) {
    set_err(c, "invalid catalog arguments");
    return SUB_EINVAL;
  }
  if (n > ((int64_t)1 << 40)) { set_err(c, "catalog too large"); return SUB_EINVAL; }
  CatalogRef ref = {nullptr, nullptr, nullptr, (long long)n, 1, 0};
  if (where == SUB_HOST_MAPPED && n > 0) {
    ref.A = mapped_address(A);
    ref.f = mapped_address(f);
    ref.fdot = mapped_address(fdot);
    if (!ref.A || !ref.f || !ref.fdot) {
      set_err(c, "SUB_HOST_MAPPED needs page-locked (pinned) host memory");
      return SUB_EINVAL;
    }
    ref.staged = 0;
  }
  {
    int rc = reserve_sources(c, n);
    if (rc) return rc;
  }
  if (where != SUB_HOST_MAPPED) {
    ref.A = c->A;
    ref.f = c->f;
    ref.fdot = c->fdot;
    if (n > 0) {
      cudaMemcpyKind k = where == SUB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
      CU(cudaMemcpyAsync(c->A, A, (size_t)n * 8, k, c->stream), c);
      CU(cudaMemcpyAsync(c->f, f, (size_t)n * 8, k, c->stream), c);
      CU(cudaMemcpyAsync(c->fdot, fdot, (size_t)n * 8, k, c->stream), c);
    }
  }
  launch_set_catalog(c->dcat, ref, c->stream);
  CU(cudaGetLastError(), c);
  c->N = n;
  c->ran = false;
  c->cat_kind = where == SUB_HOST_MAPPED ? kCatHostMapped : kCatDevice;
  c->cat_host[0] = A;
  c->cat_host[1] = f;
  c->cat_host[2] = fdot;
  return SUB_OK;
}

extern "C" int sub_load_generated(sub_ctx* c, int64_t n, uint64_t seed, double gamma,
                                  double shape, int32_t fused) {
  if (!c) return SUB_EINVAL;
  if (n < 0 || n > ((int64_t)1 << 40) || !(gamma >= -8.0 && gamma <= 10.0) ||
      !(shape >= 1.0 && shape <= 1e6)) {
    set_err(c, "generated catalog: need 0 <= n <= 2^40, -8 <= gamma <= 10, 1 <= shape <= 1e6");
    return SUB_EINVAL;
  }
  {
    int rc = reserve_sources(c, n);
    if (rc) return rc;
  }
  if (fused) {
    launch_gen_setup(c->dcat, n, seed, gamma, shape, nullptr, nullptr, nullptr, c->stream);
  } else {
    launch_gen_setup(c->dcat, n, seed, gamma, shape, c->A, c->f, c->fdot, c->stream);
    launch_generate(c->dcat, 0, n, c->A, c->f, c->fdot, c->stream);
  }
  CU(cudaGetLastError(), c);
  c->N = n;
  c->ran = false;
  c->cat_kind = fused ? kCatGenerated : kCatDevice;
  return SUB_OK;
}

extern "C" int sub_load_population(sub_ctx* c, int64_t n, uint64_t seed, const sub_population* pop,
                                   int32_t fused) {
  if (!c) return SUB_EINVAL;
  if (!pop || n < 0 || n > ((int64_t)1 << 40) || !(pop->alpha_pl >= -10.0 && pop->alpha_pl <= 8.0) ||
      !(pop->alpha_g >= 1.0 && pop->alpha_g <= 1e3) || !(pop->beta_g > 0.0 && pop->beta_g <= 1e3) ||
      !(pop->mu_g >= -40.0 && pop->mu_g <= 0.0) || !(pop->mu >= -40.0 && pop->mu <= 0.0) ||
      !(pop->sigma > 0.0 && pop->sigma <= 10.0) || !(pop->rho >= 0.0 && pop->rho < 1.0)) {
    set_err(c, "population catalog: need 0 <= n <= 2^40, -10 <= alpha_pl <= 8, 1 <= alpha_g <= "
               "1e3, 0 < beta_g <= 1e3, -40 <= mu_g, mu <= 0, 0 < sigma <= 10, 0 <= rho < 1");
    return SUB_EINVAL;
  }
  {
    int rc = reserve_sources(c, n);
    if (rc) return rc;
  }
  PaperPop pp;
  pp.alpha_pl = pop->alpha_pl;
  pp.alpha_g = pop->alpha_g;
  pp.beta_g = pop->beta_g;
  pp.mu_g = pop->mu_g;
  pp.mu = pop->mu;
  pp.sigma = pop->sigma;
  pp.rho = pop->rho;
  if (fused) {
    launch_gen_setup_paper(c->dcat, n, seed, pp, nullptr, nullptr, nullptr, c->stream);
  } else {
    launch_gen_setup_paper(c->dcat, n, seed, pp, c->A, c->f, c->fdot, c->stream);
    launch_generate(c->dcat, 0, n, c->A, c->f, c->fdot, c->stream);
  }
  CU(cudaGetLastError(), c);
  c->N = n;
  c->ran = false;
  c->cat_kind = fused ? kCatGenerated : kCatDevice;
  return SUB_OK;
}

extern "C" int sub_get_catalog(sub_ctx* c, double* A, double* f, double* fdot, int64_t start,
                               int64_t n, int where) {
  if (!c) return SUB_EINVAL;
  if (where != SUB_HOST && where != SUB_DEVICE) { set_err(c, "bad where"); return SUB_EINVAL; }
  if (c->N < 0) { set_err(c, "no catalog loaded"); return SUB_ESTATE; }
  if (start < 0 || n < 0 || start + n > c->N || (n > 0 && (!A || !f || !fdot))) {
    set_err(c, "sub_get_catalog: need 0 <= start, start + n <= %lld and three buffers",
            (long long)c->N);
    return SUB_EINVAL;
  }
  if (n == 0) return SUB_OK;
  cudaStream_t st = c->stream;
  const size_t b = (size_t)n * 8;
  double* out[3] = {A, f, fdot};
  if (c->cat_kind == kCatGenerated) {
    if (where == SUB_DEVICE) {
      launch_generate(c->dcat, start, n, A, f, fdot, st);
    } else {  // through the (otherwise unused) catalog arrays
      launch_generate(c->dcat, start, n, c->A, c->f, c->fdot, st);
      const double* src[3] = {c->A, c->f, c->fdot};
      for (int i = 0; i < 3; ++i)
        CU(cudaMemcpyAsync(out[i], src[i], b, cudaMemcpyDeviceToHost, st), c);
    }
  } else {
    const double* dev[3] = {c->A, c->f, c->fdot};
    for (int i = 0; i < 3; ++i) {
      const double* src = (c->cat_kind == kCatHostMapped ? c->cat_host[i] : dev[i]) + start;
      CU(cudaMemcpyAsync(out[i], src, b, cudaMemcpyDefault, st), c);
    }
  }
  CU(cudaGetLastError(), c);
  CU(cudaStreamSynchronize(st), c);
  return SUB_OK;
}

// ---------------------------------------------------------------- enqueue helpers

// Prepass thresholds on r = sum of the fixed-point contributions, rho_0^2 = 4 r 2^-96.
// Both are lowered by 1e-12 relative so that rounding can only keep more sources: an extra
// candidate cannot change the result, since S_n >= S_instr makes rho <= rho_0.
static double thr_kappa_of(const sub_ctx* c) {
  double pre = c->p.kappa * c->p.rho_th;
  return pre * pre / 4.0 * kQScale * (1.0 - 1e-12);
}
static double thr_live_of(const sub_ctx* c) {
  return c->p.rho_th * c->p.rho_th / 4.0 * kQScale * (1.0 - 1e-12);
}

static Tables tables_of(const sub_ctx* c) {
  Tables t;
  t.S = c->S;
  t.R = c->R;
  t.gq = c->gq;
  t.Gf = c->Gf;
  t.invSf = c->invSf;
  return t;
}

static int snr_mode(const sub_ctx* c) {
  return c->p.precision;  // 0: FP64 with FP32 screen, 1: FP32 decides, 2: FP64 always
}

// While profiling, every launch is bracketed by an event pair and its device time added
// to the kernel's total (this synchronises after each launch).
struct KTimer {
  sub_ctx* c;
  cudaStream_t st;
  int k;
  KTimer(sub_ctx* c_, cudaStream_t st_, int k_) : c(c_), st(st_), k(k_) {
    if (c->profiling) cudaEventRecord(c->ev_k[0], st);
  }
  ~KTimer() {
    if (!c->profiling) return;
    cudaEventRecord(c->ev_k[1], st);
    cudaEventSynchronize(c->ev_k[1]);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_k[0], c->ev_k[1]);
    c->prof_ms[k] += ms;
    c->prof_n[k] += 1;
    if (c->prof_iter >= 0) {
      if ((int)c->prof_iter_ms.size() < (c->prof_iter + 1) * SUB_K_COUNT)
        c->prof_iter_ms.resize((size_t)(c->prof_iter + 1) * SUB_K_COUNT, 0.f);
      c->prof_iter_ms[(size_t)c->prof_iter * SUB_K_COUNT + k] += ms;
    }
  }
};

// Dirty-chunk tracking of the run (track), or every chunk.
static Dirty dirty_of(sub_ctx* c, bool track) {
  Dirty d;
  d.base = track ? c->dirty : nullptr;
  d.lists = track ? c->lists : nullptr;
  d.counts = track ? c->list_counts : nullptr;
  d.nch = c->plan.nch;
  d.rs = c->rs;
  return d;
}

static cudaError_t enqueue_pre(sub_ctx* c, cudaStream_t st) {
  const int64_t n = c->grid.nb;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->acc, 0, (size_t)n * 32, st))) return e;
  if ((e = cudaMemsetAsync(c->rep.w, 0, (size_t)kAccReplicas * c->rep.nbins * 16, st))) return e;
  if ((e = cudaMemsetAsync(c->rs, 0, sizeof(RunState), st))) return e;
  // the first iteration reads set 0: every chunk is new
  if ((e = cudaMemsetAsync(c->dirty, 1, (size_t)c->plan.nch, st))) return e;
  if ((e = cudaMemsetAsync(c->dirty + c->plan.nch, 0, (size_t)c->plan.nch, st))) return e;
  launch_build_lists(dirty_of(c, true), c->lists, c->list_counts, c->rs, st);
  if ((e = cudaMemsetAsync(c->new_hist, 0, (size_t)c->p.max_iter * 4, st))) return e;
  // sized by the capacity, not the catalog: the captured graph serves every catalog that fits
  if ((e = cudaMemsetAsync(c->resolved, 0, (size_t)c->cap_N, st))) return e;
  {
    KTimer t(c, st, SUB_K_PREPASS);
    launch_prepass(c->dcat, c->cap_N, c->grid, tables_of(c), thr_kappa_of(c), thr_live_of(c),
                   c->acc, c->rep, c->cd, c->rs, c->nsm_run, c->test_flags, st);
  }
  return cudaGetLastError();
}

// One estimate of S_gal from `in` into c->Sg (and inv_f when with_inv).  With track, only
// the chunks whose inputs changed since the previous iteration are recomputed.
// Chunks around a changed chunk whose S_gal changes: the median and the mean read one chunk
// on each side, median-then-mean two.
static int sg_radius_of(const sub_ctx* c) { return c->p.estimator == SUB_MEDIAN_MEAN ? 2 : 1; }

static void enqueue_estimate(sub_ctx* c, cudaStream_t st, SpecIn in, int rtol_on, bool with_inv,
                             bool track) {
  const int64_t n = c->grid.nb;
  const SmoothPlan& pl = c->plan;
  Dirty d = dirty_of(c, track);
  SgOut o;
  o.out = c->Sg;
  o.inv_f = with_inv ? c->inv_f : nullptr;
  o.S = c->S;
  o.invSf = c->invSf;
  o.rtol_on = rtol_on;
  o.rs = c->rs;
  switch (c->p.estimator) {
    case SUB_MEAN: {
      { KTimer t(c, st, SUB_K_PREFIX); launch_chunk_prefix(in, n, pl, c->pre_lo, c->pre_hi, c->sig, c->uflow, c->P, d, 0, st); }
      { KTimer t(c, st, SUB_K_MEAN); launch_window_mean(c->P, n, pl, c->pre_lo, c->pre_hi, c->sig, c->uflow, o, d, 1, st); }
      break;
    }
    case SUB_MEDIAN: {
      { KTimer t(c, st, SUB_K_SORT); launch_chunk_sort(in, n, pl, c->skey, c->srank, d, st); }
      { KTimer t(c, st, SUB_K_MEDIAN); launch_running_median(c->skey, c->srank, n, pl, o, d, st); }
      break;
    }
    default: {
      SgOut om = o;
      om.out = c->M;
      om.inv_f = nullptr;
      om.rtol_on = 0;
      SpecIn mi;
      mi.acc = nullptr;
      mi.S = nullptr;
      mi.x = c->M;
      { KTimer t(c, st, SUB_K_SORT); launch_chunk_sort(in, n, pl, c->skey, c->srank, d, st); }
      { KTimer t(c, st, SUB_K_MEDIAN); launch_running_median(c->skey, c->srank, n, pl, om, d, st); }
      { KTimer t(c, st, SUB_K_PREFIX); launch_chunk_prefix(mi, n, pl, c->pre_lo, c->pre_hi, c->sig, c->uflow, nullptr, d, 1, st); }
      { KTimer t(c, st, SUB_K_MEAN); launch_window_mean(c->M, n, pl, c->pre_lo, c->pre_hi, c->sig, c->uflow, o, d, 2, st); }
      break;
    }
  }
}

static cudaError_t enqueue_body(sub_ctx* c, cudaStream_t st, unsigned long long handle, int use_cond) {
  const int rtol_on = c->p.conv_rtol > 0.0 ? 1 : 0;
  RunState* rs = c->rs;
  SpecIn in;
  in.acc = c->acc;
  in.S = c->S;
  in.x = nullptr;
  enqueue_estimate(c, st, in, rtol_on, true, true);
  double th2 = c->p.rho_th * c->p.rho_th;
  {
    KTimer t(c, st, SUB_K_SNR);
    launch_snr_resolve(c->cd, c->cap_N > 0 ? c->cap_N : 1, c->grid, tables_of(c), c->Sg, c->inv_f, th2,
                       c->p.conv_rtol, snr_mode(c), c->resolved, c->acc, rs, dirty_of(c, true),
                       c->plan.Kc, sg_radius_of(c), c->nsm_run, st);
  }
  { KTimer t(c, st, SUB_K_CONTROL); launch_control(rs, c->p.max_iter, c->p.conv_rtol, c->new_hist, handle, use_cond, c->dirty, c->plan.nch, c->lists, c->list_counts, st); }
  return cudaGetLastError();
}

cudaError_t gbsub::ctx_add_run_nodes(sub_ctx* c, cudaGraph_t g, cudaGraphNode_t* last) {
  cudaGraph_t pre = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (!e) {
    // external records become event nodes of the graph (timing the run inside the graph)
    cudaError_t e2 = cudaEventRecordWithFlags(c->ev_start, c->cap_stream, cudaEventRecordExternal);
    if (!e2) e2 = enqueue_pre(c, c->cap_stream);
    if (!e2) e2 = cudaEventRecordWithFlags(c->ev_pre, c->cap_stream, cudaEventRecordExternal);
    e = cudaStreamEndCapture(c->cap_stream, &pre);
    if (!e) e = e2;
  }
  cudaGraphNode_t pre_node = nullptr, cond_node = nullptr;
  if (!e) e = cudaGraphAddChildGraphNode(&pre_node, g, nullptr, 0, pre);
  if (pre) cudaGraphDestroy(pre);
  cudaGraphConditionalHandle h = 0;
  if (!e) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (!e) e = cudaGraphAddNode(&cond_node, g, &pre_node, nullptr, 1, &cp);
  if (!e) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (!e) {
      cudaError_t e2 = enqueue_body(c, c->cap_stream, (unsigned long long)h, 1);
      cudaGraph_t got = nullptr;
      e = cudaStreamEndCapture(c->cap_stream, &got);
      if (!e) e = e2;
    }
  }
  cudaGraphNode_t end_node = nullptr;
  if (!e) e = cudaGraphAddEventRecordNode(&end_node, g, &cond_node, 1, c->ev_end);
  if (!e) *last = end_node;
  return e;
}

static int build_graph(sub_ctx* c) {
  drop_graph(c);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e) { set_err(c, "cudaGraphCreate: %s", cudaGetErrorString(e)); return SUB_ECUDA; }
  cudaGraphNode_t last = nullptr;
  e = ctx_add_run_nodes(c, g, &last);
  if (!e) e = cudaGraphInstantiate(&c->exec, g, 0);
  if (e) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    c->exec = nullptr;
    set_err(c, "graph build failed: %s", cudaGetErrorString(e));
    return SUB_ECUDA;
  }
  c->graph = g;
  c->graph_cap = c->cap_N;
  return SUB_OK;
}

static int run_host_loop(sub_ctx* c) {
  c->prof_iter = -1;
  c->prof_iter_ms.clear();
  CU(cudaEventRecord(c->ev_start, c->stream), c);
  CU(enqueue_pre(c, c->stream), c);
  CU(cudaEventRecord(c->ev_pre, c->stream), c);
  for (int it = 0; it <= c->p.max_iter + 1; ++it) {
    c->prof_iter = it;
    CU(enqueue_body(c, c->stream, 0ull, 0), c);
    CU(cudaMemcpyAsync(c->h_rs, c->rs, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream), c);
    CU(cudaStreamSynchronize(c->stream), c);
    if (c->h_rs->stopped) break;
  }
  CU(cudaEventRecord(c->ev_end, c->stream), c);
  return SUB_OK;
}

static int fill_stats(sub_ctx* c, sub_stats* st) {
  CU(cudaMemcpyAsync(c->h_rs, c->rs, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  const RunState& r = *c->h_rs;
  int status = SUB_OK;
  if (r.err & ERR_TIMEOUT) {
    status = SUB_ETIMEOUT;
    set_err(c, "a staged copy of the catalog did not arrive in time; the run was abandoned");
  } else if (r.err & ERR_INPUT) {
    status = SUB_EINVAL;
    set_err(c, "the catalog holds non-finite values of A, f or fdot; those sources were skipped");
  } else if (r.err & ERR_RANGE) {
    status = SUB_ERANGE;
    set_err(c, "a deposited power exceeded the fixed-point range (P/S_instr >= 2^63 in one bin)");
  } else if (!r.converged) {
    status = SUB_ENOTCONVERGED;
    set_err(c, "max_iter (%d) reached before convergence", c->p.max_iter);
  }
  if (st) {
    st->iterations = r.iter;
    st->converged = r.converged;
    st->n_sources = c->N;
    st->n_candidates = (int64_t)r.ncand;
    st->n_resolved = (int64_t)r.nres;
    st->n_bins = c->grid.nb;
    st->k_lo = c->grid.k_lo;
    st->status = status;
    st->reserved = 0;
    st->n_live = (int64_t)r.nlive;
    st->n_exact = (int64_t)r.nexact;
    st->n_near = (int64_t)r.nnear;
    st->n_uncertain = (int64_t)r.nuncertain;
  }
  return status;
}


void gbsub::ctx_set_err(sub_ctx* c, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_err = buf;
}

int gbsub::ctx_fill_stats(sub_ctx* c, sub_stats* st) { return fill_stats(c, st); }

int gbsub::ctx_prepare(sub_ctx* c, int64_t cap) {
  int rc = reserve_sources(c, cap);
  if (rc) return rc;
  if (c->use_graph && c->graph_cap != c->cap_N) {
    if (build_graph(c) != SUB_OK) c->use_graph = false;
  }
  return SUB_OK;
}

void gbsub::ctx_set_test_flags(sub_ctx* c, int flags) {
  if (flags == c->test_flags) return;
  drop_graph(c);
  c->test_flags = flags;
}

// Persistent grids from the plan's launch settings, at 1/grid_div of the GPU.
static void replan(sub_ctx* c) {
  const int div = c->grid_div;
  plan_grids(c->plan);
  int* res[] = {&c->plan.res_sort, &c->plan.res_median, &c->plan.res_prefix, &c->plan.res_mean};
  for (int* r : res) *r = (*r / div) > 0 ? *r / div : 1;
  c->nsm_run = c->nsm / div > 0 ? c->nsm / div : 1;
}

void gbsub::ctx_set_grid_div(sub_ctx* c, int div) {
  if (div < 1) div = 1;
  if (div == c->grid_div) return;
  drop_graph(c);
  c->grid_div = div;
  replan(c);
}

int gbsub::ctx_set_tuning(sub_ctx* c, int knob, int value) {
  if (knob == SUB_TUNE_GRID_DIV) {
    if (value < 1 || value > 64) return SUB_EINVAL;
    ctx_set_grid_div(c, value);
    return SUB_OK;
  }
  if (knob == SUB_TUNE_SORT_E) {
    const bool ok = value == 0 || ((value == 2 || value == 4 || value == 8) &&
                                   c->plan.kpad / value >= 32 && c->plan.kpad / value <= 1024);
    if (!ok) return SUB_EINVAL;
    if (value == c->plan.sort_e) return SUB_OK;
    drop_graph(c);
    c->plan.sort_e = value;
  } else if (knob == SUB_TUNE_MEDIAN_THREADS) {
    if (!(value == 0 || (value % 32 == 0 && value >= 32 && value <= 512))) return SUB_EINVAL;
    if (value == c->plan.median_th) return SUB_OK;
    drop_graph(c);
    c->plan.median_th = value;
  } else {
    return SUB_EINVAL;
  }
  replan(c);
  return SUB_OK;
}

extern "C" int sub_run(sub_ctx* c, sub_stats* st) {
  if (!c) return SUB_EINVAL;
  if (c->N < 0) { set_err(c, "no catalog loaded"); return SUB_ESTATE; }
  if (c->use_graph && c->graph_cap != c->cap_N) {
    if (build_graph(c) != SUB_OK) c->use_graph = false;  // conditional nodes unavailable
  }
  if (c->use_graph) {
    CU(cudaGraphLaunch(c->exec, c->stream), c);
  } else {
    int rc = run_host_loop(c);
    if (rc) return rc;
  }
  c->ran = true;
  if (!st) return SUB_OK;
  return fill_stats(c, st);
}

extern "C" int sub_get_stats(sub_ctx* c, sub_stats* st) {
  if (!c || !st) return SUB_EINVAL;
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  return fill_stats(c, st);
}

extern "C" int sub_get_spectrum(sub_ctx* c, double* S_gal, int64_t cap, int64_t* n_bins,
                                int64_t* k_lo, int where) {
  if (!c) return SUB_EINVAL;
  if (n_bins) *n_bins = c->grid.nb;
  if (k_lo) *k_lo = c->grid.k_lo;
  if (!S_gal) return SUB_OK;
  if (cap < c->grid.nb) { set_err(c, "cap %lld < n_bins %lld", (long long)cap, (long long)c->grid.nb); return SUB_EINVAL; }
  if (where != SUB_HOST && where != SUB_DEVICE) { set_err(c, "bad where"); return SUB_EINVAL; }
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  CU(cudaMemcpyAsync(S_gal, c->Sg, (size_t)c->grid.nb * 8,
                     where == SUB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  return SUB_OK;
}

extern "C" int sub_get_resolved_mask(sub_ctx* c, uint8_t* mask, int64_t n, int where) {
  if (!c) return SUB_EINVAL;
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  if (n != c->N || (n > 0 && !mask)) { set_err(c, "mask length %lld != catalog %lld", (long long)n, (long long)c->N); return SUB_EINVAL; }
  if (where != SUB_HOST && where != SUB_DEVICE) { set_err(c, "bad where"); return SUB_EINVAL; }
  if (n == 0) return SUB_OK;
  CU(cudaMemcpyAsync(mask, c->resolved, (size_t)n,
                     where == SUB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  return SUB_OK;
}

extern "C" int sub_get_history(sub_ctx* c, int32_t* hist, int32_t cap) {
  if (!c || (cap > 0 && !hist)) return SUB_EINVAL;
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  CU(cudaMemcpyAsync(c->h_rs, c->rs, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  int m = c->h_rs->iter < cap ? c->h_rs->iter : cap;
  if (m > 0) {
    CU(cudaMemcpy(hist, c->new_hist, (size_t)m * 4, cudaMemcpyDeviceToHost), c);
  }
  return m;
}

extern "C" int sub_estimate(sub_ctx* c, const double* P, double* out, int64_t n, int where) {
  if (!c) return SUB_EINVAL;
  if (n != c->grid.nb || !P || !out) { set_err(c, "sub_estimate needs n == n_bins (%lld) and two buffers", (long long)c->grid.nb); return SUB_EINVAL; }
  if (where != SUB_HOST && where != SUB_DEVICE) { set_err(c, "bad where"); return SUB_EINVAL; }
  cudaStream_t st = c->stream;
  cudaMemcpyKind k_in = where == SUB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyKind k_out = where == SUB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  // the input goes through the Sg buffer (as an input it is read before Sg is written)
  double* in_buf = c->estimate_in;
  CU(cudaMemcpyAsync(in_buf, P, (size_t)n * 8, k_in, st), c);
  CU(cudaMemsetAsync(c->rs, 0, sizeof(RunState), st), c);
  SpecIn in;
  in.acc = nullptr;
  in.S = nullptr;
  in.x = in_buf;
  enqueue_estimate(c, st, in, 0, false, false);
  CU(cudaGetLastError(), c);
  CU(cudaMemcpyAsync(out, c->Sg, (size_t)n * 8, k_out, st), c);
  CU(cudaStreamSynchronize(st), c);
  c->ran = false;  // the run's S_gal was overwritten
  return SUB_OK;
}

// First grid index of every coarse bin (Sec. "Coarse-graining of the data"): edges
// e_k = 10^(log10 f_min + k (log10 f_max - log10 f_min) / nb); a grid frequency
// f_i = (k_lo + i) / T belongs to the highest bin whose lower edge is <= f_i (bin 0 takes
// everything below e_1).  Each boundary is settled by the same FP64 comparison f_i >= e_k.
static void coarse_bounds(double T, double f_min, double f_max, int64_t k_lo, int64_t n, int nb,
                          std::vector<long long>& idx) {
  const double l0 = std::log10(f_min), l1 = std::log10(f_max);
  idx.assign((size_t)nb + 1, 0);
  idx[nb] = n;
  for (int k = 1; k < nb; ++k) {
    const double e = std::pow(10.0, l0 + (double)k * (l1 - l0) / (double)nb);
    long long i = (long long)std::ceil(e * T) - k_lo;
    if (i < 0) i = 0;
    if (i > n) i = n;
    while (i > 0 && (double)(k_lo + i - 1) / T >= e) --i;
    while (i < n && (double)(k_lo + i) / T < e) ++i;
    idx[k] = i < idx[k - 1] ? idx[k - 1] : i;
  }
}

extern "C" int sub_coarse_grain(sub_ctx* c, const double* x, int32_t add_instr, int32_t nbins,
                                double* S_out, double* f_out, int64_t* count_out, int where) {
  if (!c) return SUB_EINVAL;
  if (nbins < 1 || nbins > (1 << 20)) { set_err(c, "nbins must be in 1 .. 2^20"); return SUB_EINVAL; }
  if (where != SUB_HOST && where != SUB_DEVICE) { set_err(c, "bad where"); return SUB_EINVAL; }
  if (!x && !c->ran) { set_err(c, "no run yet (and no series given)"); return SUB_ESTATE; }
  const int64_t n = c->grid.nb;
  cudaStream_t st = c->stream;
  if (nbins > c->cg_cap) {
    dfree(c, c->cg);
    c->cg = nullptr;
    c->cg_cap = 0;
    int rc = dalloc(c, (void**)&c->cg, (size_t)nbins * 32 + 8);
    if (rc) return rc;
    c->cg_cap = nbins;
  }
  double* dS = c->cg;
  double* df = dS + c->cg_cap;
  long long* dc = (long long*)(df + c->cg_cap);
  long long* de = dc + c->cg_cap;
  std::vector<long long> idx;
  coarse_bounds(c->p.T_obs, c->p.f_min, c->p.f_max, c->grid.k_lo, n, nbins, idx);
  CU(cudaMemcpyAsync(de, idx.data(), idx.size() * 8, cudaMemcpyHostToDevice, st), c);
  const double* in = c->Sg;
  if (x && where == SUB_DEVICE) {
    in = x;
  } else if (x) {
    CU(cudaMemcpyAsync(c->estimate_in, x, (size_t)n * 8, cudaMemcpyHostToDevice, st), c);
    in = c->estimate_in;
  }
  launch_coarse_grain(in, add_instr ? c->S : nullptr, de, nbins, c->grid.k_lo, c->p.T_obs, dS, df,
                      dc, st);
  CU(cudaGetLastError(), c);
  const cudaMemcpyKind k = where == SUB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (S_out) CU(cudaMemcpyAsync(S_out, dS, (size_t)nbins * 8, k, st), c);
  if (f_out) CU(cudaMemcpyAsync(f_out, df, (size_t)nbins * 8, k, st), c);
  if (count_out) CU(cudaMemcpyAsync(count_out, dc, (size_t)nbins * 8, k, st), c);
  CU(cudaStreamSynchronize(st), c);
  return SUB_OK;
}

extern "C" int sub_get_power(sub_ctx* c, double* P, int64_t n, int where) {
  if (!c) return SUB_EINVAL;
  if (n != c->grid.nb || !P) { set_err(c, "n must equal n_bins"); return SUB_EINVAL; }
  if (where != SUB_HOST && where != SUB_DEVICE) { set_err(c, "bad where"); return SUB_EINVAL; }
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  launch_power_out(c->acc, c->S, n, c->estimate_in, c->stream);
  CU(cudaGetLastError(), c);
  CU(cudaMemcpyAsync(P, c->estimate_in, (size_t)n * 8,
                     where == SUB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  return SUB_OK;
}

extern "C" int sub_get_tables(sub_ctx* c, double* S, double* R, int64_t n, int where) {
  if (!c) return SUB_EINVAL;
  if (n != c->grid.nb) { set_err(c, "n must equal n_bins"); return SUB_EINVAL; }
  if (where != SUB_HOST && where != SUB_DEVICE) { set_err(c, "bad where"); return SUB_EINVAL; }
  cudaMemcpyKind k = where == SUB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (S) CU(cudaMemcpyAsync(S, c->S, (size_t)n * 8, k, c->stream), c);
  if (R) CU(cudaMemcpyAsync(R, c->R, (size_t)n * 8, k, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  return SUB_OK;
}

extern "C" int sub_get_timing(sub_ctx* c, float* prepass_ms, float* loop_ms, float* total_ms) {
  if (!c) return SUB_EINVAL;
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  CU(cudaEventSynchronize(c->ev_end), c);
  float a = 0.f, b = 0.f;
  CU(cudaEventElapsedTime(&a, c->ev_start, c->ev_pre), c);
  CU(cudaEventElapsedTime(&b, c->ev_pre, c->ev_end), c);
  if (prepass_ms) *prepass_ms = a;
  if (loop_ms) *loop_ms = b;
  if (total_ms) *total_ms = a + b;
  return SUB_OK;
}

extern "C" int sub_get_work(sub_ctx* c, int64_t* work, int32_t n) {
  if (!c || (n > 0 && !work)) return SUB_EINVAL;
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  CU(cudaMemcpyAsync(c->h_rs, c->rs, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  for (int i = 0; i < n && i < 4; ++i) work[i] = (int64_t)c->h_rs->work[i];
  return SUB_OK;
}

extern "C" int sub_profile(sub_ctx* c, float ms[SUB_K_COUNT], int32_t launches[SUB_K_COUNT],
                           sub_stats* st) {
  if (!c) return SUB_EINVAL;
  if (c->N < 0) { set_err(c, "no catalog loaded"); return SUB_ESTATE; }
  for (int k = 0; k < SUB_K_COUNT; ++k) { c->prof_ms[k] = 0.f; c->prof_n[k] = 0; }
  CU(cudaStreamSynchronize(c->stream), c);
  c->profiling = true;
  int rc = run_host_loop(c);
  c->profiling = false;
  if (rc) return rc;
  c->ran = true;
  for (int k = 0; k < SUB_K_COUNT; ++k) {
    if (ms) ms[k] = c->prof_ms[k];
    if (launches) launches[k] = c->prof_n[k];
  }
  return fill_stats(c, st);
}

extern "C" int sub_snr_check(sub_ctx* c, int64_t* src, float* rho2_screen, double* rho2_exact,
                             int32_t* nbins, int64_t cap, int64_t* n_out) {
  if (!c) return SUB_EINVAL;
  if (!c->ran) { set_err(c, "no run yet"); return SUB_ESTATE; }
  CU(cudaMemcpyAsync(c->h_rs, c->rs, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream), c);
  CU(cudaStreamSynchronize(c->stream), c);
  const int64_t m = (int64_t)c->h_rs->nlive;
  if (n_out) *n_out = m;
  if (cap < m) { set_err(c, "cap %lld < kept candidates %lld", (long long)cap, (long long)m); return SUB_EINVAL; }
  if (m == 0) return SUB_OK;
  if (!src || !rho2_screen || !rho2_exact || !nbins) { set_err(c, "null output"); return SUB_EINVAL; }
  void* buf = nullptr;
  int rc = dalloc(c, &buf, (size_t)m * 24);
  if (rc) return rc;
  long long* d_src = (long long*)buf;
  double* d_ex = (double*)(d_src + m);
  float* d_sc = (float*)(d_ex + m);
  int* d_k = (int*)(d_sc + m);
  launch_snr_check(c->cd, m, c->grid, tables_of(c), c->Sg, c->inv_f, c->rs, d_src, d_sc, d_ex, d_k,
                   c->stream);
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(src, d_src, (size_t)m * 8, cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaMemcpyAsync(rho2_exact, d_ex, (size_t)m * 8, cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaMemcpyAsync(rho2_screen, d_sc, (size_t)m * 4, cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaMemcpyAsync(nbins, d_k, (size_t)m * 4, cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  dfree(c, buf);
  if (e) { set_err(c, "sub_snr_check: %s", cudaGetErrorString(e)); return SUB_ECUDA; }
  return SUB_OK;
}

extern "C" int sub_get_profile_iterations(sub_ctx* c, float* ms, int32_t cap) {
  if (!c || (cap > 0 && !ms)) return SUB_EINVAL;
  const int m = (int)(c->prof_iter_ms.size() / SUB_K_COUNT);
  const int w = m < cap ? m : cap;
  for (int i = 0; i < w * SUB_K_COUNT; ++i) ms[i] = c->prof_iter_ms[(size_t)i];
  return m;
}

extern "C" int64_t sub_device_bytes(const sub_ctx* c) { return c ? c->bytes : 0; }

extern "C" void sub_destroy(sub_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  for (auto& q : c->allocs) cudaFree(q.first);
  c->allocs.clear();
  if (c->h_rs) cudaFreeHost(c->h_rs);
  cudaEvent_t evs[] = {c->ev_start, c->ev_pre, c->ev_end, c->ev_k[0], c->ev_k[1]};
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" const char* sub_last_error(const sub_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}
