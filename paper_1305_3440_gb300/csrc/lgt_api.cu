// lgt_api.cu -- the C ABI (include/lgt.h): contexts, the precision ladder and
// the driver loop of Sec. 4 (sweep both parities until theta < tol).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lgt.h"
#include "lgt_api_internal.h"
#include "lgt_internal.h"

using namespace lgt;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void lgt_set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

extern "C" const char *lgt_last_error(void) { return g_last_error.c_str(); }

// Host-side fault injection for tests: LGT_FAULT is a comma-separated list of
// failure names ("alloc": device allocations of contexts and servers fail).
bool lgt_fault_injected(const char *what) {
  const char *f = getenv("LGT_FAULT");
  if (!f || !*f) return false;
  const size_t n = strlen(what);
  for (const char *p = f; (p = strstr(p, what)) != nullptr; p += n) {
    const bool start = p == f || p[-1] == ',';
    const bool end = p[n] == '\0' || p[n] == ',';
    if (start && end) return true;
  }
  return false;
}

extern "C" const char *lgt_version(void) { return "liblgt 0.1 (sm_103a)"; }

#define LGT_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      lgt_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? LGT_ENOMEM : LGT_ECUDA;                      \
    }                                                                                       \
  } while (0)

// ------------------------------------------------------------------ params
extern "C" lgt_status lgt_params_default(lgt_params *p) {
  if (!p) {
    lgt_set_error("lgt_params_default: NULL");
    return LGT_EINVAL;
  }
  memset(p, 0, sizeof *p);
  p->gauge = LGT_LANDAU;
  p->algo = LGT_OR;
  p->bulk = LGT_FP64;
  p->transform_temporal = 1;
  p->omega = 1.7;
  p->p = 0.0;
  p->seed = 0;
  p->sweep_offset = 0;
  p->theta_tol = 1e-14;
  p->theta_switch = 1e-13;
  p->max_sweeps = 10000;
  p->check_every = 10;
  p->reunit_every = 50;
  p->block_size = 0;
  p->polish = LGT_POLISH_ANCHOR;
  p->launch_config = 0;
  p->sa_sweeps = 0;
  p->polish_algo = LGT_POLISH_SAME;
  p->sa_beta0 = 1.0;
  p->sa_beta1 = 100.0;
  p->omega_polish = 1.3;
  p->omega_late = 0.0;
  p->theta_omega = 0.0;
  return LGT_OK;
}

lgt_status lgt_validate_params(const lgt_params *p) {
  if (!p) {
    lgt_set_error("params is NULL");
    return LGT_EINVAL;
  }
  for (int d = 0; d < 4; d++)
    if (p->dims[d] < 2 || (p->dims[d] & 1)) {
      lgt_set_error("dims[%d] = %d: every extent must be even and >= 2", d, p->dims[d]);
      return LGT_EINVAL;
    }
  const double vol = (double)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
  if (vol / 2 > 2.0e9) {
    lgt_set_error("lattice too large (V/2 must fit in 32 bits)");
    return LGT_EINVAL;
  }
  if (p->gauge != LGT_LANDAU && p->gauge != LGT_COULOMB && p->gauge != LGT_MAG) {
    lgt_set_error("gauge %d unknown", p->gauge);
    return LGT_EINVAL;
  }
  if (p->gauge == LGT_MAG && p->sa_sweeps > 0) {
    lgt_set_error("simulated annealing is not available for the maximally Abelian gauge");
    return LGT_EINVAL;
  }
  if (p->algo != LGT_OR && p->algo != LGT_SR) {
    lgt_set_error("algo %d unknown", p->algo);
    return LGT_EINVAL;
  }
  if (p->bulk != LGT_FP64 && p->bulk != LGT_FP32_18 && p->bulk != LGT_FP32_12) {
    lgt_set_error("bulk precision %d unknown", p->bulk);
    return LGT_EINVAL;
  }
  if (p->algo == LGT_OR && !(p->omega >= 1.0 && p->omega < 2.0)) {
    lgt_set_error("omega = %g outside [1, 2)", p->omega);
    return LGT_EINVAL;
  }
  if ((p->algo == LGT_OR || p->polish_algo == LGT_POLISH_OR) && p->omega_polish != 0.0 &&
      !(p->omega_polish >= 1.0 && p->omega_polish < 2.0)) {
    lgt_set_error("omega_polish = %g outside [1, 2) (0: same as omega)", p->omega_polish);
    return LGT_EINVAL;
  }
  if (p->omega_late != 0.0 && !(p->omega_late >= 1.0 && p->omega_late < 2.0)) {
    lgt_set_error("omega_late = %g outside [1, 2) (0: no omega schedule)", p->omega_late);
    return LGT_EINVAL;
  }
  if (!(p->theta_omega >= 0.0)) {
    lgt_set_error("theta_omega must be >= 0");
    return LGT_EINVAL;
  }
  if (p->algo == LGT_SR && !(p->p >= 0.0 && p->p <= 1.0)) {
    lgt_set_error("p = %g outside [0, 1]", p->p);
    return LGT_EINVAL;
  }
  if (!(p->theta_tol > 0.0) || !(p->theta_switch >= 0.0)) {
    lgt_set_error("theta_tol must be > 0 and theta_switch >= 0");
    return LGT_EINVAL;
  }
  if (p->max_sweeps < 0 || p->check_every < 1 || p->reunit_every < 0) {
    lgt_set_error("max_sweeps >= 0, check_every >= 1, reunit_every >= 0 required");
    return LGT_EINVAL;
  }
  if (p->polish != LGT_POLISH_PAIR && p->polish != LGT_POLISH_FP64 && p->polish != LGT_POLISH_ANCHOR) {
    lgt_set_error("polish %d unknown", p->polish);
    return LGT_EINVAL;
  }
  if (p->block_size != 0 && p->block_size != 64 && p->block_size != 128 && p->block_size != 256) {
    lgt_set_error("block_size must be 0, 64, 128 or 256");
    return LGT_EINVAL;
  }
  if (p->sa_sweeps < 0 || (p->sa_sweeps > 0 && !(p->sa_beta0 > 0.0 && p->sa_beta0 <= p->sa_beta1 &&
                                                  p->sa_beta1 < 1e300))) {
    lgt_set_error("sa_sweeps >= 0 and 0 < sa_beta0 <= sa_beta1 (finite) required");
    return LGT_EINVAL;
  }
  if (p->polish_algo != LGT_POLISH_SAME && p->polish_algo != LGT_POLISH_OR) {
    lgt_set_error("polish_algo %d unknown", p->polish_algo);
    return LGT_EINVAL;
  }
  if (p->polish_algo == LGT_POLISH_OR && p->algo == LGT_SR && p->omega_polish == 0.0 &&
      !(p->omega >= 1.0 && p->omega < 2.0)) {
    lgt_set_error("polish_algo = LGT_POLISH_OR needs omega_polish or omega in [1, 2)");
    return LGT_EINVAL;
  }
  if (p->launch_config < 0 || p->launch_config > LGT_NCFG) {
    lgt_set_error("launch_config must be in [0, %d]", LGT_NCFG);
    return LGT_EINVAL;
  }
  return LGT_OK;
}

Geom lgt_make_geom(const int32_t dims[4]) {
  Geom g;
  g.nt = dims[0];
  g.n3 = dims[1];
  g.n2 = dims[2];
  g.n1 = dims[3];
  g.half1 = g.n1 / 2;
  g.vs_half = g.n1 * g.n2 * g.n3 / 2;
  g.vh = g.vs_half * g.nt;
  return g;
}

static unsigned long long sr_threshold(double p) {
  if (!(p > 0.0)) return 0ull;
  if (p >= 1.0) return 1ull << 32;
  return (unsigned long long)floor(p * 4294967296.0);
}

static int fmt_of(int32_t prec) { return prec == LGT_FP32_18 ? FMT_F32_18 : (prec == LGT_FP32_12 ? FMT_F32_12 : FMT_F64); }

size_t lgt_ctx_device_bytes(const lgt_params *p) {
  const Geom g = lgt_make_geom(p->dims);
  lgt_params own = *p;
  if (own.gauge == LGT_MAG) own.polish = LGT_POLISH_FP64;  // as lgt_create
  p = &own;
  size_t b = field_bytes(FMT_F64, g.vh) + workspace_bytes(g, 64) + 4096;
  if (p->bulk != LGT_FP64) b += field_bytes(fmt_of(p->bulk), g.vh) + g_bytes(g.vh);
  if (p->bulk != LGT_FP64 && p->polish == LGT_POLISH_ANCHOR) b += k0_bytes(g.vh) + d_bytes(g.vh) - g_bytes(g.vh);
  return b;
}

// ------------------------------------------------------------------ context
struct lgt_ctx {
  lgt_params prm;
  Geom g;
  cudaStream_t stream;
  int phase;      // 0 bulk (FP32), 1 FP64 storage, 2 FP32-pair storage (in u64), 3 anchored polish
  int bulk_fmt;   // FMT_* of the bulk phase
  void *u64;      // FP64 links (the input while in the bulk phase)
  void *u32;      // bulk working links
  void *G;        // accumulated transformation of the bulk phase; D = G - 1 of the anchored polish
  void *k0;       // anchored polish: K0 (pairs)
  int anchored;   // anchored polish: K0, the FP32-12 copy in u32 and D refer to the field in u64
  int d_dirty;    // anchored polish: D != 0 (sweeps since the field in u64 was last formed)
  int64_t anchor_sweeps;  // anchored polish: sweeps since the last anchor set-up
  int sa_pending;         // the loaded field has not had its annealing sweeps yet
  void *ws_base;  // workspace allocation
  Workspace ws;
  double *host;   // pinned readback buffer
  int cfg_bulk, cfg_polish;  // launch configurations of the bulk / polish sweep kernels
  int active_slices;         // slices updated by masked sweeps (from the last estimate/measurement)
  int last_sites;            // sites per block of the sweeps behind the current fused estimate
  int64_t sweeps_bulk, sweeps_fp64;
  uint64_t sweep_index;  // number of the next sweep (RNG counter)
  SweepCfg cfg;
  double *stage;  // device staging buffer for host links (AoS), lazily allocated
  // timing: event pairs around batches of kernel launches, resolved at sync points
  struct Pending {
    cudaEvent_t a, b;
    int kind;  // 0 bulk sweeps, 1 FP64 sweeps, 2 measurement
  };
  std::vector<Pending> *pending;
  std::vector<cudaEvent_t> *event_pool;
  lgt_stats stats;
  // device loops of lgt_fix: [0] bulk sweeps, [1] sweeps after promotion
  int use_loops;                   // 0: host-driven chunks only (LGT_FIX_GRAPHS=0, or a loop failed to build)
  LoopState *d_loop, *h_loop;      // loop state (device) and its pinned copy
  cudaGraphExec_t loop_exec[2];
  int loop_sweep_launches[2];      // sweep kernel launches in one chunk of each loop
  int *h_err;                      // pinned copy of the workspace's error word
  int omega_switched;              // the omega schedule has moved to omega_late
  // temporal slab (lgt_slab_create): local slices 0 and 1 are the halo (local
  // slice 1 holds U_0 of the global slice before the slab), 2 .. nt-1 the owned
  // slices t0 .. t0 + nt - 3
  int slab;
  int32_t slab_t0, slab_nt_global;
  // fault injection for the streaming launches of lgt_sweep / lgt_half_sweep
  // (lgt_inject_stream_stall; cleared by lgt_load)
  unsigned long long inj_wait_ns;
  unsigned inj_skip;
};

static void resolve_events(lgt_ctx *c);

static void ctx_free(lgt_ctx *c) {
  if (!c) return;
  if (c->pending) {
    for (auto &pe : *c->pending) {
      cudaEventDestroy(pe.a);
      cudaEventDestroy(pe.b);
    }
    delete c->pending;
  }
  if (c->event_pool) {
    for (auto e : *c->event_pool) cudaEventDestroy(e);
    delete c->event_pool;
  }
  for (int k = 0; k < 2; k++)
    if (c->loop_exec[k]) cudaGraphExecDestroy(c->loop_exec[k]);
  if (c->d_loop) cudaFree(c->d_loop);
  if (c->h_loop) cudaFreeHost(c->h_loop);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->stage) cudaFree(c->stage);
  if (c->u64) cudaFree(c->u64);
  if (c->u32) cudaFree(c->u32);
  if (c->G) cudaFree(c->G);
  if (c->k0) cudaFree(c->k0);
  if (c->ws_base) cudaFree(c->ws_base);
  if (c->host) cudaFreeHost(c->host);
  delete c;
}

static cudaEvent_t take_event(lgt_ctx *c) {
  if (!c->event_pool->empty()) {
    cudaEvent_t e = c->event_pool->back();
    c->event_pool->pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// open a timed batch on the context's stream; returns its index or -1
static int batch_begin(lgt_ctx *c, int kind) {
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (!a || !b) return -1;
  if (cudaEventRecord(a, c->stream) != cudaSuccess) return -1;
  c->pending->push_back({a, b, kind});
  return (int)c->pending->size() - 1;
}

static void batch_end(lgt_ctx *c, int idx) {
  if (idx >= 0) cudaEventRecord((*c->pending)[idx].b, c->stream);
}

// after a stream synchronisation: fold finished batches into the counters
static void resolve_events(lgt_ctx *c) {
  for (auto &pe : *c->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
      if (pe.kind < 2) c->stats.sweep_ms[pe.kind] += ms;
      else c->stats.measure_ms += ms;
    }
    c->event_pool->push_back(pe.a);
    c->event_pool->push_back(pe.b);
  }
  c->pending->clear();
}

// A streaming sweep launch that gave up waiting for a neighbouring slice (it
// never should: see the streaming body) leaves bit LGT_ERR_STREAM_WAIT in the
// error word and the field half-updated; every synchronisation reports it
// until the next lgt_load.
static lgt_status sync_stream(lgt_ctx *c) {
  const bool streaming = lgt_cfg_stream(c->cfg_bulk) && c->h_err;
  if (streaming) LGT_CUDA(cudaMemcpyAsync(c->h_err, c->ws.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LGT_CUDA(cudaStreamSynchronize(c->stream));
  resolve_events(c);
  if (streaming && (*c->h_err & LGT_ERR_STREAM_WAIT)) {
    lgt_set_error("a streaming sweep launch timed out waiting for a neighbouring slice; the field is invalid");
    return LGT_ETIMEOUT;
  }
  return LGT_OK;
}

static lgt_status read_back(lgt_ctx *c, const void *dev, size_t bytes) {
  LGT_CUDA(cudaMemcpyAsync(c->host, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  return sync_stream(c);
}


// (re)load a field: ingest into FP64 (and the bulk format), G = 1, reset counters
static lgt_status load_field(lgt_ctx *c, const double *links, int links_on_device) {
  if (!links) {
    lgt_set_error("links is NULL");
    return LGT_EINVAL;
  }
  const Geom &g = c->g;
  const size_t aos_bytes = (size_t)g.vh * 2 * 4 * 18 * sizeof(double);
  const double *src = links;
  if (!links_on_device) {
    if (!c->stage) LGT_CUDA(cudaMalloc(&c->stage, aos_bytes));
    LGT_CUDA(cudaMemcpyAsync(c->stage, links, aos_bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->stage;
  }
  LGT_CUDA(cudaMemsetAsync(c->ws.err, 0, sizeof(int), c->stream));
  c->inj_wait_ns = 0;
  c->inj_skip = 0;
  LGT_CUDA(cudaMemsetAsync(c->ws.active, 1, (size_t)g.nt, c->stream));
  LGT_CUDA(launch_ingest(FMT_F64, g, src, c->u64, c->ws.err, c->stream));
  c->stats.launches++;
  if (c->u32) {
    LGT_CUDA(launch_ingest(c->bulk_fmt, g, src, c->u32, c->ws.err, c->stream));
    LGT_CUDA(launch_g_identity(g, c->G, c->stream));
    c->stats.launches += 2;
  }
  lgt_status st = read_back(c, c->ws.err, sizeof(int));
  if (st != LGT_OK) return st;
  if (*(int *)c->host != 0) {
    lgt_set_error("input links are not all finite SU(3) matrices (|U^dag U - 1| or |det U - 1| >= 1e-10)");
    return LGT_EINVAL;
  }
  c->phase = c->prm.bulk == LGT_FP64 ? 1 : 0;
  c->anchored = c->d_dirty = 0;
  c->sa_pending = c->prm.sa_sweeps > 0;
  c->active_slices = g.nt;
  c->cfg.omega = c->prm.omega;  // omega_late may take over (omega schedule), omega_polish at promotion
  c->cfg.algo = c->prm.algo == LGT_SR ? ALGO_SR : ALGO_OR;  // polish_algo may switch it at promotion
  c->omega_switched = 0;
  c->sweeps_bulk = c->sweeps_fp64 = 0;
  c->sweep_index = c->prm.sweep_offset;
  return LGT_OK;
}

extern "C" lgt_status lgt_create(const lgt_params *params, const double *links, int links_on_device,
                                 void *cuda_stream, lgt_ctx **out) {
  if (!out) {
    lgt_set_error("out is NULL");
    return LGT_EINVAL;
  }
  *out = nullptr;
  lgt_status st = lgt_validate_params(params);
  if (st != LGT_OK) return st;
  if (!links) {
    lgt_set_error("links is NULL");
    return LGT_EINVAL;
  }
  if (lgt_fault_injected("alloc")) {
    lgt_set_error("lgt_create: device allocation failed (injected by LGT_FAULT)");
    return LGT_ENOMEM;
  }
  // the maximally Abelian gauge polishes in FP64 (the pair and anchored
  // polishes are built on K(x), which its quadratic functional lacks)
  lgt_params own = *params;
  if (own.gauge == LGT_MAG) own.polish = LGT_POLISH_FP64;
  params = &own;
  lgt_ctx *c = new lgt_ctx();
  memset((void *)c, 0, sizeof *c);
  c->pending = new std::vector<lgt_ctx::Pending>();
  c->event_pool = new std::vector<cudaEvent_t>();
  c->prm = *params;
  c->g = lgt_make_geom(params->dims);
  c->stream = (cudaStream_t)cuda_stream;
  c->bulk_fmt = fmt_of(params->bulk);
  c->cfg.gauge = params->gauge == LGT_COULOMB ? GAUGE_COULOMB : (params->gauge == LGT_MAG ? GAUGE_MAG : GAUGE_LANDAU);
  c->cfg.algo = params->algo == LGT_SR ? ALGO_SR : ALGO_OR;
  c->cfg.omega = params->omega;
  c->cfg.sr_thr = sr_threshold(params->p);
  c->cfg.seed = params->seed;
  c->cfg.transform_temporal = params->transform_temporal ? 1 : 0;
  const Geom &g = c->g;
#define CTX_CUDA(call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      lgt_set_error("%s failed: %s", #call, cudaGetErrorString(e_));                           \
      ctx_free(c);                                                                             \
      return e_ == cudaErrorMemoryAllocation ? LGT_ENOMEM : LGT_ECUDA;                         \
    }                                                                                          \
  } while (0)
  CTX_CUDA(cudaMalloc(&c->u64, field_bytes(FMT_F64, g.vh)));
  if (params->bulk != LGT_FP64) {
    CTX_CUDA(cudaMalloc(&c->u32, field_bytes(c->bulk_fmt, g.vh)));
    if (params->polish == LGT_POLISH_ANCHOR) {
      CTX_CUDA(cudaMalloc(&c->G, d_bytes(g.vh)));  // G of the bulk phase, then D
      CTX_CUDA(cudaMalloc(&c->k0, k0_bytes(g.vh)));
    } else {
      CTX_CUDA(cudaMalloc(&c->G, g_bytes(g.vh)));
    }
  }
  const size_t wsb = workspace_bytes(g, 64);
  CTX_CUDA(cudaMalloc(&c->ws_base, wsb));
  CTX_CUDA(cudaMemsetAsync(c->ws_base, 0, wsb, c->stream));
  workspace_carve(c->ws_base, g, 64, &c->ws);
  CTX_CUDA(cudaMallocHost(&c->host, 4096 + sizeof(double) * 2 * (size_t)g.nt));
  CTX_CUDA(cudaMalloc(&c->d_loop, sizeof(LoopState)));
  CTX_CUDA(cudaMallocHost(&c->h_loop, sizeof(LoopState)));
  CTX_CUDA(cudaMallocHost(&c->h_err, sizeof(int)));
  *c->h_err = 0;
  {
    const char *lv = getenv("LGT_FIX_GRAPHS");  // "0": lgt_fix drives every chunk from the host
    c->use_loops = !(lv && lv[0] == '0');
  }
  // block sizes: given, or timed on the still-empty buffers
  const int polish_fmt = params->bulk == LGT_FP64 ? (int)FMT_F64
                         : (params->polish == LGT_POLISH_PAIR ? (int)FMT_PAIR
                            : (params->polish == LGT_POLISH_ANCHOR ? (int)FMT_ANCHOR : (int)FMT_F64));
  c->cfg_bulk = c->cfg_polish = lgt_cfg_of_block(params->block_size);
  if (params->launch_config > 0) {
    const int k = params->launch_config - 1;
    c->cfg_bulk = lgt_cfg_supported_gauge(c->u32 ? c->bulk_fmt : (int)FMT_F64, c->cfg.gauge, k) ? k : 0;
    c->cfg_polish = lgt_cfg_supported_gauge(polish_fmt, c->cfg.gauge, k) ? k : 0;
  } else if (!params->block_size) {
    cudaError_t te = cudaSuccess;
    if (c->u32) c->cfg_bulk = lgt_tune_sweep(g, c->bulk_fmt, c->cfg, c->u32, c->G, c->ws, c->stream, &te);
    if (te == cudaSuccess) {
      if (polish_fmt == FMT_ANCHOR)
        c->cfg_polish = lgt_tune_sweep(g, polish_fmt, c->cfg, c->u32, c->G, c->ws, c->stream, &te, c->k0);
      else
        c->cfg_polish = lgt_tune_sweep(g, polish_fmt, c->cfg, c->u64, nullptr, c->ws, c->stream, &te);
    }
    CTX_CUDA(te);
    if (!c->u32) c->cfg_bulk = c->cfg_polish;
  }
  c->last_sites = lgt_cfg_sites(c->cfg_bulk);
#undef CTX_CUDA
  st = load_field(c, links, links_on_device);
  if (st != LGT_OK) {
    ctx_free(c);
    return st;
  }
  *out = c;
  return LGT_OK;
}

// A slab's local field in public layout in the staging buffer: the two halo
// slices unit links, then the caller's owned slices.
static lgt_status slab_stage(lgt_ctx *c, const double *links, int links_on_device) {
  const Geom &g = c->g;
  const size_t slice_doubles = (size_t)g.vs_half * 2 * 4 * 18;
  if (!c->stage) LGT_CUDA(cudaMalloc(&c->stage, slice_doubles * g.nt * sizeof(double)));
  LGT_CUDA(launch_fill_unit_aos(c->stage, (long long)(2 * slice_doubles / 18), c->stream));
  LGT_CUDA(cudaMemcpyAsync(c->stage + 2 * slice_doubles, links, slice_doubles * (g.nt - 2) * sizeof(double),
                           links_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  return LGT_OK;
}

extern "C" lgt_status lgt_load(lgt_ctx *ctx, const double *links, int links_on_device) {
  if (ctx && ctx->slab && links) {
    lgt_status st = slab_stage(ctx, links, links_on_device);
    if (st != LGT_OK) return st;
    return load_field(ctx, ctx->stage, 1);
  }
  if (!ctx) {
    lgt_set_error("lgt_load: NULL context");
    return LGT_EINVAL;
  }
  memset(&ctx->stats, 0, sizeof ctx->stats);
  return load_field(ctx, links, links_on_device);
}

extern "C" lgt_status lgt_get_stats(lgt_ctx *ctx, lgt_stats *out) {
  if (!ctx || !out) {
    lgt_set_error("lgt_get_stats: bad arguments");
    return LGT_EINVAL;
  }
  lgt_status st = sync_stream(ctx);
  if (st != LGT_OK) return st;
  *out = ctx->stats;
  out->launch_config[0] = ctx->cfg_bulk;
  out->launch_config[1] = ctx->cfg_polish;
  return LGT_OK;
}

extern "C" void lgt_destroy(lgt_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  ctx_free(ctx);
}

// ------------------------------------------------------------------ sweeps
// half-sweeps [first_parity .. first_parity + n_half) (parity alternating);
// the sweep counter advances after each odd half
// storage format (and kernel) of the working field in the current phase
// storage format of the working field (the anchored polish measures the
// formed field in u64, FP64)
static int work_fmt(const lgt_ctx *c) {
  return c->phase == 0 ? c->bulk_fmt : (c->phase == 2 ? (int)FMT_PAIR : (int)FMT_F64);
}

static int skip_temporal(const lgt_ctx *c) {
  return (c->prm.gauge == LGT_COULOMB && !c->prm.transform_temporal) ? 1 : 0;
}

// anchored polish: form U <- G U G^+ in u64 from the anchor and D (then D is
// spent: the next sweep re-anchors)
static lgt_status anchor_materialise(lgt_ctx *c) {
  if (c->phase != 3 || !c->d_dirty) return LGT_OK;
  LGT_CUDA(launch_apply_D(c->g, c->G, c->u64, c->u64, nullptr, skip_temporal(c), c->stream));
  c->stats.launches++;
  c->d_dirty = 0;
  c->anchored = 0;
  return LGT_OK;
}

static lgt_status anchor_setup(lgt_ctx *c) {
  if (c->phase != 3 || c->anchored) return LGT_OK;
  LGT_CUDA(launch_anchor_setup(c->g, c->u64, c->u32, c->k0, c->G, c->cfg.gauge, c->stream));
  c->stats.launches++;
  c->anchored = 1;
  c->anchor_sweeps = 0;
  return LGT_OK;
}

// anchored polish: after LGT_REANCHOR_SWEEPS sweeps on one anchor, form the
// field (the next sweep sets up a new anchor with D = 0)
static lgt_status anchor_refresh(lgt_ctx *c) {
  if (c->phase == 3 && c->anchored && c->anchor_sweeps >= LGT_REANCHOR_SWEEPS) return anchor_materialise(c);
  return LGT_OK;
}

static lgt_status run_halves(lgt_ctx *c, int first_parity, int n_half, int use_mask) {
  const bool anch = c->phase == 3;
  const int fmt = anch ? (int)FMT_ANCHOR : work_fmt(c);
  void *links = (c->phase == 0 || anch) ? c->u32 : c->u64;
  void *G = ((c->phase == 0 && !c->slab) || anch) ? c->G : nullptr;  // a slab is never promoted
  const int kind = c->phase == 0 ? 0 : 1;
  if (n_half <= 0) return LGT_OK;
  if (anch) {
    lgt_status st = anchor_setup(c);
    if (st != LGT_OK) return st;
    c->d_dirty = 1;
  }
  const int bt = batch_begin(c, kind);
  const int lc = c->phase == 0 ? c->cfg_bulk : c->cfg_polish;
  const int reunit_every = c->phase == 0 ? c->prm.reunit_every : 0;
  int launches = 0;
  SweepCfg sc = c->cfg;
  sc.stream_wait_ns = c->inj_wait_ns;
  sc.stream_skip = c->inj_skip;
  LGT_CUDA(launch_half_sweeps(fmt, c->g, links, G, c->ws, sc, first_parity, n_half, c->sweep_index, c->sweeps_bulk,
                              reunit_every, use_mask, lc, c->stream, anch ? c->k0 : nullptr, nullptr, &launches));
  c->last_sites = lgt_cfg_sites(lc);
  const int64_t done = (first_parity + n_half) / 2;  // sweeps whose odd half ran
  c->sweep_index += (uint64_t)done;
  if (c->phase == 0) c->sweeps_bulk += done;
  else c->sweeps_fp64 += done;
  batch_end(c, bt);
  if (anch) c->anchor_sweeps += n_half / 2;
  c->stats.sweep_launches[kind] += n_half;
  c->stats.launches += launches;
  const int64_t slices = use_mask ? c->active_slices : c->g.nt;
  c->stats.site_updates[kind] += (int64_t)n_half * (int64_t)c->g.vs_half * slices;
  return LGT_OK;
}

static lgt_status run_sweeps(lgt_ctx *c, int n, int use_mask) { return run_halves(c, 0, 2 * n, use_mask); }

extern "C" lgt_status lgt_half_sweep(lgt_ctx *ctx, int32_t parity) {
  if (ctx && ctx->slab) {
    lgt_set_error("lgt_half_sweep: a temporal slab is swept and measured through the lgt_slab_* calls");
    return LGT_EINVAL;
  }
  if (!ctx || (parity != 0 && parity != 1)) {
    lgt_set_error("lgt_half_sweep: bad arguments");
    return LGT_EINVAL;
  }
  lgt_status st = run_halves(ctx, parity, 1, 0);
  if (st != LGT_OK) return st;
  return sync_stream(ctx);
}

extern "C" lgt_status lgt_sweep(lgt_ctx *ctx, int32_t n) {
  if (ctx && ctx->slab) {
    lgt_set_error("lgt_sweep: a temporal slab is swept and measured through the lgt_slab_* calls");
    return LGT_EINVAL;
  }
  if (!ctx || n < 0) {
    lgt_set_error("lgt_sweep: bad arguments");
    return LGT_EINVAL;
  }
  lgt_status st = run_sweeps(ctx, n, 0);
  if (st != LGT_OK) return st;
  return sync_stream(ctx);
}

// ------------------------------------------------------------ measurement
struct Meas {
  double F, theta, plaq, theta_mean;
  int active;
};

static void fill_meas(const lgt_ctx *c, const double *t, Meas *m) {
  if (c->prm.gauge == LGT_COULOMB) {
    m->F = t[TOT_F_COULOMB];
    m->theta = t[TOT_THETA_COULOMB_MAX];
    m->theta_mean = t[TOT_THETA_COULOMB_MEAN];
  } else {
    m->F = t[TOT_F_LANDAU];
    m->theta = t[TOT_THETA_LANDAU];
    m->theta_mean = m->theta;
  }
  m->plaq = t[TOT_PLAQ];
  m->active = (int)t[TOT_ACTIVE_SLICES];
}

// exact measurement of the working field; coulomb_target >= 0 updates masks
static lgt_status measure(lgt_ctx *c, int with_plaq, double coulomb_target, Meas *m) {
  lgt_status mst = anchor_materialise(c);
  if (mst != LGT_OK) return mst;
  const int fmt = work_fmt(c);
  const void *links = c->phase == 0 ? c->u32 : c->u64;
  const int bt = batch_begin(c, 2);
  LGT_CUDA(launch_measure(fmt, c->g, links, c->ws, with_plaq, coulomb_target, 128, c->stream,
                          c->prm.gauge == LGT_MAG ? 1 : 0));
  batch_end(c, bt);
  c->stats.measure_launches++;
  c->stats.launches++;
  lgt_status st = read_back(c, c->ws.totals, sizeof(double) * TOT_N);
  if (st != LGT_OK) return st;
  fill_meas(c, c->host, m);
  c->active_slices = m->active;
  return LGT_OK;
}

// fused estimate from the last sweep's own K(x) (theta lagged by half a sweep)
static lgt_status estimate(lgt_ctx *c, double coulomb_target, Meas *m) {
  LGT_CUDA(launch_fused_finish(c->g, c->ws, c->cfg.gauge, c->last_sites, coulomb_target, c->stream));
  c->stats.launches++;
  lgt_status st = read_back(c, c->ws.fused_totals, sizeof(double) * TOT_N);
  if (st != LGT_OK) return st;
  fill_meas(c, c->host, m);
  c->active_slices = m->active;
  return LGT_OK;
}

// Omega schedule: the relaxation sweeps before promotion (every sweep of an
// FP64 run) switch to omega_late at the first check with theta < theta_omega.
static bool omega_schedule_open(const lgt_ctx *c) {
  return c->prm.omega_late != 0.0 && !c->omega_switched && (c->phase == 0 || c->prm.bulk == LGT_FP64);
}
static void omega_check(lgt_ctx *c, double theta) {
  if (omega_schedule_open(c) && theta < c->prm.theta_omega) {
    c->cfg.omega = c->prm.omega_late;
    c->omega_switched = 1;
  }
}

extern "C" lgt_status lgt_measure(lgt_ctx *ctx, double *F, double *theta, double *plaq) {
  if (ctx && ctx->slab) {
    lgt_set_error("lgt_measure: a temporal slab is swept and measured through the lgt_slab_* calls");
    return LGT_EINVAL;
  }
  if (!ctx) {
    lgt_set_error("lgt_measure: NULL context");
    return LGT_EINVAL;
  }
  Meas m;
  lgt_status st = measure(ctx, plaq != nullptr, -1.0, &m);
  if (st != LGT_OK) return st;
  if (F) *F = m.F;
  if (theta) *theta = m.theta;
  if (plaq) *plaq = m.plaq;
  return LGT_OK;
}

extern "C" lgt_status lgt_measure_slices(lgt_ctx *ctx, double *F_t, double *theta_t) {
  if (ctx && ctx->slab) {
    lgt_set_error("lgt_measure_slices: a temporal slab is swept and measured through the lgt_slab_* calls");
    return LGT_EINVAL;
  }
  if (!ctx) {
    lgt_set_error("lgt_measure_slices: NULL context");
    return LGT_EINVAL;
  }
  Meas m;
  lgt_status st = measure(ctx, 0, -1.0, &m);
  if (st != LGT_OK) return st;
  const size_t nb = sizeof(double) * (size_t)ctx->g.nt;
  if (F_t) {
    LGT_CUDA(cudaMemcpyAsync(F_t, ctx->ws.slice_F, nb, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (theta_t) {
    LGT_CUDA(cudaMemcpyAsync(theta_t, ctx->ws.slice_theta, nb, cudaMemcpyDeviceToHost, ctx->stream));
  }
  return sync_stream(ctx);
}

// the fused estimate of a slab over its owned slices (per slice as lgt_estimate;
// F, theta: means over the owned slices, Coulomb: max theta_t)
static lgt_status slab_estimate(lgt_ctx *c, double *F, double *theta, double *F_t, double *theta_t) {
  const int nt = c->g.nt, L = nt - 2;
  LGT_CUDA(launch_slice_mask(c->ws.active, nt, 2, nt, c->stream));
  Meas m;
  lgt_status st = estimate(c, -1.0, &m);
  if (st != LGT_OK) return st;
  std::vector<double> sl((size_t)nt * 2);
  LGT_CUDA(cudaMemcpyAsync(sl.data(), c->ws.fused_slice, sizeof(double) * sl.size(), cudaMemcpyDeviceToHost,
                           c->stream));
  st = sync_stream(c);
  if (st != LGT_OK) return st;
  const bool coulomb = c->cfg.gauge == GAUGE_COULOMB;
  const double vs = 2.0 * (double)c->g.vs_half, nd = coulomb ? 3.0 : 4.0;
  double fs = 0.0, ts = 0.0, tmax = 0.0;
  for (int k = 0; k < L; k++) {
    const double ft = sl[2 * (k + 2)] / (3.0 * nd * vs), th = sl[2 * (k + 2) + 1] / (3.0 * vs);
    if (F_t) F_t[k] = ft;
    if (theta_t) theta_t[k] = th;
    fs += ft;
    ts += th;
    tmax = th > tmax ? th : tmax;
  }
  if (F) *F = fs / L;
  if (theta) *theta = coulomb ? tmax : ts / L;
  return LGT_OK;
}

extern "C" lgt_status lgt_estimate(lgt_ctx *ctx, double *F, double *theta, double *F_t, double *theta_t) {
  if (!ctx) {
    lgt_set_error("lgt_estimate: NULL context");
    return LGT_EINVAL;
  }
  if (ctx->slab) return slab_estimate(ctx, F, theta, F_t, theta_t);
  Meas m;
  lgt_status st = estimate(ctx, -1.0, &m);
  if (st != LGT_OK) return st;
  if (F) *F = m.F;
  if (theta) *theta = m.theta;
  if (F_t || theta_t) {
    // per-slice sums (parity-0 Re tr K, both parities' tr Delta^2), normalised per slice
    const int nt = ctx->g.nt;
    std::vector<double> sl((size_t)nt * 2);
    LGT_CUDA(cudaMemcpyAsync(sl.data(), ctx->ws.fused_slice, sizeof(double) * sl.size(), cudaMemcpyDeviceToHost,
                             ctx->stream));
    st = sync_stream(ctx);
    if (st != LGT_OK) return st;
    const double vs = 2.0 * (double)ctx->g.vs_half, nd = ctx->cfg.gauge == GAUGE_COULOMB ? 3.0 : 4.0;
    for (int t = 0; t < nt; t++) {
      if (F_t) F_t[t] = sl[2 * t] / (3.0 * nd * vs);
      if (theta_t) theta_t[t] = sl[2 * t + 1] / (3.0 * vs);
    }
  }
  return LGT_OK;
}

extern "C" lgt_status lgt_inject_stream_stall(lgt_ctx *ctx, uint64_t wait_ns, uint32_t skip_items) {
  if (!ctx) {
    lgt_set_error("lgt_inject_stream_stall: NULL context");
    return LGT_EINVAL;
  }
  if (wait_ns > LGT_STREAM_WAIT_NS) {
    lgt_set_error("lgt_inject_stream_stall: wait_ns above the built-in bound of %llu ns", LGT_STREAM_WAIT_NS);
    return LGT_EINVAL;
  }
  ctx->inj_wait_ns = wait_ns;
  ctx->inj_skip = skip_items;
  return LGT_OK;
}

// ------------------------------------------------------ temporal slabs (Sec. 5)
extern "C" lgt_status lgt_slab_create(const lgt_params *params, int32_t nt_global, int32_t t0, const double *links,
                                      int links_on_device, void *cuda_stream, lgt_ctx **out) {
  if (!out || !params || !links) {
    lgt_set_error("lgt_slab_create: NULL argument");
    return LGT_EINVAL;
  }
  *out = nullptr;
  const int L = params->dims[0];
  if (L < 2 || (L & 1) || nt_global < 2 || (nt_global & 1) || t0 < 0 || (t0 & 1) || t0 + L > nt_global) {
    lgt_set_error("lgt_slab_create: need an even slab of dims[0] = %d >= 2 slices starting at an even t0 = %d "
                  "within the %d slices of the lattice", L, t0, nt_global);
    return LGT_EINVAL;
  }
  if (params->gauge != LGT_LANDAU && params->gauge != LGT_COULOMB) {
    lgt_set_error("lgt_slab_create: Landau or Coulomb gauge only");
    return LGT_EINVAL;
  }
  if (params->sa_sweeps != 0) {
    lgt_set_error("lgt_slab_create: no simulated annealing on slabs");
    return LGT_EINVAL;
  }
  lgt_status st = lgt_validate_params(params);
  if (st != LGT_OK) return st;
  lgt_params local = *params;
  local.dims[0] = L + 2;
  const Geom g = lgt_make_geom(local.dims);
  const size_t slice_doubles = (size_t)g.vs_half * 2 * 4 * 18;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  double *buf = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&buf, slice_doubles * g.nt * sizeof(double), stream);
  if (e == cudaSuccess) e = launch_fill_unit_aos(buf, (long long)(2 * slice_doubles / 18), stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf + 2 * slice_doubles, links, slice_doubles * L * sizeof(double),
                        links_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) {
    if (buf) cudaFreeAsync(buf, stream);
    lgt_set_error("lgt_slab_create: staging the slab failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LGT_ENOMEM : LGT_ECUDA;
  }
  lgt_ctx *c = nullptr;
  st = lgt_create(&local, buf, 1, cuda_stream, &c);
  cudaFreeAsync(buf, stream);
  cudaStreamSynchronize(stream);
  if (st != LGT_OK) return st;
  c->slab = 1;
  c->slab_t0 = t0;
  c->slab_nt_global = nt_global;
  c->cfg.t_offset = t0 - 2;  // the random streams count global sites
  // the streaming configuration orders whole slices itself: a slab uses the pipelined one
  if (lgt_cfg_stream(c->cfg_bulk)) c->cfg_bulk = 7;
  if (lgt_cfg_stream(c->cfg_polish)) c->cfg_polish = 0;
  *out = c;
  return LGT_OK;
}

extern "C" lgt_status lgt_slab_half_sweep(lgt_ctx *ctx, int32_t parity, int32_t first, int32_t count) {
  if (!ctx || !ctx->slab || (parity != 0 && parity != 1)) {
    lgt_set_error("lgt_slab_half_sweep: bad arguments (or not a slab)");
    return LGT_EINVAL;
  }
  lgt_ctx *c = ctx;
  const int L = c->g.nt - 2;
  if (first < 0 || count < 1 || first + count > L) {
    lgt_set_error("lgt_slab_half_sweep: slices [%d, %d) outside the %d owned slices", first, first + count, L);
    return LGT_EINVAL;
  }
  const int fmt = work_fmt(c);
  void *links = c->phase == 0 ? c->u32 : c->u64;
  const int kind = c->phase == 0 ? 0 : 1;
  const int lc = c->phase == 0 ? c->cfg_bulk : c->cfg_polish;
  const int64_t done = kind == 0 ? c->sweeps_bulk : c->sweeps_fp64;
  SweepCfg sc = c->cfg;  // the launch covers the requested slices only
  sc.t_first = 2 + first;
  sc.t_count = count;
  const int bt = batch_begin(c, kind);
  int launches = 0;
  LGT_CUDA(launch_half_sweeps(fmt, c->g, links, nullptr, c->ws, sc, parity, 1, c->sweep_index, done,
                              c->phase == 0 ? c->prm.reunit_every : 0, 0, lc, c->stream, nullptr, nullptr,
                              &launches));
  batch_end(c, bt);
  c->last_sites = lgt_cfg_sites(lc);
  if (parity == 1 && first + count == L) {  // a sweep ends with the odd half of the last owned slice
    c->sweep_index++;
    if (kind == 0) c->sweeps_bulk++;
    else c->sweeps_fp64++;
  }
  c->stats.sweep_launches[kind] += 1;
  c->stats.launches += launches;
  c->stats.site_updates[kind] += (int64_t)c->g.vs_half * count;
  return LGT_OK;
}

extern "C" lgt_status lgt_slab_boundary_bytes(lgt_ctx *ctx, size_t *bytes) {
  if (!ctx || !ctx->slab || !bytes) {
    lgt_set_error("lgt_slab_boundary_bytes: bad arguments (or not a slab)");
    return LGT_EINVAL;
  }
  *bytes = (size_t)ctx->g.vs_half * link_bytes_per_half_site(work_fmt(ctx)) / 4;
  return LGT_OK;
}

extern "C" lgt_status lgt_slab_boundary(lgt_ctx *ctx, int32_t slice, int32_t parity, void *buf, int32_t into_slab) {
  if (!ctx || !ctx->slab || !buf || (parity != 0 && parity != 1)) {
    lgt_set_error("lgt_slab_boundary: bad arguments (or not a slab)");
    return LGT_EINVAL;
  }
  lgt_ctx *c = ctx;
  const int L = c->g.nt - 2;
  if (slice < -1 || slice >= L) {
    lgt_set_error("lgt_slab_boundary: slice %d outside [-1, %d)", slice, L);
    return LGT_EINVAL;
  }
  const int fmt = work_fmt(c);
  const size_t vh = (size_t)c->g.vh, vs = (size_t)c->g.vs_half, t = (size_t)(slice + 2);
  char *base = (char *)(c->phase == 0 ? c->u32 : c->u64);
  char *b = (char *)buf;
  // the streams of (parity, mu = 0): 16-byte chunks of vh sites each
  struct Part {
    size_t offset, elem;  // bytes to the first chunk's stream, bytes per site in a chunk
    int chunks;
  } parts[2];
  int np = 1;
  if (fmt == FMT_F64 || fmt == FMT_PAIR) {
    parts[0] = {(size_t)(parity * 4) * 9 * vh * 16, 16, 9};
  } else if (fmt == FMT_F32_12) {
    parts[0] = {(size_t)(parity * 4) * 3 * vh * 16, 16, 3};
  } else {  // FP32-18: 4 float4 chunks, then the float2 chunk in its own region
    parts[0] = {(size_t)(parity * 4) * 4 * vh * 16, 16, 4};
    parts[1] = {32 * vh * 16 + (size_t)(parity * 4) * vh * 8, 8, 1};
    np = 2;
  }
  size_t off = 0;
  for (int k = 0; k < np; k++) {
    char *stream_base = base + parts[k].offset + t * vs * parts[k].elem;
    const size_t width = vs * parts[k].elem, pitch = vh * parts[k].elem;
    if (into_slab)
      LGT_CUDA(cudaMemcpy2DAsync(stream_base, pitch, b + off, width, width, parts[k].chunks,
                                 cudaMemcpyDeviceToDevice, c->stream));
    else
      LGT_CUDA(cudaMemcpy2DAsync(b + off, width, stream_base, pitch, width, parts[k].chunks,
                                 cudaMemcpyDeviceToDevice, c->stream));
    off += width * parts[k].chunks;
  }
  return LGT_OK;
}

extern "C" lgt_status lgt_measure_slice_sums(lgt_ctx *ctx, double *sums) {
  if (!ctx || !sums) {
    lgt_set_error("lgt_measure_slice_sums: bad arguments");
    return LGT_EINVAL;
  }
  lgt_ctx *c = ctx;
  lgt_status st = anchor_materialise(c);
  if (st != LGT_OK) return st;
  const int bt = batch_begin(c, 2);
  LGT_CUDA(launch_measure(work_fmt(c), c->g, c->phase == 0 ? c->u32 : c->u64, c->ws, 1, -1.0, 128, c->stream,
                          c->prm.gauge == LGT_MAG ? 1 : 0));
  batch_end(c, bt);
  c->stats.measure_launches++;
  c->stats.launches++;
  const int first = c->slab ? 2 : 0;
  const int n = c->g.nt - first;
  LGT_CUDA(cudaMemcpyAsync(sums, c->ws.slice_sum + (size_t)first * MEAS_NV, sizeof(double) * MEAS_NV * n,
                           cudaMemcpyDeviceToHost, c->stream));
  return sync_stream(c);
}

extern "C" lgt_status lgt_slab_sync(lgt_ctx *ctx) {
  if (!ctx) {
    lgt_set_error("lgt_slab_sync: NULL context");
    return LGT_EINVAL;
  }
  return sync_stream(ctx);
}

// --------------------------------------------------------------- promotion
static lgt_status promote(lgt_ctx *c) {
  if (c->phase != 0) return LGT_OK;
  LGT_CUDA(launch_apply_G(c->g, c->G, c->u64, c->u64, nullptr, skip_temporal(c), c->stream));
  c->stats.launches++;
  c->phase = 1;
  if (c->prm.polish_algo == LGT_POLISH_OR) c->cfg.algo = ALGO_OR;  // the sweeps after promotion overrelax
  if (c->prm.omega_polish != 0.0) c->cfg.omega = c->prm.omega_polish;
  if (c->prm.polish == LGT_POLISH_PAIR) {
    LGT_CUDA(launch_convert_pair(c->g, c->u64, 1, c->stream));
    c->stats.launches++;
    c->phase = 2;
  } else if (c->prm.polish == LGT_POLISH_ANCHOR) {
    c->phase = 3;
    c->anchored = c->d_dirty = 0;
    lgt_status st = anchor_setup(c);
    if (st != LGT_OK) return st;
  }
  return sync_stream(c);
}

extern "C" lgt_status lgt_promote(lgt_ctx *ctx) {
  if (ctx && ctx->slab) {
    lgt_set_error("lgt_promote: a temporal slab is swept and measured through the lgt_slab_* calls");
    return LGT_EINVAL;
  }
  if (!ctx) {
    lgt_set_error("lgt_promote: NULL context");
    return LGT_EINVAL;
  }
  return promote(ctx);
}

// ------------------------------------------------------------- device loops
// lgt_fix's chunks (check_every sweeps, the fused estimate, the decision) as
// one CUDA graph: a conditional while node whose body is the chunk's 2k
// half-sweep launches, the estimate's finish and a one-thread decide kernel
// that applies the host driver's rules to the loop state and sets the
// condition.  The sweep kernels read their sweep numbers from the loop state,
// so the body is the same for every chunk.  slot 0: bulk sweeps, 1: after
// promotion.  Built on first use; the context's buffers and parameters do not
// change afterwards.
static lgt_status build_loop(lgt_ctx *c, int slot) {
  const bool anch = c->phase == 3;
  const int fmt = anch ? (int)FMT_ANCHOR : work_fmt(c);
  void *links = (c->phase == 0 || anch) ? c->u32 : c->u64;
  void *G = (c->phase == 0 || anch) ? c->G : nullptr;
  const int lc = c->phase == 0 ? c->cfg_bulk : c->cfg_polish;
  const int k = c->prm.check_every;
  const bool coulomb = c->prm.gauge == LGT_COULOMB;
  const double target = slot == 0 ? c->prm.theta_switch : c->prm.theta_tol;
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp = {};
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  // captured on a private stream (the context's stream may be the legacy
  // default stream, which cannot capture); the graph then runs on the context's
  cudaStream_t cs = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = launch_half_sweeps(fmt, c->g, links, G, c->ws, c->cfg, 0, 2 * k, 0, 0,
                                          c->phase == 0 ? c->prm.reunit_every : 0, coulomb ? 1 : 0, lc, cs,
                                          anch ? c->k0 : nullptr, c->d_loop, &c->loop_sweep_launches[slot]);
      if (el == cudaSuccess)
        el = launch_fused_finish(c->g, c->ws, c->cfg.gauge, lgt_cfg_sites(lc), coulomb ? target : -1.0, cs);
      if (el == cudaSuccess) el = launch_loop_decide(c->d_loop, c->ws.fused_totals, c->cfg.gauge, k, c->g.vs_half, h, cs);
      e = cudaStreamEndCapture(cs, &body);
      if (el != cudaSuccess) e = el;
    }
  }
  if (cs) cudaStreamDestroy(cs);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->loop_exec[slot], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();  // the host-driven chunks take over
    c->loop_exec[slot] = nullptr;
    c->use_loops = 0;
    return LGT_EAGAIN;
  }
  return LGT_OK;
}

// Run whole chunks on the device while the driver's rules allow (at least
// one; the caller checked them and remaining >= check_every).  Updates the
// counters, *best / *stall (bulk), *remaining and the estimate in *m.
static lgt_status run_loop(lgt_ctx *c, int slot, double *best, int *stall, int64_t *remaining, Meas *m) {
  const int k = c->prm.check_every;
  const int kind = c->phase == 0 ? 0 : 1;
  const int lc = c->phase == 0 ? c->cfg_bulk : c->cfg_polish;
  if (c->phase == 3) {  // the anchored sweeps need a current anchor
    lgt_status st = anchor_setup(c);
    if (st != LGT_OK) return st;
    c->d_dirty = 1;
  }
  LoopState &L = *c->h_loop;
  L.sweep = c->sweep_index;
  L.count = kind == 0 ? c->sweeps_bulk : c->sweeps_fp64;
  L.remaining = *remaining;
  L.site_updates = 0;
  L.target = slot == 0 ? c->prm.theta_switch : c->prm.theta_tol;
  L.best = best ? *best : 0.0;
  L.theta = 0.0;
  L.stall = stall ? *stall : 0;
  L.bulk = slot == 0 ? 1 : 0;
  L.active = c->active_slices;
  L.iters = 0;
  L.max_iters = (int)(*remaining / k);
  L.omega = c->cfg.omega;
  L.omega_late = c->prm.omega_late;
  L.theta_omega = c->prm.theta_omega;
  L.omega_switch = omega_schedule_open(c) ? 1 : 0;
  if (c->phase == 3) {  // end the launch where the anchor is due for renewal
    const int64_t left = LGT_REANCHOR_SWEEPS - c->anchor_sweeps;
    const int64_t cap = left > 0 ? (left + k - 1) / k : 1;
    if (cap < L.max_iters) L.max_iters = (int)cap;
  }
  LGT_CUDA(cudaMemcpyAsync(c->d_loop, c->h_loop, sizeof(LoopState), cudaMemcpyHostToDevice, c->stream));
  const int bt = batch_begin(c, kind);
  LGT_CUDA(cudaGraphLaunch(c->loop_exec[slot], c->stream));
  batch_end(c, bt);
  LGT_CUDA(cudaMemcpyAsync(c->host, c->ws.fused_totals, sizeof(double) * TOT_N, cudaMemcpyDeviceToHost, c->stream));
  LGT_CUDA(cudaMemcpyAsync(c->h_loop, c->d_loop, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
  lgt_status st = sync_stream(c);
  if (st != LGT_OK) return st;
  const int64_t n = (int64_t)L.iters * k;
  c->sweep_index += (uint64_t)n;
  if (c->phase == 3) c->anchor_sweeps += n;
  if (kind == 0) c->sweeps_bulk += n;
  else c->sweeps_fp64 += n;
  *remaining = L.remaining;
  if (L.omega_switch == 0 && omega_schedule_open(c)) {  // the device loop switched omega
    c->cfg.omega = L.omega;
    c->omega_switched = 1;
  }
  if (best) *best = L.best;
  if (stall) *stall = L.stall;
  c->last_sites = lgt_cfg_sites(lc);
  c->stats.sweep_launches[kind] += 2 * n;
  c->stats.launches += (int64_t)L.iters * (c->loop_sweep_launches[slot] + 2);
  c->stats.site_updates[kind] += L.site_updates;
  c->stats.loop_launches++;
  c->stats.loop_chunks += L.iters;
  fill_meas(c, c->host, m);
  c->active_slices = m->active;
  return LGT_OK;
}

// whether the next chunks can run as a device loop (built on demand)
static bool loop_ready(lgt_ctx *c, int slot, int64_t remaining) {
  if (!c->use_loops || remaining < c->prm.check_every) return false;
  if (!c->loop_exec[slot] && build_loop(c, slot) != LGT_OK) return false;
  return true;
}

// ------------------------------------------------------ simulated annealing
// beta of annealing sweep i of n: geometric from beta0 to beta1
static double sa_beta(double beta0, double beta1, int n, int i) {
  if (n <= 1) return beta1;
  return beta0 * pow(beta1 / beta0, (double)i / (double)(n - 1));
}

// The loaded field's annealing sweeps (heat bath, launch configuration 0),
// counted as sweeps of the current phase.
static lgt_status run_annealing(lgt_ctx *c, int64_t *remaining) {
  const int n = (int)(c->prm.sa_sweeps < *remaining ? c->prm.sa_sweeps : *remaining);
  const int fmt = work_fmt(c);
  void *links = c->phase == 0 ? c->u32 : c->u64;
  void *G = c->phase == 0 ? c->G : nullptr;
  const int kind = c->phase == 0 ? 0 : 1;
  SweepCfg sc = c->cfg;
  sc.algo = ALGO_SA;
  const int bt = batch_begin(c, kind);
  for (int i = 0; i < n; i++) {
    sc.beta = sa_beta(c->prm.sa_beta0, c->prm.sa_beta1, c->prm.sa_sweeps, i);
    // Heat-bath rotations are far from the identity.  The FP32 storage keeps G
    // (and 12-real links) as two rows and rebuilds the third as a cross product,
    // so under such rotations the rows' norm error grows by about 4/3 per update
    // and overflows within some 50 sweeps: in FP32 every annealing sweep
    // reunitarises what it writes.
    const int reunit = c->phase == 0;
    for (int parity = 0; parity < 2; parity++)
      LGT_CUDA(launch_half_sweep(fmt, c->g, links, G, c->ws, sc, parity, c->sweep_index, reunit, 0, 0, c->stream));
    c->sweep_index++;
    if (kind == 0) c->sweeps_bulk++;
    else c->sweeps_fp64++;
  }
  batch_end(c, bt);
  c->last_sites = lgt_cfg_sites(0);
  c->stats.sweep_launches[kind] += 2 * n;
  c->stats.launches += 2 * n;
  c->stats.site_updates[kind] += 2LL * n * c->g.vs_half * c->g.nt;
  *remaining -= n;
  c->sa_pending = 0;
  return sync_stream(c);
}

// ------------------------------------------------------------- the driver
extern "C" lgt_status lgt_fix(lgt_ctx *ctx, lgt_result *res) {
  if (ctx && ctx->slab) {
    lgt_set_error("lgt_fix: a temporal slab is swept and measured through the lgt_slab_* calls");
    return LGT_EINVAL;
  }
  if (!ctx) {
    lgt_set_error("lgt_fix: NULL context");
    return LGT_EINVAL;
  }
  const auto t0 = std::chrono::steady_clock::now();
  lgt_ctx *c = ctx;
  const bool coulomb = c->prm.gauge == LGT_COULOMB;
  int64_t remaining = c->prm.max_sweeps;
  const int k = c->prm.check_every;
  const int64_t bulk0 = c->sweeps_bulk, fp640 = c->sweeps_fp64;
  Meas m;
  lgt_status st;
  bool promoted = false;
  if (c->sa_pending && (c->phase == 0 || c->phase == 1)) {
    st = run_annealing(c, &remaining);
    if (st != LGT_OK) return st;
  }
  if (c->phase == 0) {
    // bulk FP32 phase: until the working field's theta drops below theta_switch
    // or stops improving (the FP32 rounding floor)
    const double target = c->prm.theta_switch;
    st = measure(c, 0, coulomb ? target : -1.0, &m);
    if (st != LGT_OK) return st;
    omega_check(c, m.theta);
    double best = m.theta;
    int stall = 0;
    while (m.theta >= target && remaining > 0 && stall < LGT_STALL_CHECKS) {
      if (loop_ready(c, 0, remaining)) {  // whole chunks, decided on the device
        st = run_loop(c, 0, &best, &stall, &remaining, &m);
        if (st != LGT_OK) return st;
        continue;
      }
      const int n = (int)(remaining < k ? remaining : k);
      st = run_sweeps(c, n, coulomb ? 1 : 0);
      if (st != LGT_OK) return st;
      remaining -= n;
      st = estimate(c, coulomb ? target : -1.0, &m);
      if (st != LGT_OK) return st;
      omega_check(c, m.theta);
      if (m.theta < best) {
        best = m.theta;
        stall = 0;
      } else {
        stall = m.theta < LGT_STALL_CEILING ? stall + 1 : 0;
      }
    }
    st = promote(c);
    if (st != LGT_OK) return st;
    promoted = true;
  }
  // FP64-accurate phase to theta < tol
  const double tol = c->prm.theta_tol;
  bool certified = false;  // m is an exact measurement with the plaquette
  if (promoted) {
    // the promoted field carries the rounding of the FP32 G (theta ~ 1e-8, far
    // above any tolerance): polish first, every slice taking part until the
    // first estimate
    LGT_CUDA(cudaMemsetAsync(c->ws.active, 1, (size_t)c->g.nt, c->stream));
    c->active_slices = c->g.nt;
    m.theta = HUGE_VAL;
  } else {
    st = measure(c, 0, coulomb ? tol : -1.0, &m);
    if (st != LGT_OK) return st;
    omega_check(c, m.theta);
  }
  while (m.theta >= tol && remaining > 0) {
    st = anchor_refresh(c);
    if (st != LGT_OK) return st;
    if (loop_ready(c, 1, remaining)) {  // whole chunks, decided on the device
      st = run_loop(c, 1, nullptr, nullptr, &remaining, &m);
      if (st != LGT_OK) return st;
    } else {
      const int n = (int)(remaining < k ? remaining : k);
      st = run_sweeps(c, n, coulomb ? 1 : 0);
      if (st != LGT_OK) return st;
      remaining -= n;
      st = estimate(c, coulomb ? tol : -1.0, &m);
      if (st != LGT_OK) return st;
      omega_check(c, m.theta);
    }
    certified = false;
    if (m.theta < tol) {  // the estimate says converged: certify with the exact measurement
      st = measure(c, 1, coulomb ? tol : -1.0, &m);
      if (st != LGT_OK) return st;
      certified = true;
    }
  }
  // all slices active again for later calls
  LGT_CUDA(cudaMemsetAsync(c->ws.active, 1, (size_t)c->g.nt, c->stream));
  c->active_slices = c->g.nt;
  Meas fin = m;  // the certifying measurement covers every slice and the plaquette
  if (!certified) {
    st = measure(c, 1, -1.0, &fin);
    if (st != LGT_OK) return st;
  }
  const bool conv = m.theta < tol;
  if (res) {
    res->F = fin.F;
    res->theta = fin.theta;
    res->plaquette = fin.plaq;
    res->sweeps_bulk = c->sweeps_bulk - bulk0;
    res->sweeps_fp64 = c->sweeps_fp64 - fp640;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    res->status = conv ? LGT_OK : LGT_ENOTCONV;
    res->reserved = 0;
  }
  if (!conv) {
    lgt_set_error("not converged: theta = %.3e after %d sweeps", m.theta, c->prm.max_sweeps);
    return LGT_ENOTCONV;
  }
  return LGT_OK;
}

// ------------------------------------------------------------- egress
static lgt_status to_output(lgt_ctx *c, double *out, int out_on_device, int working) {
  const Geom &g = c->g;
  const size_t aos_bytes = (size_t)g.vh * 2 * 4 * 18 * sizeof(double);
  double *dst = out;
  double *tmp = nullptr;
  if (!out_on_device) {
    if (!c->stage) {
      cudaError_t e = cudaMalloc(&c->stage, aos_bytes);
      if (e != cudaSuccess) {
        lgt_set_error("cudaMalloc of the staging buffer failed: %s", cudaGetErrorString(e));
        return LGT_ENOMEM;
      }
    }
    tmp = c->stage;
    dst = tmp;
  }
  cudaError_t e;
  if (c->phase == 3 && c->d_dirty) e = launch_apply_D(g, c->G, c->u64, nullptr, dst, skip_temporal(c), c->stream);
  else if (c->phase >= 1) e = launch_egress(work_fmt(c), g, c->u64, dst, c->stream);
  else if (working) e = launch_egress(c->bulk_fmt, g, c->u32, dst, c->stream);
  else e = launch_apply_G(g, c->G, c->u64, nullptr, dst, skip_temporal(c), c->stream);
  c->stats.launches++;
  if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(out, tmp, aos_bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  resolve_events(c);
  if (e != cudaSuccess) {
    lgt_set_error("link egress failed: %s", cudaGetErrorString(e));
    return LGT_ECUDA;
  }
  return LGT_OK;
}

// a slab's owned slices of its working links (public layout, FP64)
static lgt_status slab_output(lgt_ctx *c, double *out, int out_on_device) {
  const Geom &g = c->g;
  const size_t slice_doubles = (size_t)g.vs_half * 2 * 4 * 18;
  if (!c->stage) LGT_CUDA(cudaMalloc(&c->stage, slice_doubles * g.nt * sizeof(double)));
  LGT_CUDA(launch_egress(work_fmt(c), g, c->phase == 0 ? c->u32 : c->u64, c->stage, c->stream));
  c->stats.launches++;
  LGT_CUDA(cudaMemcpyAsync(out, c->stage + 2 * slice_doubles, slice_doubles * (g.nt - 2) * sizeof(double),
                           out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return sync_stream(c);
}

extern "C" lgt_status lgt_get_links(lgt_ctx *ctx, double *out, int out_on_device) {
  if (!ctx || !out) {
    lgt_set_error("lgt_get_links: bad arguments");
    return LGT_EINVAL;
  }
  if (ctx->slab) return slab_output(ctx, out, out_on_device);
  return to_output(ctx, out, out_on_device, 0);
}

extern "C" lgt_status lgt_get_working_links(lgt_ctx *ctx, double *out, int out_on_device) {
  if (!ctx || !out) {
    lgt_set_error("lgt_get_working_links: bad arguments");
    return LGT_EINVAL;
  }
  if (ctx->slab) return slab_output(ctx, out, out_on_device);
  return to_output(ctx, out, out_on_device, 1);
}

extern "C" lgt_status lgt_get_progress(lgt_ctx *ctx, int64_t *sweeps_bulk, int64_t *sweeps_fp64, int32_t *phase) {
  if (!ctx) {
    lgt_set_error("lgt_get_progress: NULL context");
    return LGT_EINVAL;
  }
  if (sweeps_bulk) *sweeps_bulk = ctx->sweeps_bulk;
  if (sweeps_fp64) *sweeps_fp64 = ctx->sweeps_fp64;
  if (phase) *phase = ctx->phase;
  return LGT_OK;
}
