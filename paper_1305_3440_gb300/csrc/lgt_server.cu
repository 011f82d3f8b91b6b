// lgt_server.cu -- continuous-batching gauge-fixing server (include/lgt.h).
//
// One worker thread owns a CUDA stream and a device memory pool.  Each tick:
//   1. admit queued jobs (FIFO) while their device footprint fits the HBM
//      budget: allocate, upload, ingest (SU(3) check), measure;
//   2. advance every live job by up to check_every sweeps: for each sweep and
//      parity, one batched half-sweep launch per kernel variant (storage
//      format x gauge x algorithm) covers the sites of all live jobs of that
//      variant;
//   3. one batched reduction of the sweeps' fused estimates gives each job's
//      F and theta; jobs that start, or whose estimate says converged, get a
//      batched exact measurement instead (with the plaquette when it
//      certifies; one device->host copy for all jobs);
//   4. per job, the same ladder decisions as lgt_fix (Sec. 4 driver): bulk FP32
//      until theta < theta_switch (or the FP32 floor), promotion, polishing to
//      theta < theta_tol, or max_sweeps; finished jobs are copied out (measured
//      once more unless a certifying measurement holds the result) and their
//      memory released, which admits the next ones.
// The tick's launch sequence is captured into a CUDA graph and replayed while
// its shape repeats (see tick()).
// A job's sequence of kernels and decisions depends only on its own
// parameters, so its result is bit-identical alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "lgt_api_internal.h"
#include "lgt_internal.h"

using namespace lgt;

namespace {

using Clock = std::chrono::steady_clock;

enum { JOB_QUEUED = 0, JOB_RUNNING = 1, JOB_DONE = 2 };

constexpr int kServerBlock = 128;
constexpr int kMaxSlots = 4096;

int fmt_of_prec(int32_t prec) {
  return prec == LGT_FP32_18 ? FMT_F32_18 : (prec == LGT_FP32_12 ? FMT_F32_12 : FMT_F64);
}

unsigned long long sr_thr_of(double p) {
  if (!(p > 0.0)) return 0ull;
  if (p >= 1.0) return 1ull << 32;
  return (unsigned long long)floor(p * 4294967296.0);
}

struct Job {
  uint64_t id = 0;
  lgt_params prm;
  std::vector<double> input, output;
  lgt_result res;
  int state = JOB_QUEUED;
  bool cancel = false;
  Clock::time_point t_submit, t_start, t_end;
  size_t bytes = 0;
  int slot = -1;
  // device state
  Geom g;
  void *u64 = nullptr, *u32 = nullptr, *G = nullptr, *k0 = nullptr, *ws_base = nullptr;
  Workspace ws;
  int phase = 0, bulk_fmt = FMT_F64;  // phase as lgt_get_progress (3: anchored polish)
  bool anchored = false, d_dirty = false;
  int64_t anchor_sweeps = 0;  // anchored polish: sweeps since the last anchor set-up
  SweepCfg cfg;
  int64_t sweeps_bulk = 0, sweeps_fp64 = 0, remaining = 0;
  uint64_t sweep_index = 0;
  double best = 0.0;
  int stall = 0;
  bool omega_switched = false;  // omega schedule: the sweeps run at omega_late
  bool measure_only = true;  // next tick measures without sweeping
  bool certify = false;      // that measurement certifies convergence (with the plaquette)
  int nthis = 0;             // sweeps in the current tick
  int nbx = 0;

  // storage of the field that measurements read (the anchored polish measures
  // the formed field in u64)
  int work_fmt() const { return phase == 0 ? bulk_fmt : (phase == 2 ? (int)FMT_PAIR : (int)FMT_F64); }
  void *work_links() const { return phase == 0 ? u32 : u64; }
  // kernel variant and links of the sweeps
  int sweep_fmt() const { return phase == 3 ? (int)FMT_ANCHOR : work_fmt(); }
  void *sweep_links() const { return (phase == 0 || phase == 3) ? u32 : u64; }
  int skip_temporal() const { return (prm.gauge == LGT_COULOMB && !prm.transform_temporal) ? 1 : 0; }
  double theta_of(const double *tot) const {
    return prm.gauge == LGT_COULOMB ? tot[TOT_THETA_COULOMB_MAX] : tot[TOT_THETA_LANDAU];
  }
  double F_of(const double *tot) const {
    return prm.gauge == LGT_COULOMB ? tot[TOT_F_COULOMB] : tot[TOT_F_LANDAU];
  }
};

size_t aos_bytes_of(const Geom &g) { return (size_t)g.vh * 2 * 4 * 18 * sizeof(double); }

constexpr size_t kMaxGraphs = 16;

// One captured tick: its launch shape and executable graph.
struct TickGraph {
  std::vector<long long> sig;
  cudaGraphExec_t exec;
  uint64_t used;
};

}  // namespace

struct lgt_server {
  size_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job *> queue;
  std::map<uint64_t, Job *> jobs;
  uint64_t next_id = 1, done = 0;
  size_t used = 0;
  bool stop = false;
  std::thread worker;
  // worker-owned
  std::vector<Job *> live;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  double *d_totals = nullptr, *h_totals = nullptr;
  std::vector<int> free_slots;
  BatchSweep *d_sweep = nullptr, *h_sweep = nullptr;
  BatchMeas *d_meas = nullptr, *h_meas = nullptr;
  BatchFused *d_fused = nullptr, *h_fused = nullptr;
  size_t sweep_cap = 0, meas_cap = 0, fused_cap = 0;
  // captured ticks (worker-owned) and counters (read under mu)
  std::vector<TickGraph> graphs;
  std::vector<long long> prev_sig;
  bool use_graphs = true;
  uint64_t ticks = 0, graph_launches = 0, graph_captures = 0, kernel_launches = 0;
  cudaError_t fatal = cudaSuccess;
};

namespace {

cudaError_t dev_alloc(lgt_server *s, void **p, size_t n) { return cudaMallocFromPoolAsync(p, n, s->pool, s->stream); }

void release_job_device(lgt_server *s, Job *j) {
  void **ptrs[] = {&j->u64, &j->u32, &j->G, &j->k0, &j->ws_base};
  for (void **p : ptrs)
    if (*p) {
      cudaFreeAsync(*p, s->stream);
      *p = nullptr;
    }
  if (j->slot >= 0) {
    s->free_slots.push_back(j->slot);
    j->slot = -1;
  }
}

// under s->mu
void finish_locked(lgt_server *s, Job *j, int status) {
  j->state = JOB_DONE;
  j->t_end = Clock::now();
  j->res.status = status;
  j->res.seconds = std::chrono::duration<double>(j->t_end - j->t_submit).count();
  j->res.sweeps_bulk = j->sweeps_bulk;
  j->res.sweeps_fp64 = j->sweeps_fp64;
  s->used -= j->bytes;
  j->bytes = 0;
  s->done++;
  s->cv.notify_all();
}

// allocate, upload and ingest one job (worker thread; j->slot already taken)
cudaError_t admit(lgt_server *s, Job *j, int *bad_input) {
  const lgt_params &p = j->prm;
  j->g = lgt_make_geom(p.dims);
  const Geom &g = j->g;
  j->bulk_fmt = fmt_of_prec(p.bulk);
  j->phase = p.bulk == LGT_FP64 ? 1 : 0;
  j->cfg.gauge = p.gauge == LGT_COULOMB ? GAUGE_COULOMB : GAUGE_LANDAU;
  j->cfg.algo = p.algo == LGT_SR ? ALGO_SR : ALGO_OR;
  j->cfg.omega = p.omega;  // omega_polish takes over at promotion
  j->cfg.sr_thr = sr_thr_of(p.p);
  j->cfg.seed = p.seed;
  j->cfg.transform_temporal = p.transform_temporal ? 1 : 0;
  j->sweep_index = p.sweep_offset;
  j->remaining = p.max_sweeps;
  j->nbx = (g.vs_half + kServerBlock - 1) / kServerBlock;
  cudaError_t e;
  if ((e = dev_alloc(s, &j->u64, field_bytes(FMT_F64, g.vh))) != cudaSuccess) return e;
  if (p.bulk != LGT_FP64) {
    if ((e = dev_alloc(s, &j->u32, field_bytes(j->bulk_fmt, g.vh))) != cudaSuccess) return e;
    const bool anch = p.polish == LGT_POLISH_ANCHOR;
    if ((e = dev_alloc(s, &j->G, anch ? d_bytes(g.vh) : g_bytes(g.vh))) != cudaSuccess) return e;
    if (anch && (e = dev_alloc(s, &j->k0, k0_bytes(g.vh))) != cudaSuccess) return e;
  }
  const size_t wsb = workspace_bytes(g, 64);
  if ((e = dev_alloc(s, &j->ws_base, wsb)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(j->ws_base, 0, wsb, s->stream)) != cudaSuccess) return e;
  workspace_carve(j->ws_base, g, 64, &j->ws);
  j->ws.totals = s->d_totals + (size_t)j->slot * TOT_N;
  j->ws.fused_totals = s->d_totals + ((size_t)kMaxSlots + j->slot) * TOT_N;
  if ((e = cudaMemsetAsync(j->ws.active, 1, (size_t)g.nt, s->stream)) != cudaSuccess) return e;
  void *stage = nullptr;
  if ((e = dev_alloc(s, &stage, aos_bytes_of(g))) != cudaSuccess) return e;
  e = cudaMemcpyAsync(stage, j->input.data(), aos_bytes_of(g), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = launch_ingest(FMT_F64, g, (const double *)stage, j->u64, j->ws.err, s->stream);
  if (e == cudaSuccess && j->u32) e = launch_ingest(j->bulk_fmt, g, (const double *)stage, j->u32, j->ws.err, s->stream);
  if (e == cudaSuccess && j->G) e = launch_g_identity(g, j->G, s->stream);
  int err_h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err_h, j->ws.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(stage, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  std::vector<double>().swap(j->input);
  *bad_input = err_h != 0;
  return e;
}

// anchored polish: form U <- G U' G^+ in u64 (the job's measured field; the
// next sweep re-anchors), and the anchor set-up
cudaError_t anchor_materialise(lgt_server *s, Job *j) {
  if (j->phase != 3 || !j->d_dirty) return cudaSuccess;
  j->d_dirty = j->anchored = false;
  return launch_apply_D(j->g, j->G, j->u64, j->u64, nullptr, j->skip_temporal(), s->stream);
}

cudaError_t anchor_setup(lgt_server *s, Job *j) {
  if (j->phase != 3 || j->anchored) return cudaSuccess;
  j->anchored = true;
  j->anchor_sweeps = 0;
  return launch_anchor_setup(j->g, j->u64, j->u32, j->k0, j->G, j->cfg.gauge, s->stream);
}

double coulomb_target(const Job *j) {
  if (j->prm.gauge != LGT_COULOMB) return -1.0;
  return j->phase == 0 ? j->prm.theta_switch : j->prm.theta_tol;
}

struct Segment {
  int fmt, gauge, algo, s;
  size_t offset;
  int n, blocks;
};

void drop_graphs(lgt_server *s) {
  for (TickGraph &t : s->graphs) cudaGraphExecDestroy(t.exec);
  s->graphs.clear();
  s->prev_sig.clear();
}

cudaError_t ensure_tables(lgt_server *s, size_t nsweep, size_t nmeas, size_t nfused) {
  cudaError_t e = cudaSuccess;
  if (nfused > s->fused_cap || nsweep > s->sweep_cap || nmeas > s->meas_cap) drop_graphs(s);  // tables move
  if (nfused > s->fused_cap) {
    size_t cap = std::max(nfused, 2 * s->fused_cap);
    if (s->d_fused) cudaFree(s->d_fused);
    if (s->h_fused) cudaFreeHost(s->h_fused);
    s->d_fused = nullptr;
    s->h_fused = nullptr;
    if ((e = cudaMalloc(&s->d_fused, cap * sizeof(BatchFused))) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&s->h_fused, cap * sizeof(BatchFused))) != cudaSuccess) return e;
    s->fused_cap = cap;
  }
  if (nsweep > s->sweep_cap) {
    size_t cap = std::max(nsweep, 2 * s->sweep_cap);
    if (s->d_sweep) cudaFree(s->d_sweep);
    if (s->h_sweep) cudaFreeHost(s->h_sweep);
    s->d_sweep = nullptr;
    s->h_sweep = nullptr;
    if ((e = cudaMalloc(&s->d_sweep, cap * sizeof(BatchSweep))) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&s->h_sweep, cap * sizeof(BatchSweep))) != cudaSuccess) return e;
    s->sweep_cap = cap;
  }
  if (nmeas > s->meas_cap) {
    size_t cap = std::max(nmeas, 2 * s->meas_cap);
    if (s->d_meas) cudaFree(s->d_meas);
    if (s->h_meas) cudaFreeHost(s->h_meas);
    s->d_meas = nullptr;
    s->h_meas = nullptr;
    if ((e = cudaMalloc(&s->d_meas, cap * sizeof(BatchMeas))) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&s->h_meas, cap * sizeof(BatchMeas))) != cudaSuccess) return e;
    s->meas_cap = cap;
  }
  return e;
}

// The launch shape of one tick: which batched launches, over how many rows
// and blocks.  The rows themselves live in the pinned host tables and are
// copied to the device by the tick's first operations, so two ticks with the
// same shape run the same operations on different table contents.
struct TickPlan {
  int kmax, hi_slot, fblocks;
  size_t nrows, nmrows, nfrows;
  std::vector<Segment> segs, msegs;

  std::vector<long long> signature() const {
    std::vector<long long> v = {kmax, hi_slot, fblocks, (long long)nrows, (long long)nmrows, (long long)nfrows};
    for (const std::vector<Segment> *L : {&segs, &msegs})
      for (const Segment &g : *L) {
        const long long f[] = {g.fmt, g.gauge, g.algo, g.s, (long long)g.offset, g.n, g.blocks};
        v.insert(v.end(), f, f + 7);
      }
    return v;
  }
  long long launches() const { return 2 * (long long)segs.size() + (nfrows ? 1 : 0) + (long long)msegs.size(); }
};

// Stream operations of one tick: table uploads, the batched sweeps (for each
// sweep offset both parities, every kernel variant), the batched fused
// estimate, the batched exact measurements, and the totals read-back.
cudaError_t issue(lgt_server *s, const TickPlan &P) {
  cudaError_t e = cudaSuccess;
  if (P.nfrows &&
      (e = cudaMemcpyAsync(s->d_fused, s->h_fused, P.nfrows * sizeof(BatchFused), cudaMemcpyHostToDevice,
                           s->stream)) != cudaSuccess)
    return e;
  if (P.nrows &&
      (e = cudaMemcpyAsync(s->d_sweep, s->h_sweep, P.nrows * sizeof(BatchSweep), cudaMemcpyHostToDevice,
                           s->stream)) != cudaSuccess)
    return e;
  if (P.nmrows &&
      (e = cudaMemcpyAsync(s->d_meas, s->h_meas, P.nmrows * sizeof(BatchMeas), cudaMemcpyHostToDevice,
                           s->stream)) != cudaSuccess)
    return e;
  size_t si = 0;
  for (int sw = 0; sw < P.kmax; sw++) {
    const size_t first = si;
    while (si < P.segs.size() && P.segs[si].s == sw) si++;
    for (int parity = 0; parity < 2; parity++)
      for (size_t q = first; q < si; q++) {
        const Segment &g = P.segs[q];
        e = launch_half_sweep_batch(g.fmt, g.gauge, g.algo, s->d_sweep + g.offset, g.n, g.blocks, parity, sw,
                                    kServerBlock, s->stream);
        if (e != cudaSuccess) return e;
      }
  }
  if (P.nfrows && (e = launch_fused_finish_batch(s->d_fused, (int)P.nfrows, P.fblocks, s->stream)) != cudaSuccess)
    return e;
  for (const Segment &g : P.msegs)
    if ((e = launch_measure_batch(g.fmt, s->d_meas + g.offset, g.n, g.blocks, kServerBlock, s->stream)) !=
        cudaSuccess)
      return e;
  // exact totals of slots [0, hi_slot), then the fused estimates of the same slots
  const size_t n = sizeof(double) * TOT_N * (size_t)P.hi_slot;
  if ((e = cudaMemcpyAsync(s->h_totals, s->d_totals, n, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess) return e;
  return cudaMemcpyAsync(s->h_totals + (size_t)kMaxSlots * TOT_N, s->d_totals + (size_t)kMaxSlots * TOT_N, n,
                         cudaMemcpyDeviceToHost, s->stream);
}

// One tick over the live jobs: sweeps, measurement, read back.
cudaError_t tick(lgt_server *s) {
  std::vector<Job *> &live = s->live;
  int kmax = 0;
  for (Job *j : live) {
    j->nthis = j->measure_only ? 0 : (int)std::min<int64_t>(j->prm.check_every, j->remaining);
    kmax = std::max(kmax, j->nthis);
  }
  // anchored polish jobs: the exact measurement reads the formed field, the
  // sweeps need a current anchor (rare: at promotion and certification; issued
  // before, and outside, the tick's captured sequence)
  for (Job *j : live) {
    cudaError_t e = cudaSuccess;
    // as lgt_fix: a measurement forms the field; so does an anchor that has
    // served LGT_REANCHOR_SWEEPS sweeps (the next sweeps set up a new one)
    if (j->measure_only || (j->phase == 3 && j->anchored && j->anchor_sweeps >= LGT_REANCHOR_SWEEPS))
      e = anchor_materialise(s, j);
    if (e == cudaSuccess && !j->measure_only) e = anchor_setup(s, j);
    if (e != cudaSuccess) return e;
    if (!j->measure_only && j->phase == 3) j->d_dirty = true;
  }
  // sweep segments: for each sweep offset s, jobs grouped by kernel variant
  std::vector<Segment> segs;
  std::vector<BatchSweep> rows;
  std::vector<Job *> order(live);
  std::stable_sort(order.begin(), order.end(), [](const Job *a, const Job *b) {
    const int ka = (a->sweep_fmt() * 2 + a->cfg.gauge) * 2 + a->cfg.algo;
    const int kb = (b->sweep_fmt() * 2 + b->cfg.gauge) * 2 + b->cfg.algo;
    return ka < kb;
  });
  for (int sw = 0; sw < kmax; sw++) {
    size_t i = 0;
    while (i < order.size()) {
      const Job *h = order[i];
      Segment seg = {h->sweep_fmt(), h->cfg.gauge, h->cfg.algo, sw, rows.size(), 0, 0};
      size_t k = i;
      for (; k < order.size(); k++) {
        Job *j = order[k];
        if (j->sweep_fmt() != seg.fmt || j->cfg.gauge != seg.gauge || j->cfg.algo != seg.algo) break;
        if (sw >= j->nthis) continue;
        BatchSweep r{};
        fill_sweep_args(&r.a, j->g, j->sweep_links(), (j->phase == 0 || j->phase == 3) ? j->G : nullptr, j->ws,
                        j->cfg, j->sweep_index, 0, j->prm.gauge == LGT_COULOMB ? 1 : 0);
        r.a.aux = j->phase == 3 ? j->k0 : nullptr;
        r.a.reunit_every = j->phase == 0 ? j->prm.reunit_every : 0;
        r.a.count_base = j->sweeps_bulk;
        r.block_begin = seg.blocks;
        r.nbx = j->nbx;
        rows.push_back(r);
        seg.n++;
        seg.blocks += j->nbx * j->g.nt;
      }
      if (seg.n) segs.push_back(seg);
      i = k;
    }
  }
  // fused-estimate rows: every job that sweeps this tick (one block per slice)
  std::vector<BatchFused> frows;
  int fblocks = 0;
  for (Job *j : live) {
    if (j->measure_only) continue;
    BatchFused r{};
    fill_fused_args(&r.a, j->g, j->ws, j->cfg.gauge, kServerBlock, coulomb_target(j));  // one thread per site
    r.block_begin = fblocks;
    r.nbx = 0;
    frows.push_back(r);
    fblocks += j->g.nt;
  }
  // exact-measurement segments (jobs in a measurement-only tick): one per storage format
  std::vector<Segment> msegs;
  std::vector<BatchMeas> mrows;
  std::vector<Job *> morder;
  for (Job *j : live)
    if (j->measure_only) morder.push_back(j);
  std::stable_sort(morder.begin(), morder.end(),
                   [](const Job *a, const Job *b) { return a->work_fmt() < b->work_fmt(); });
  for (size_t i = 0; i < morder.size();) {
    Segment seg = {morder[i]->work_fmt(), 0, 0, 0, mrows.size(), 0, 0};
    size_t k = i;
    for (; k < morder.size() && morder[k]->work_fmt() == seg.fmt; k++) {
      Job *j = morder[k];
      BatchMeas r{};
      fill_meas_args(&r.a, j->g, j->work_links(), j->ws, j->certify ? 1 : 0, coulomb_target(j));
      r.block_begin = seg.blocks;
      r.nbx = j->nbx;
      mrows.push_back(r);
      seg.n++;
      seg.blocks += 2 * j->nbx * j->g.nt;
    }
    msegs.push_back(seg);
    i = k;
  }
  int hi_slot = 0;  // totals of slots [0, hi_slot) come back to the host
  for (Job *j : live) hi_slot = std::max(hi_slot, j->slot + 1);
  cudaError_t e = ensure_tables(s, rows.size(), mrows.size(), frows.size());
  if (e != cudaSuccess) return e;
  if (!frows.empty()) memcpy(s->h_fused, frows.data(), frows.size() * sizeof(BatchFused));
  if (!rows.empty()) memcpy(s->h_sweep, rows.data(), rows.size() * sizeof(BatchSweep));
  if (!mrows.empty()) memcpy(s->h_meas, mrows.data(), mrows.size() * sizeof(BatchMeas));
  TickPlan P{kmax, hi_slot, fblocks, rows.size(), mrows.size(), frows.size(), std::move(segs), std::move(msegs)};
  const std::vector<long long> sig = P.signature();
  s->ticks++;
  s->kernel_launches += P.launches();
  TickGraph *hit = nullptr;
  for (TickGraph &t : s->graphs)
    if (t.sig == sig) hit = &t;
  if (!hit && s->use_graphs && sig == s->prev_sig) {
    // the same launch shape two ticks in a row: capture it once, replay it while it lasts
    if ((e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    const cudaError_t ei = issue(s, P);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s->stream, &graph);
    if (ei != cudaSuccess) e = ei;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (s->graphs.size() >= kMaxGraphs) {
      auto lru = std::min_element(s->graphs.begin(), s->graphs.end(),
                                  [](const TickGraph &x, const TickGraph &y) { return x.used < y.used; });
      cudaGraphExecDestroy(lru->exec);
      s->graphs.erase(lru);
    }
    s->graphs.push_back({sig, exec, 0});
    s->graph_captures++;
    hit = &s->graphs.back();
  }
  s->prev_sig = sig;
  if (hit) {
    hit->used = s->ticks;
    s->graph_launches++;
    e = cudaGraphLaunch(hit->exec, s->stream);
  } else {
    e = issue(s, P);
  }
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s->stream);
}

// final measurement with plaquette and copy-out of a finished job
cudaError_t collect(lgt_server *s, Job *j) {
  cudaError_t e = anchor_materialise(s, j);
  if (e != cudaSuccess) return e;
  if (!j->certify) {  // a certifying measurement already holds F, theta and the plaquette
    e = launch_measure(j->work_fmt(), j->g, j->work_links(), j->ws, 1, -1.0, kServerBlock, s->stream);
    if (e != cudaSuccess) return e;
  }
  void *stage = nullptr;
  if ((e = dev_alloc(s, &stage, aos_bytes_of(j->g))) != cudaSuccess) return e;
  if (j->phase >= 1) e = launch_egress(j->work_fmt(), j->g, j->u64, (double *)stage, s->stream);
  else e = launch_apply_G(j->g, j->G, j->u64, nullptr, (double *)stage,
                          (j->prm.gauge == LGT_COULOMB && !j->prm.transform_temporal) ? 1 : 0, s->stream);
  j->output.resize(aos_bytes_of(j->g) / sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(j->output.data(), stage, aos_bytes_of(j->g), cudaMemcpyDeviceToHost, s->stream);
  double tot[TOT_N];
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot, j->ws.totals, sizeof tot, cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(stage, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return e;
  j->res.F = j->F_of(tot);
  j->res.theta = j->theta_of(tot);
  j->res.plaquette = tot[TOT_PLAQ];
  return cudaSuccess;
}

cudaError_t promote_job(lgt_server *s, Job *j) {
  cudaError_t e = launch_apply_G(j->g, j->G, j->u64, j->u64, nullptr, j->skip_temporal(), s->stream);
  j->phase = 1;
  if (j->prm.polish_algo == LGT_POLISH_OR) j->cfg.algo = ALGO_OR;  // the sweeps after promotion overrelax
  if (j->prm.omega_polish != 0.0) j->cfg.omega = j->prm.omega_polish;
  if (e == cudaSuccess && j->prm.polish == LGT_POLISH_PAIR) {
    e = launch_convert_pair(j->g, j->u64, 1, s->stream);
    j->phase = 2;
  } else if (j->prm.polish == LGT_POLISH_ANCHOR) {
    j->phase = 3;
    j->anchored = j->d_dirty = false;
  }
  // as lgt_fix: no measurement of the promoted field (its theta is far above any
  // tolerance); every slice takes part until the first estimate
  if (e == cudaSuccess) e = cudaMemsetAsync(j->ws.active, 1, (size_t)j->g.nt, s->stream);
  j->measure_only = false;
  return e;
}

void worker_main(lgt_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // admission (FIFO, by budget)
    while (!s->stop && s->fatal == cudaSuccess && !s->queue.empty()) {
      Job *j = s->queue.front();
      if (j->cancel) {
        s->queue.pop_front();
        finish_locked(s, j, LGT_ECANCELLED);
        continue;
      }
      const size_t need = lgt_ctx_device_bytes(&j->prm);
      const size_t stage = aos_bytes_of(lgt_make_geom(j->prm.dims));
      if (s->used + need + stage > s->budget || s->free_slots.empty()) break;
      s->queue.pop_front();
      j->bytes = need;
      s->used += need;
      j->slot = s->free_slots.back();
      s->free_slots.pop_back();
      j->state = JOB_RUNNING;
      j->t_start = Clock::now();
      int bad = 0;
      lk.unlock();
      cudaError_t e = admit(s, j, &bad);
      lk.lock();
      if (e != cudaSuccess) {
        s->fatal = e;
        release_job_device(s, j);
        finish_locked(s, j, e == cudaErrorMemoryAllocation ? LGT_ENOMEM : LGT_ECUDA);
        break;
      }
      if (bad) {
        release_job_device(s, j);
        finish_locked(s, j, LGT_EINVAL);
        continue;
      }
      s->live.push_back(j);
    }
    if (s->stop) break;
    if (s->live.empty()) {
      s->cv.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    // cancelled jobs leave at the tick boundary
    for (size_t i = 0; i < s->live.size();) {
      Job *j = s->live[i];
      if (j->cancel) {
        release_job_device(s, j);
        finish_locked(s, j, LGT_ECANCELLED);
        s->live.erase(s->live.begin() + i);
      } else {
        i++;
      }
    }
    if (s->live.empty()) continue;
    lk.unlock();
    cudaError_t e = tick(s);
    std::vector<Job *> finished;
    std::vector<int> fstatus;
    if (e == cudaSuccess) {
      // the same decisions as lgt_fix: exact measurements (measure-only ticks) at
      // the start, after promotion and to certify; the sweeps' fused estimate
      // otherwise
      for (Job *j : s->live) {
        const bool exact = j->measure_only;
        const double *tot = s->h_totals + ((exact ? 0 : (size_t)kMaxSlots) + j->slot) * TOT_N;
        const double theta = j->theta_of(tot);
        if (!exact) {
          if (j->phase == 0) j->sweeps_bulk += j->nthis;
          else j->sweeps_fp64 += j->nthis;
          if (j->phase == 3) j->anchor_sweeps += j->nthis;
          j->remaining -= j->nthis;
          j->sweep_index += (uint64_t)j->nthis;
        }
        j->measure_only = false;
        // omega schedule, as lgt_fix: the sweeps before promotion (every sweep of
        // an FP64 job) move to omega_late at the first check below theta_omega
        if (j->prm.omega_late != 0.0 && !j->omega_switched && (j->phase == 0 || j->prm.bulk == LGT_FP64) &&
            theta < j->prm.theta_omega) {
          j->cfg.omega = j->prm.omega_late;
          j->omega_switched = true;
        }
        const bool certified = exact && j->certify;
        j->certify = false;
        if (j->phase == 0) {
          if (exact) {
            j->best = theta;
            j->stall = 0;
          } else if (theta < j->best) {
            j->best = theta;
            j->stall = 0;
          } else {
            j->stall = theta < LGT_STALL_CEILING ? j->stall + 1 : 0;
          }
          if (theta < j->prm.theta_switch || j->remaining <= 0 || j->stall >= LGT_STALL_CHECKS) {
            if ((e = promote_job(s, j)) != cudaSuccess) break;
          }
        } else if (theta < j->prm.theta_tol) {
          if (exact) {
            j->certify = certified;  // collect() reuses the certifying measurement
            finished.push_back(j);
            fstatus.push_back(LGT_OK);
          } else {
            j->measure_only = true;  // certify next tick
            j->certify = true;
          }
        } else if (j->remaining <= 0) {
          finished.push_back(j);
          fstatus.push_back(LGT_ENOTCONV);
        }
      }
      for (size_t q = 0; q < finished.size() && e == cudaSuccess; q++) e = collect(s, finished[q]);
    }
    lk.lock();
    if (e != cudaSuccess) {
      s->fatal = e;
      lgt_set_error("server worker: %s", cudaGetErrorString(e));
      for (Job *j : s->live) {
        release_job_device(s, j);
        finish_locked(s, j, LGT_ECUDA);
      }
      s->live.clear();
      continue;
    }
    for (size_t q = 0; q < finished.size(); q++) {
      Job *j = finished[q];
      release_job_device(s, j);
      finish_locked(s, j, fstatus[q]);
      s->live.erase(std::find(s->live.begin(), s->live.end(), j));
    }
  }
  // shutdown: queued and live jobs are cancelled
  for (Job *j : s->live) {
    release_job_device(s, j);
    finish_locked(s, j, LGT_ECANCELLED);
  }
  s->live.clear();
  while (!s->queue.empty()) {
    finish_locked(s, s->queue.front(), LGT_ECANCELLED);
    s->queue.pop_front();
  }
  lk.unlock();
  cudaStreamSynchronize(s->stream);
}

}  // namespace

extern "C" lgt_status lgt_server_create(size_t hbm_budget_bytes, int device, lgt_server **out) {
  if (!out) {
    lgt_set_error("lgt_server_create: out is NULL");
    return LGT_EINVAL;
  }
  *out = nullptr;
  if (lgt_fault_injected("alloc")) {
    lgt_set_error("lgt_server_create: device allocation failed (injected by LGT_FAULT)");
    return LGT_ENOMEM;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    lgt_set_error("lgt_server_create: no CUDA device %d (%s)", device, cudaGetErrorString(e));
    return e == cudaSuccess ? LGT_EINVAL : LGT_ECUDA;
  }
  lgt_server *s = new lgt_server();
  const char *gv = getenv("LGT_SERVER_GRAPHS");  // "0": issue every tick's launches directly
  s->use_graphs = !(gv && gv[0] == '0');
  s->budget = hbm_budget_bytes;
  s->device = device;
  e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&s->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached for the next admissions
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  // exact totals in slots [0, kMaxSlots), fused estimates in [kMaxSlots, 2 kMaxSlots)
  if (e == cudaSuccess) e = cudaMalloc(&s->d_totals, sizeof(double) * TOT_N * 2 * kMaxSlots);
  if (e == cudaSuccess) e = cudaMemset(s->d_totals, 0, sizeof(double) * TOT_N * 2 * kMaxSlots);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_totals, sizeof(double) * TOT_N * 2 * kMaxSlots);
  if (e != cudaSuccess) {
    lgt_set_error("lgt_server_create: %s", cudaGetErrorString(e));
    if (s->d_totals) cudaFree(s->d_totals);
    if (s->h_totals) cudaFreeHost(s->h_totals);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return e == cudaErrorMemoryAllocation ? LGT_ENOMEM : LGT_ECUDA;
  }
  for (int k = kMaxSlots - 1; k >= 0; k--) s->free_slots.push_back(k);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return LGT_OK;
}

extern "C" lgt_status lgt_submit(lgt_server *s, const lgt_params *params, const double *links, uint64_t *job_id) {
  if (!s || !links || !job_id) {
    lgt_set_error("lgt_submit: bad arguments");
    return LGT_EINVAL;
  }
  lgt_status st = lgt_validate_params(params);
  if (st != LGT_OK) return st;
  if (params->sa_sweeps > 0) {
    lgt_set_error("lgt_submit: simulated annealing runs in lgt_fix only (sa_sweeps must be 0)");
    return LGT_EINVAL;
  }
  if (params->gauge == LGT_MAG) {
    lgt_set_error("lgt_submit: the maximally Abelian gauge runs in lgt_fix only");
    return LGT_EINVAL;
  }
  const size_t need = lgt_ctx_device_bytes(params) + aos_bytes_of(lgt_make_geom(params->dims));
  if (need > s->budget) {
    lgt_set_error("job needs %zu device bytes, more than the server budget %zu", need, s->budget);
    return LGT_ENOMEM;
  }
  Job *j = new Job();
  j->prm = *params;
  memset(&j->res, 0, sizeof j->res);
  const Geom g = lgt_make_geom(params->dims);
  j->input.assign(links, links + aos_bytes_of(g) / sizeof(double));
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete j;
    lgt_set_error("lgt_submit: server is stopping");
    return LGT_EBUSY;
  }
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  *job_id = j->id;
  s->cv.notify_all();
  return LGT_OK;
}

extern "C" lgt_status lgt_poll(lgt_server *s, uint64_t job_id, lgt_result *res, double *links_out) {
  if (!s) {
    lgt_set_error("lgt_poll: NULL server");
    return LGT_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) {
    lgt_set_error("lgt_poll: unknown job %llu", (unsigned long long)job_id);
    return LGT_ENOTFOUND;
  }
  Job *j = it->second;
  if (j->state != JOB_DONE) return LGT_EAGAIN;
  if (res) *res = j->res;
  if (links_out && !j->output.empty()) memcpy(links_out, j->output.data(), j->output.size() * sizeof(double));
  const lgt_status st = (lgt_status)j->res.status;
  s->jobs.erase(it);
  delete j;
  return st;
}

extern "C" lgt_status lgt_cancel(lgt_server *s, uint64_t job_id) {
  if (!s) {
    lgt_set_error("lgt_cancel: NULL server");
    return LGT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) {
    lgt_set_error("lgt_cancel: unknown job %llu", (unsigned long long)job_id);
    return LGT_ENOTFOUND;
  }
  it->second->cancel = true;
  s->cv.notify_all();
  return LGT_OK;
}

extern "C" lgt_status lgt_server_stats(lgt_server *s, uint64_t *jobs_done, uint64_t *jobs_live, size_t *bytes_in_use) {
  if (!s) {
    lgt_set_error("lgt_server_stats: NULL server");
    return LGT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (jobs_done) *jobs_done = s->done;
  if (jobs_live) *jobs_live = s->live.size();
  if (bytes_in_use) *bytes_in_use = s->used;
  return s->fatal == cudaSuccess ? LGT_OK : LGT_ECUDA;
}

extern "C" lgt_status lgt_server_counters(lgt_server *s, uint64_t *ticks, uint64_t *graph_launches,
                                          uint64_t *graph_captures, uint64_t *kernel_launches) {
  if (!s) {
    lgt_set_error("lgt_server_counters: NULL server");
    return LGT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticks) *ticks = s->ticks;
  if (graph_launches) *graph_launches = s->graph_launches;
  if (graph_captures) *graph_captures = s->graph_captures;
  if (kernel_launches) *kernel_launches = s->kernel_launches;
  return s->fatal == cudaSuccess ? LGT_OK : LGT_ECUDA;
}

extern "C" void lgt_server_destroy(lgt_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->jobs) delete kv.second;
  drop_graphs(s);
  if (s->d_sweep) cudaFree(s->d_sweep);
  if (s->h_sweep) cudaFreeHost(s->h_sweep);
  if (s->d_meas) cudaFree(s->d_meas);
  if (s->h_meas) cudaFreeHost(s->h_meas);
  if (s->d_fused) cudaFree(s->d_fused);
  if (s->h_fused) cudaFreeHost(s->h_fused);
  if (s->d_totals) cudaFree(s->d_totals);
  if (s->h_totals) cudaFreeHost(s->h_totals);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}
