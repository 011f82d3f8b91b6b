// lgt_kernels.cu -- single-lattice launches: half-sweep dispatch, exact
// measurement, fused-estimate finish, ingest/egress, the accumulated
// transformation G and the FP64 <-> FP32-pair conversion.  The sweep kernels
// themselves live in lgt_sweep_f32.cu and lgt_sweep_hi.cu (block-size
// variants, compiled in parallel), their bodies in lgt_sweep.cuh.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "lgt_device.cuh"
#include "lgt_internal.h"
#include "lgt_measure.cuh"
#include "lgt_pair.cuh"
#include "lgt_sweep.cuh"

namespace lgt {

static inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// fused-estimate slots per slice: one per 8 sites, plus the ragged last block
// of the widest launch (256 sites)
static int warps_per_slice(const Geom &g) { return ceil_div(g.vs_half, LGT_FUSED_GROUP) + 256 / LGT_FUSED_GROUP; }

size_t workspace_bytes(const Geom &g, int min_block) {
  const int gx = ceil_div(g.vs_half, min_block);
  size_t b = 0;
  b += sizeof(double2) * 2 * (size_t)g.nt * warps_per_slice(g);  // warp_part
  b += sizeof(double) * (size_t)g.nt * 2 + sizeof(unsigned);     // fused_slice, fused_counter
  b += sizeof(double) * TOT_N;                                    // fused_totals
  b += sizeof(double) * (size_t)g.nt * 2 * gx * MEAS_NV;   // meas_partial
  b += sizeof(double) * (size_t)g.nt * MEAS_NV;            // slice_sum
  b += sizeof(double) * (size_t)g.nt * 2;                  // slice_F, slice_theta
  b += sizeof(double) * TOT_N;                             // totals
  b += sizeof(unsigned) * ((size_t)g.nt + 1);              // counters
  b += (size_t)g.nt + sizeof(int);                         // active, err
  b += sizeof(unsigned) * ((size_t)g.nt + 2);              // stream_ctr
  b += sizeof(unsigned) * LGT_STREAM_MAX_HALF * (size_t)g.nt;  // stream_order
  return b + 16 * 21;                                      // alignment slack
}

static char *align16(char *p) { return (char *)(((uintptr_t)p + 15) & ~(uintptr_t)15); }

void workspace_carve(void *base, const Geom &g, int min_block, Workspace *w) {
  const int gx = ceil_div(g.vs_half, min_block);
  char *p = align16((char *)base);
  w->wps = warps_per_slice(g);
  w->warp_part = (double2 *)p;
  p = align16(p + sizeof(double2) * 2 * (size_t)g.nt * w->wps);
  w->fused_slice = (double *)p;
  p = align16(p + sizeof(double) * (size_t)g.nt * 2);
  w->fused_counter = (unsigned *)p;
  p = align16(p + sizeof(unsigned));
  w->fused_totals = (double *)p;
  p = align16(p + sizeof(double) * TOT_N);
  w->meas_partial = (double *)p;
  p = align16(p + sizeof(double) * (size_t)g.nt * 2 * gx * MEAS_NV);
  w->slice_sum = (double *)p;
  p = align16(p + sizeof(double) * (size_t)g.nt * MEAS_NV);
  w->slice_F = (double *)p;
  p = align16(p + sizeof(double) * (size_t)g.nt);
  w->slice_theta = (double *)p;
  p = align16(p + sizeof(double) * (size_t)g.nt);
  w->totals = (double *)p;
  p = align16(p + sizeof(double) * TOT_N);
  w->meas_counter = (unsigned *)p;
  p = align16(p + sizeof(unsigned) * (size_t)g.nt);
  w->glob_counter = (unsigned *)p;
  p = align16(p + sizeof(unsigned));
  w->err = (int *)p;
  p = align16(p + sizeof(int));
  w->stream_ctr = (unsigned *)p;
  p = align16(p + sizeof(unsigned) * ((size_t)g.nt + 2));
  w->stream_order = (unsigned *)p;
  p = align16(p + sizeof(unsigned) * LGT_STREAM_MAX_HALF * (size_t)g.nt);
  w->active = (uint8_t *)p;
}

void fill_sweep_args(SweepArgs *a, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                     unsigned long long sweep, int reunit, int use_mask) {
  a->g = g;
  a->links = links;
  a->G = G;
  a->aux = nullptr;
  a->loop = nullptr;
  a->active = use_mask ? w.active : nullptr;
  a->warp_part = w.warp_part;
  a->wps = w.wps;
  a->omega = c.omega;
  a->sr_thr = c.sr_thr;
  a->seed = c.seed;
  a->sweep = sweep;
  a->beta = c.beta;
  a->transform_temporal = c.transform_temporal;
  a->reunit = reunit;
  a->reunit_every = 0;
  a->count_base = 0;
  a->stream = w.stream_ctr;
  a->err = w.err;
  a->n_half = 1;
  static const int tiles = [] {
    const char *v = getenv("LGT_STREAM_TILES");
    const int n = v ? atoi(v) : 0;
    return n >= 1 && n <= 64 ? n : LGT_STREAM_TILES;
  }();
  a->stream_tiles = tiles;
  // LGT_SWEEP_SNAKE=0 in the environment: every half-sweep in forward order
  static const int snake = [] {
    const char *v = getenv("LGT_SWEEP_SNAKE");
    return (v && v[0] == '0') ? 0 : 1;
  }();
  a->snake = snake;
  a->stream_wait_ns = c.stream_wait_ns ? c.stream_wait_ns : LGT_STREAM_WAIT_NS;
  a->stream_skip = c.stream_skip;
  a->stream_order = nullptr;  // half-sweep after half-sweep
  a->stream_shift = 1;
  a->t_offset = c.t_offset;
  a->t_first = c.t_first;
  a->t_count = c.t_count > 0 ? c.t_count : g.nt;
}

// SMs of the current device, looked up once per device ordinal
static int device_sms() {
  static int sms_of[64];
  int dev = 0;
  cudaGetDevice(&dev);
  int &sms = sms_of[dev & 63];
  if (!sms) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Within a run of half-sweeps every launch after the first, whose predecessor in
// the stream is then a sweep kernel, carries programmatic stream serialisation
// (configurations with blocks per site tile; not the persistent ones)
// (the kernels begin with griddepcontrol.wait): the next half-sweep's blocks are
// scheduled while the previous one drains.  LGT_SWEEP_PDL=0 in the
// environment: plain launches only.
static bool use_pdl() {
  static const bool on = [] {
    const char *v = getenv("LGT_SWEEP_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}

static cudaError_t launch_fn(sweep_fn fn, dim3 grid, int block, int smem, cudaStream_t st, const SweepArgs &a,
                             int parity, bool pdl) {
  if (!pdl || !use_pdl()) {
    fn<<<grid, block, smem, st>>>(a, parity);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = dim3(block);
  lc.dynamicSmemBytes = (size_t)smem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, fn, a, parity);
}

// one launch of a sweep kernel (n_half > 1: streaming configuration only)
static cudaError_t launch_sweep_kernel(sweep_fn fn, int cfg, const Geom &g, SweepArgs &a, int parity, cudaStream_t st,
                                       bool pdl = false) {
  const int block = lgt_cfg_threads(cfg);
  if (lgt_cfg_pipe(cfg) || lgt_cfg_stream(cfg)) {
    // persistent: lgt_cfg_minblocks blocks per SM over the (half-sweep, slice, tile) list
    const int smem = LGT_PIPE_SMEM_PER_THREAD * block;
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)ceil_div(g.vs_half, block) * a.t_count * a.n_half;
    const long long cap = (long long)device_sms() * lgt_cfg_minblocks(cfg);
    const int blocks = (int)(tiles < cap ? tiles : cap);
    if (lgt_cfg_stream(cfg)) {  // counters start at zero in every launch
      e = cudaMemsetAsync(a.stream, 0, sizeof(unsigned) * ((size_t)g.nt + 2), st);
      if (e != cudaSuccess) return e;
    }
    // (persistent blocks fill the SMs' shared memory, so the successor's blocks
    // could only be placed as they exit: measured a little slower, left plain)
    return launch_fn(fn, dim3(blocks), block, smem, st, a, parity & 1, false);
  }
  int smem = 0;
  if (lgt_cfg_staged(cfg)) {  // one tile per block, its sites' operands staged in shared memory
    smem = 16 * lgt_cfg_stage_chunks(cfg) * block;
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return launch_fn(fn, dim3(ceil_div(g.vs_half, lgt_cfg_sites(cfg)), a.t_count), block, smem, st, a, parity & 1, pdl);
}

static sweep_fn pick_sweep(int fmt, const SweepCfg &c, int cfg) {
  return (fmt == FMT_F32_18 || fmt == FMT_F32_12) ? pick_sweep_f32(fmt, c.gauge, c.algo, cfg)
                                                  : pick_sweep_hi(fmt, c.gauge, c.algo, cfg);
}

static cudaError_t half_sweep(int fmt, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                              int parity, unsigned long long sweep, int reunit, int use_mask, int cfg,
                              cudaStream_t st, const void *aux, const LoopState *loop, int reunit_every, bool pdl) {
  sweep_fn fn = pick_sweep(fmt, c, cfg);
  if (!fn || !lgt_cfg_supported_gauge(fmt, c.gauge, cfg)) return cudaErrorInvalidValue;
  SweepArgs a{};
  fill_sweep_args(&a, g, links, G, w, c, sweep, reunit, use_mask);
  a.aux = aux;
  a.loop = loop;
  a.reunit_every = reunit_every;
  if (lgt_cfg_stream(cfg) && loop) a.count_base = 0;  // the loop's count is added on the device
  return launch_sweep_kernel(fn, cfg, g, a, parity, st, pdl);
}

cudaError_t launch_half_sweep(int fmt, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                              int parity, unsigned long long sweep, int reunit, int use_mask, int cfg,
                              cudaStream_t st, const void *aux, const LoopState *loop, int reunit_every) {
  return half_sweep(fmt, g, links, G, w, c, parity, sweep, reunit, use_mask, cfg, st, aux, loop, reunit_every, false);
}

// The rolling band's table: slot stream_band_rank(h, k) holds (h, k).
__global__ void k_stream_order(unsigned *order, int nt, int n_half, int D) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nt * n_half) return;
  const int h = idx / nt, k = idx - h * nt;
  order[stream_band_rank(h, k, nt, n_half, D)] = ((unsigned)h << 16) | (unsigned)k;
}

// Shape of the rolling band on nt slices: about B half-sweeps at once (D =
// ceil(nt / B) waves apart), G slices apart (S = D - G); B and G from
// LGT_STREAM_BAND="B,G" when set, read at each launch.
static void band_shape(int nt, int *D, int *S) {
  int B = LGT_BAND_ACTIVE, G = LGT_BAND_GAP;
  if (const char *v = getenv("LGT_STREAM_BAND")) {
    int b = 0, gap = 0;
    if (sscanf(v, "%d,%d", &b, &gap) == 2 && b >= 1 && b <= 64 && gap >= 1 && gap <= 64) B = b, G = gap;
  }
  int d = ceil_div(nt, B);
  if (d < G + 1) d = G + 1;  // 1 <= S <= D - 1
  *D = d;
  *S = d - G;
}
static int band_tiles() {
  const char *v = getenv("LGT_STREAM_BAND_TILES");
  const int n = v ? atoi(v) : 0;
  return n >= 1 && n <= 64 ? n : LGT_BAND_TILES;
}

cudaError_t launch_half_sweeps(int fmt, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                               int p0, int n_half, unsigned long long sweep0, long long count_base, int reunit_every,
                               int use_mask, int cfg, cudaStream_t st, const void *aux, const LoopState *loop,
                               int *launches) {
  if (launches) *launches = 0;
  if (n_half <= 0) return cudaSuccess;
  if (!lgt_cfg_stream(cfg)) {
    for (int h = 0; h < n_half; h++) {
      const int s = (p0 + h) >> 1;
      cudaError_t e;
      if (loop) {  // sweep number and schedule from the loop state (sweep0 + s: offset in the chunk)
        e = half_sweep(fmt, g, links, G, w, c, p0 + h, sweep0 + s, 0, use_mask, cfg, st, aux, loop, reunit_every,
                       h > 0);
      } else {
        const int reunit = reunit_every > 0 && ((count_base + s + 1) % reunit_every) == 0;
        e = half_sweep(fmt, g, links, G, w, c, p0 + h, sweep0 + s, reunit, use_mask, cfg, st, aux, nullptr, 0, h > 0);
      }
      if (e != cudaSuccess) return e;
      if (launches) ++*launches;
    }
    return cudaSuccess;
  }
  sweep_fn fn = pick_sweep(fmt, c, cfg);
  if (!fn || !lgt_cfg_supported_gauge(fmt, c.gauge, cfg)) return cudaErrorInvalidValue;
  int band_d = 0, band_s = 1, band_n = 0;  // rolling band: wave stagger, slice shift, table built for band_n
  const bool band = lgt_cfg_band(cfg) && g.nt <= 0xffff;  // the table packs k in 16 bits (else configuration 10's order)
  if (band) band_shape(g.nt, &band_d, &band_s);
  // launches of at most LGT_STREAM_MAX_HALF half-sweeps (and 2^30 tiles: the
  // ticket and slice counters are 32-bit)
  const long long tiles_half = (long long)ceil_div(g.vs_half, lgt_cfg_threads(cfg)) * g.nt;
  long long per_launch = (1ll << 30) / (tiles_half > 0 ? tiles_half : 1);
  if (per_launch > LGT_STREAM_MAX_HALF) per_launch = LGT_STREAM_MAX_HALF;
  if (per_launch < 1) per_launch = 1;
  for (int h0 = 0; h0 < n_half; h0 += (int)per_launch) {
    const int n = (int)((n_half - h0) < per_launch ? (n_half - h0) : per_launch);
    const int p = (p0 + h0) & 1;
    const long long s0 = (p0 + h0 - p) / 2;  // sweeps of the run before this launch's first
    SweepArgs a{};
    fill_sweep_args(&a, g, links, G, w, c, sweep0 + (unsigned long long)s0, 0, use_mask);
    a.aux = aux;
    a.loop = loop;
    a.reunit_every = reunit_every;
    a.count_base = loop ? 0 : count_base + s0;
    a.n_half = n;
    if (band) {
      a.stream_tiles = band_tiles();
      a.stream_shift = band_s;
      a.stream_order = w.stream_order;
      if (n != band_n) {  // the table of this launch's n half-sweeps (stream-ordered after the last reader)
        const int pairs = n * g.nt;
        k_stream_order<<<ceil_div(pairs, 256), 256, 0, st>>>(w.stream_order, g.nt, n, band_d);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        band_n = n;
      }
    }
    cudaError_t e = launch_sweep_kernel(fn, cfg, g, a, p, st);
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
  }
  return cudaSuccess;
}

template <int FMT>
__global__ void __launch_bounds__(256) k_measure(MeasArgs a) {
  measure_body<FMT>(a, blockIdx.y, blockIdx.z, blockIdx.x, gridDim.x);
}

void fill_meas_args(MeasArgs *a, const Geom &g, const void *links, const Workspace &w, int with_plaq,
                    double coulomb_target) {
  a->g = g;
  a->links = links;
  a->partial = w.meas_partial;
  a->counter = w.meas_counter;
  a->glob = w.glob_counter;
  a->slice_sum = w.slice_sum;
  a->slice_F = w.slice_F;
  a->slice_theta = w.slice_theta;
  a->totals = w.totals;
  a->active = w.active;
  a->coulomb_target = coulomb_target;
  a->with_plaq = with_plaq;
  a->mag = 0;  // the maximally Abelian gauge's measurement is asked for explicitly (launch_measure)
}

cudaError_t launch_measure(int fmt, const Geom &g, const void *links, const Workspace &w, int with_plaq,
                           double coulomb_target, int block, cudaStream_t st, int mag) {
  MeasArgs a{};
  fill_meas_args(&a, g, links, w, with_plaq, coulomb_target);
  a.mag = mag;
  dim3 grid(ceil_div(g.vs_half, block), g.nt, 2);
  if (fmt == FMT_F64) k_measure<FMT_F64><<<grid, block, 0, st>>>(a);
  else if (fmt == FMT_F32_18) k_measure<FMT_F32_18><<<grid, block, 0, st>>>(a);
  else if (fmt == FMT_F32_12) k_measure<FMT_F32_12><<<grid, block, 0, st>>>(a);
  else if (fmt == FMT_PAIR) k_measure<FMT_PAIR><<<grid, block, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ------------------------------------------------------- layout / ingest
// thread -> (parity, direction, within-parity index); lexicographic site
__device__ __forceinline__ bool link_of_thread(const Geom &g, long long gid, int &p, int &mu, int &i, Coords &c,
                                               long long &lex) {
  if (gid >= (long long)g.vh * 8) return false;
  i = (int)(gid % g.vh);
  const int pm = (int)(gid / g.vh);
  p = pm >> 2;
  mu = pm & 3;
  const int t = i / g.vs_half;
  c = coords_in_slice(g, p, t, i - t * g.vs_half);
  lex = (long long)c.x1 + (long long)g.n1 * (c.x2 + (long long)g.n2 * (c.x3 + (long long)g.n3 * c.t));
  return true;
}

template <int FMT>
__global__ void k_ingest(Geom g, const double *aos, void *soa, int *err) {
  int p, mu, i;
  Coords c;
  long long lex;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!link_of_thread(g, gid, p, mu, i, c, lex)) return;
  const double *src = aos + ((size_t)lex * 4 + mu) * 18;
  double u[18];
  bool finite = true;
#pragma unroll
  for (int k = 0; k < 18; k++) {
    u[k] = src[k];
    finite = finite && isfinite(u[k]);
  }
  // SU(3) check: |U^dagger U - 1|_max and |det U - 1|
  double worst = 0.0;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 3; k++) {  // sum_k conj(U_ka) U_kb
        re += u[LGT_RE(k, a)] * u[LGT_RE(k, b)] + u[LGT_IM(k, a)] * u[LGT_IM(k, b)];
        im += u[LGT_RE(k, a)] * u[LGT_IM(k, b)] - u[LGT_IM(k, a)] * u[LGT_RE(k, b)];
      }
      re -= (a == b) ? 1.0 : 0.0;
      worst = fmax(worst, fmax(fabs(re), fabs(im)));
    }
  double dre = 0.0, dim = 0.0;
#pragma unroll
  for (int cc = 0; cc < 3; cc++) {
    const int a1 = (cc + 1) % 3, b1 = (cc + 2) % 3;
    const double mre = u[LGT_RE(1, a1)] * u[LGT_RE(2, b1)] - u[LGT_IM(1, a1)] * u[LGT_IM(2, b1)] -
                       (u[LGT_RE(1, b1)] * u[LGT_RE(2, a1)] - u[LGT_IM(1, b1)] * u[LGT_IM(2, a1)]);
    const double mim = u[LGT_RE(1, a1)] * u[LGT_IM(2, b1)] + u[LGT_IM(1, a1)] * u[LGT_RE(2, b1)] -
                       (u[LGT_RE(1, b1)] * u[LGT_IM(2, a1)] + u[LGT_IM(1, b1)] * u[LGT_RE(2, a1)]);
    dre += u[LGT_RE(0, cc)] * mre - u[LGT_IM(0, cc)] * mim;
    dim += u[LGT_RE(0, cc)] * mim + u[LGT_IM(0, cc)] * mre;
  }
  worst = fmax(worst, fmax(fabs(dre - 1.0), fabs(dim)));
  if (!finite || !(worst < 1e-10)) atomicOr(err, 1);
  typedef typename LinkIO<FMT>::real R;
  R r[18];
#pragma unroll
  for (int k = 0; k < 18; k++) r[k] = (R)u[k];
  LinkIO<FMT>::store(soa, g.vh, p, mu, i, r);
}

template <int FMT>
__global__ void k_egress(Geom g, const void *soa, double *aos) {
  int p, mu, i;
  Coords c;
  long long lex;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!link_of_thread(g, gid, p, mu, i, c, lex)) return;
  double u[18];
  load_d<FMT>(soa, g.vh, p, mu, i, u);
  double *dst = aos + ((size_t)lex * 4 + mu) * 18;
#pragma unroll
  for (int k = 0; k < 18; k++) dst[k] = u[k];
}

cudaError_t launch_ingest(int fmt, const Geom &g, const double *aos, void *soa, int *err, cudaStream_t st) {
  const long long n = (long long)g.vh * 8;
  const int blk = 256;
  const unsigned grid = (unsigned)((n + blk - 1) / blk);
  if (fmt == FMT_F64) k_ingest<FMT_F64><<<grid, blk, 0, st>>>(g, aos, soa, err);
  else if (fmt == FMT_F32_18) k_ingest<FMT_F32_18><<<grid, blk, 0, st>>>(g, aos, soa, err);
  else if (fmt == FMT_F32_12) k_ingest<FMT_F32_12><<<grid, blk, 0, st>>>(g, aos, soa, err);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_egress(int fmt, const Geom &g, const void *soa, double *aos, cudaStream_t st) {
  const long long n = (long long)g.vh * 8;
  const int blk = 256;
  const unsigned grid = (unsigned)((n + blk - 1) / blk);
  if (fmt == FMT_F64) k_egress<FMT_F64><<<grid, blk, 0, st>>>(g, soa, aos);
  else if (fmt == FMT_F32_18) k_egress<FMT_F32_18><<<grid, blk, 0, st>>>(g, soa, aos);
  else if (fmt == FMT_F32_12) k_egress<FMT_F32_12><<<grid, blk, 0, st>>>(g, soa, aos);
  else if (fmt == FMT_PAIR) k_egress<FMT_PAIR><<<grid, blk, 0, st>>>(g, soa, aos);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ------------------------------------------------ accumulated transformation
__global__ void k_g_identity(Geom g, void *G) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)g.vh * 2) return;
  const int p = (int)(gid / g.vh), i = (int)(gid % g.vh);
  float m[18];
  mat_zero(m);
  m[LGT_RE(0, 0)] = m[LGT_RE(1, 1)] = m[LGT_RE(2, 2)] = 1.0f;
  GIO::store(G, g.vh, p, i, m);
}

cudaError_t launch_g_identity(const Geom &g, void *G, cudaStream_t st) {
  const long long n = (long long)g.vh * 2;
  const int blk = 256;
  k_g_identity<<<(unsigned)((n + blk - 1) / blk), blk, 0, st>>>(g, G);
  return cudaGetLastError();
}

__device__ __forceinline__ void load_G_fp64(const void *G, int vh, int p, int i, double m[18]) {
  float f[18];
  GIO::load(G, vh, p, i, f);
#pragma unroll
  for (int k = 0; k < 18; k++) m[k] = (double)f[k];
  reunitarise(m);
}

// G = 1 + D of the anchored polish in FP64 (pairs widened, row 2 rebuilt in
// FP64, rows orthonormalised: unitary to FP64 rounding)
__device__ __forceinline__ void load_G_from_D(const void *D, int vh, int p, int i, double m[18]) {
  f2 d[18];
  DIO::load_pair(D, vh, p, i, d);
#pragma unroll
  for (int k = 0; k < 12; k++) m[k] = (double)d[k].hi + (double)d[k].lo;
  m[LGT_RE(0, 0)] += 1.0;
  m[LGT_RE(1, 1)] += 1.0;
  reunitarise(m);
}

// U_mu(x) <- G(x) U_mu(x) G(x+mu)^+ in FP64; SRC 0: G of the bulk phase
// (FP32), SRC 1: G = 1 + D of the anchored polish (pairs)
template <int SRC>
__global__ void k_apply_G(Geom g, const void *G, const void *u_in, void *u_out, double *aos_out, int skip_temporal) {
  int p, mu, i;
  Coords c;
  long long lex;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!link_of_thread(g, gid, p, mu, i, c, lex)) return;
  double u[18], r[18], gx[18], gy[18], tmp[18];
  LinkIO<FMT_F64>::load(u_in, g.vh, p, mu, i, u);
  if (skip_temporal && mu == 0) {
#pragma unroll
    for (int k = 0; k < 18; k++) r[k] = u[k];
  } else {
    if (SRC == 0) {
      load_G_fp64(G, g.vh, p, i, gx);
      load_G_fp64(G, g.vh, p ^ 1, cb_shift(g, c, mu, +1), gy);
    } else {
      load_G_from_D(G, g.vh, p, i, gx);
      load_G_from_D(G, g.vh, p ^ 1, cb_shift(g, c, mu, +1), gy);
    }
    mat_mul(gx, u, tmp);
    mat_mul_dag(tmp, gy, r);
  }
  if (aos_out) {
    double *dst = aos_out + ((size_t)lex * 4 + mu) * 18;
#pragma unroll
    for (int k = 0; k < 18; k++) dst[k] = r[k];
  } else {
    LinkIO<FMT_F64>::store(u_out, g.vh, p, mu, i, r);
  }
}

cudaError_t launch_apply_G(const Geom &g, const void *G, const void *u64_in, void *u64_out, double *aos_out,
                           int skip_temporal, cudaStream_t st) {
  const long long n = (long long)g.vh * 8;
  const int blk = 128;
  k_apply_G<0><<<(unsigned)((n + blk - 1) / blk), blk, 0, st>>>(g, G, u64_in, u64_out, aos_out, skip_temporal);
  return cudaGetLastError();
}

cudaError_t launch_apply_D(const Geom &g, const void *D, const void *u64_in, void *u64_out, double *aos_out,
                           int skip_temporal, cudaStream_t st) {
  const long long n = (long long)g.vh * 8;
  const int blk = 128;
  k_apply_G<1><<<(unsigned)((n + blk - 1) / blk), blk, 0, st>>>(g, D, u64_in, u64_out, aos_out, skip_temporal);
  return cudaGetLastError();
}

// ------------------------------------------------ anchored polish set-up
// For every site of either parity: K0(x) = sum_{mu >= mu0} U_mu(x) + U_mu(x-mu)^+
// in FP64, stored as FP32 pairs (hi = fl32(v), lo = fl32(v - hi)); the FP32-12
// copy of the site's forward links; D(x) = 0.
__global__ void k_anchor_setup(Geom g, const void *u64, void *u32, void *K0, void *D, int mu0) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)g.vh * 2) return;
  const int p = (int)(gid / g.vh), i = (int)(gid % g.vh);
  const int t = i / g.vs_half;
  const Coords c = coords_in_slice(g, p, t, i - t * g.vs_half);
  double K[18];
  mat_zero(K);
  for (int mu = 0; mu < 4; mu++) {
    double u[18];
    float uf[18];
    LinkIO<FMT_F64>::load(u64, g.vh, p, mu, i, u);
#pragma unroll
    for (int k = 0; k < 18; k++) uf[k] = __double2float_rn(u[k]);
    LinkIO<FMT_F32_12>::store(u32, g.vh, p, mu, i, uf);
    if (mu >= mu0) {
      acc_add(K, u);
      LinkIO<FMT_F64>::load(u64, g.vh, p ^ 1, mu, cb_shift(g, c, mu, -1), u);
      acc_add_dag(K, u);
    }
  }
  f2 k2[18], z[18];
#pragma unroll
  for (int k = 0; k < 18; k++) {
    const float hi = __double2float_rn(K[k]);
    k2[k] = {hi, __double2float_rn(K[k] - (double)hi)};
    z[k] = {0.0f, 0.0f};
  }
  K0IO::store(K0, g.vh, p, i, k2);
  DIO::store_pair(D, g.vh, p, i, z);
}

cudaError_t launch_anchor_setup(const Geom &g, const void *u64, void *u32, void *K0, void *D, int gauge,
                                cudaStream_t st) {
  const long long n = (long long)g.vh * 2;
  const int blk = 128;
  k_anchor_setup<<<(unsigned)((n + blk - 1) / blk), blk, 0, st>>>(g, u64, u32, K0, D,
                                                                 gauge == GAUGE_COULOMB ? 1 : 0);
  return cudaGetLastError();
}

// --------------------------------------------- unit links (autotuning runs)
template <int FMT>
__global__ void k_fill_unit(Geom g, void *soa) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)g.vh * 8) return;
  const int i = (int)(gid % g.vh), pm = (int)(gid / g.vh);
  typedef typename LinkIO<FMT>::real R;
  R m[18];
  mat_zero(m);
  m[LGT_RE(0, 0)] = m[LGT_RE(1, 1)] = m[LGT_RE(2, 2)] = R(1);
  LinkIO<FMT>::store(soa, g.vh, pm >> 2, pm & 3, i, m);
}

__global__ void k_fill_unit_pair(Geom g, void *soa) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)g.vh * 8) return;
  const int i = (int)(gid % g.vh), pm = (int)(gid / g.vh);
  f2 m[18];
  for (int e = 0; e < 18; e++) m[e] = f2{0.0f, 0.0f};
  m[LGT_RE(0, 0)] = m[LGT_RE(1, 1)] = m[LGT_RE(2, 2)] = f2{1.0f, 0.0f};
  LinkIO<FMT_PAIR>::store(soa, g.vh, pm >> 2, pm & 3, i, m);
}

cudaError_t launch_fill_unit(int fmt, const Geom &g, void *soa, cudaStream_t st) {
  const long long n = (long long)g.vh * 8;
  const int blk = 256;
  const unsigned grid = (unsigned)((n + blk - 1) / blk);
  if (fmt == FMT_F64) k_fill_unit<FMT_F64><<<grid, blk, 0, st>>>(g, soa);
  else if (fmt == FMT_F32_18) k_fill_unit<FMT_F32_18><<<grid, blk, 0, st>>>(g, soa);
  else if (fmt == FMT_F32_12) k_fill_unit<FMT_F32_12><<<grid, blk, 0, st>>>(g, soa);
  else if (fmt == FMT_PAIR) k_fill_unit_pair<<<grid, blk, 0, st>>>(g, soa);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ------------------------------------------- FP64 <-> FP32-pair, in place
// Each thread owns one 16-byte element chunk: (re, im) as double2 or
// (hi_re, lo_re, hi_im, lo_im) as float4 at the same address.
__global__ void k_f64_to_pair(double2 *u, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double2 v = u[k];
  const float hr = __double2float_rn(v.x), hi = __double2float_rn(v.y);
  const float lr = __double2float_rn(v.x - (double)hr), li = __double2float_rn(v.y - (double)hi);
  reinterpret_cast<float4 *>(u)[k] = make_float4(hr, lr, hi, li);
}

__global__ void k_pair_to_f64(double2 *u, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float4 v = reinterpret_cast<const float4 *>(u)[k];
  u[k] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

cudaError_t launch_convert_pair(const Geom &g, void *u, int to_pair, cudaStream_t st) {
  const long long n = (long long)g.vh * 2 * 4 * 9;
  const int blk = 256;
  const unsigned grid = (unsigned)((n + blk - 1) / blk);
  if (to_pair) k_f64_to_pair<<<grid, blk, 0, st>>>(reinterpret_cast<double2 *>(u), n);
  else k_pair_to_f64<<<grid, blk, 0, st>>>(reinterpret_cast<double2 *>(u), n);
  return cudaGetLastError();
}


// ------------------------------------------------- fused estimate, finish
void fill_fused_args(FusedArgs *a, const Geom &g, const Workspace &w, int gauge, int sweep_sites,
                     double coulomb_target) {
  a->g = g;
  a->warp_part = w.warp_part;
  a->wps = w.wps;
  a->nw = ceil_div(g.vs_half, sweep_sites) * (sweep_sites / LGT_FUSED_GROUP);
  a->gauge = gauge;
  a->slice = w.fused_slice;
  a->counter = w.fused_counter;
  a->totals = w.fused_totals;
  a->active = w.active;
  a->coulomb_target = coulomb_target;
}

__global__ void __launch_bounds__(256) k_fused_finish(FusedArgs a) { fused_finish_body(a, blockIdx.x); }

cudaError_t launch_fused_finish(const Geom &g, const Workspace &w, int gauge, int sweep_sites, double coulomb_target,
                                cudaStream_t st) {
  FusedArgs a{};
  fill_fused_args(&a, g, w, gauge, sweep_sites, coulomb_target);
  k_fused_finish<<<g.nt, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------ device loop decision
// After a chunk of k sweeps and its fused estimate: advance the loop's counters
// and decide, with the host driver's rules, whether another chunk follows.
__global__ void k_loop_decide(LoopState *L, const double *tot, int gauge, int k, int vs_half,
                              cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double theta = gauge == GAUGE_COULOMB ? tot[TOT_THETA_COULOMB_MAX] : tot[TOT_THETA_LANDAU];
  L->site_updates += 2LL * k * (long long)vs_half * L->active;
  L->active = (int)tot[TOT_ACTIVE_SLICES];
  L->sweep += (unsigned long long)k;
  L->count += k;
  L->remaining -= k;
  L->iters += 1;
  L->theta = theta;
  if (L->omega_switch && theta < L->theta_omega) {  // omega schedule: the later sweeps at omega_late
    L->omega = L->omega_late;
    L->omega_switch = 0;
  }
  bool go = theta >= L->target;
  if (L->bulk) {
    if (theta < L->best) {
      L->best = theta;
      L->stall = 0;
    } else {
      L->stall = theta < LGT_STALL_CEILING ? L->stall + 1 : 0;
    }
    go = go && L->stall < LGT_STALL_CHECKS;
  }
  // only whole chunks run on the device; the host takes a shorter last chunk
  go = go && L->remaining >= k && L->iters < L->max_iters;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_slice_mask(uint8_t *active, int nt, int lo, int hi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nt) active[t] = (t >= lo && t < hi) ? 1 : 0;
}

cudaError_t launch_slice_mask(uint8_t *active, int nt, int lo, int hi, cudaStream_t st) {
  k_slice_mask<<<(nt + 127) / 128, 128, 0, st>>>(active, nt, lo, hi);
  return cudaGetLastError();
}

__global__ void k_fill_unit_aos(double *aos, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double *u = aos + k * 18;
#pragma unroll
  for (int e = 0; e < 18; e++) u[e] = (e == 0 || e == 8 || e == 16) ? 1.0 : 0.0;
}

cudaError_t launch_fill_unit_aos(double *aos, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fill_unit_aos<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(aos, n);
  return cudaGetLastError();
}

cudaError_t launch_loop_decide(LoopState *L, const double *fused_totals, int gauge, int k, int vs_half,
                               cudaGraphConditionalHandle h, cudaStream_t st) {
  k_loop_decide<<<1, 32, 0, st>>>(L, fused_totals, gauge, k, vs_half, h);
  return cudaGetLastError();
}

}  // namespace lgt
