// lgt_kernels.cu -- the sweep, measurement and layout kernels for sm_103a.
//
// Half-sweep (Sec. 3 and Sec. 4 of Schroeck & Vogt): one thread per site of
// the active parity.  The thread gathers K(x) from the 4 forward links of its
// site and the 4 backward links U_mu(x-mu) (which belong to sites of the other
// parity), runs the Cabibbo-Marinari local update, and writes g U_mu(x) and
// U_mu(x-mu) g^dagger back in place.  Sites of one parity touch disjoint links,
// so the launch is race-free.  While K(x) is in registers the thread also
// adds Re tr K and tr[Delta Delta^dagger] to a deterministic per-slice sum
// (the fused estimate of F and theta).
//
// FP32 formats keep all 8 links in registers between the gather and the
// write-back (each link is read once and written once per half-sweep, no
// reuse).  FP64 links are 2x larger and FP64 arithmetic is the bottleneck on
// this part, so the FP64 kernel gathers K streaming and re-reads each link
// for the write-back (an L2 hit).
#include <cuda_runtime.h>
#include <stdint.h>

#include "lgt_device.cuh"
#include "lgt_internal.h"
#include "lgt_pair.cuh"

namespace lgt {

static inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

static int warps_per_slice(const Geom &g) { return ceil_div(g.vs_half, 32) + 8; }

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
  return b + 16 * 20;                                      // alignment slack
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
  w->active = (uint8_t *)p;
}

// ----------------------------------------------------------------- sweeps


// The fused estimate: each warp's sum of (Re tr K, tr Delta^2) over its sites
// goes to its own slot (xor butterfly: fixed order; no block barrier, no
// atomics); k_fused_finish reduces the slots when an estimate is wanted.
template <typename T>
__device__ __forceinline__ void fused_store(const SweepArgs &a, int p, int t, int bx, T acc[2]) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  if ((threadIdx.x & 31) == 0) {
    const int w = bx * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    a.warp_part[((size_t)p * a.g.nt + t) * a.wps + w] = make_double2((double)acc[0], (double)acc[1]);
  }
}

__device__ __forceinline__ uint4 sr_draws(const SweepArgs &a, const Coords &c) {
  const unsigned long long lex =
      (unsigned long long)c.x1 +
      (unsigned long long)a.g.n1 * ((unsigned long long)c.x2 +
                                    (unsigned long long)a.g.n2 * ((unsigned long long)c.x3 +
                                                                  (unsigned long long)a.g.n3 * (unsigned long long)c.t));
  const uint4 ctr = make_uint4((uint32_t)lex, (uint32_t)(lex >> 32), (uint32_t)a.sweep, LGT_SR_TAG);
  const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
  return philox4x32_10(ctr, key);
}

// FP32 link formats: all links of the site in registers.  12-real links stay
// compressed (rows 0, 1) and row 2 is rebuilt where it is needed.
template <int FMT, int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_f32(const SweepArgs &a, int p, int t, int bx, int nbx) {
  typedef LinkIO<FMT> IO;
  if (a.active && !a.active[t]) return;  // whole block belongs to one slice
  const int j = bx * blockDim.x + threadIdx.x;
  float acc[2] = {0.0f, 0.0f};
  if (j < a.g.vs_half) {
    constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    float uf[4][18], ub[4][18];
    int nb[4];
#pragma unroll
    for (int mu = MU0; mu < 4; mu++) {
      nb[mu] = cb_shift(a.g, c, mu, -1);
      IO::load_raw(a.links, a.g.vh, p, mu, i, uf[mu]);
      IO::load_raw(a.links, a.g.vh, q, mu, nb[mu], ub[mu]);
    }
    float W[18];
    mat_zero(W);
#pragma unroll
    for (int mu = MU0; mu < 4; mu++) {
      if (IO::kCompressed) {
        float full[18];
#pragma unroll
        for (int e = 0; e < 18; e++) full[e] = uf[mu][e];
        rebuild_row2(full);
        acc_add(W, full);
#pragma unroll
        for (int e = 0; e < 18; e++) full[e] = ub[mu][e];
        rebuild_row2(full);
        acc_add_dag(W, full);
      } else {
        acc_add(W, uf[mu]);
        acc_add_dag(W, ub[mu]);
      }
    }
    violation_of_K(W, acc[0], acc[1]);
    uint4 draws = make_uint4(0, 0, 0, 0);
    if (ALGO == ALGO_SR) draws = sr_draws(a, c);
    float gm[18];
    local_update<float, ALGO>(W, gm, (float)a.omega, a.sr_thr, draws);
#pragma unroll
    for (int mu = MU0; mu < 4; mu++) {
      float r[18];
      if (IO::kCompressed) rebuild_row2(uf[mu]);  // g U needs row 2 of U
      mat_mul(gm, uf[mu], r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, p, mu, i, r);
      mat_mul_dag(ub[mu], gm, r);  // rows 0, 1 of U g^dagger need rows 0, 1 of U only
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, q, mu, nb[mu], r);
    }
    if (GAUGE == GAUGE_COULOMB && a.transform_temporal) {
      const int nb0 = cb_shift(a.g, c, 0, -1);
      float u[18], r[18];
      IO::load(a.links, a.g.vh, p, 0, i, u);
      mat_mul(gm, u, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, p, 0, i, r);
      IO::load(a.links, a.g.vh, q, 0, nb0, u);
      mat_mul_dag(u, gm, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, q, 0, nb0, r);
    }
    if (a.G) {
      float gx[18], r[18];
      GIO::load(a.G, a.g.vh, p, i, gx);
      mat_mul(gm, gx, r);
      if (a.reunit) reunitarise(r);
      GIO::store(a.G, a.g.vh, p, i, r);
    }
  }
  fused_store<float>(a, p, t, bx, acc);
}

template <int FMT, int GAUGE, int ALGO>
__global__ void __launch_bounds__(256) k_sweep_f32(SweepArgs a, int p) {
  sweep_body_f32<FMT, GAUGE, ALGO>(a, p, blockIdx.y, blockIdx.x, gridDim.x);
}

// FP64: K gathered streaming, links re-read for the write-back.
template <int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_f64(const SweepArgs &a, int p, int t, int bx, int nbx) {
  typedef LinkIO<FMT_F64> IO;
  if (a.active && !a.active[t]) return;
  const int j = bx * blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (j < a.g.vs_half) {
    constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    int nb[4];
    double W[18];
    mat_zero(W);
#pragma unroll
    for (int mu = MU0; mu < 4; mu++) {
      double u[18];
      nb[mu] = cb_shift(a.g, c, mu, -1);
      IO::load(a.links, a.g.vh, p, mu, i, u);
      acc_add(W, u);
      IO::load(a.links, a.g.vh, q, mu, nb[mu], u);
      acc_add_dag(W, u);
    }
    violation_of_K(W, acc[0], acc[1]);
    uint4 draws = make_uint4(0, 0, 0, 0);
    if (ALGO == ALGO_SR) draws = sr_draws(a, c);
    double gm[18];
    local_update<double, ALGO>(W, gm, a.omega, a.sr_thr, draws);
    const int mu_lo = (GAUGE == GAUGE_COULOMB && a.transform_temporal) ? 0 : MU0;
    for (int mu = mu_lo; mu < 4; mu++) {
      const int nbm = mu < MU0 ? cb_shift(a.g, c, 0, -1) : nb[mu];
      double u[18], r[18];
      IO::load(a.links, a.g.vh, p, mu, i, u);
      mat_mul(gm, u, r);
      IO::store(a.links, a.g.vh, p, mu, i, r);
      IO::load(a.links, a.g.vh, q, mu, nbm, u);
      mat_mul_dag(u, gm, r);
      IO::store(a.links, a.g.vh, q, mu, nbm, r);
    }
  }
  fused_store<double>(a, p, t, bx, acc);
}

template <int GAUGE, int ALGO>
__global__ void __launch_bounds__(256) k_sweep_f64(SweepArgs a, int p) {
  sweep_body_f64<GAUGE, ALGO>(a, p, blockIdx.y, blockIdx.x, gridDim.x);
}

// FP32-pair polishing sweep (FMT_PAIR storage): K(x) in pair arithmetic, the
// rotation angles in FP32, g = R2 R1 R0 formed in pair precision (unitary to
// ~2^-48) and applied to every link as U + delta U / U + U delta^dagger in
// pair arithmetic (see lgt_pair.cuh).  Links are re-read for the write-back.
// The loops over directions are not unrolled: the body is instruction-bound
// and a compact loop keeps it in the instruction cache.
template <int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_pair(const SweepArgs &a, int p, int t, int bx, int nbx) {
  typedef LinkIO<FMT_PAIR> IO;
  if (a.active && !a.active[t]) return;
  const int j = bx * blockDim.x + threadIdx.x;
  float acc[2] = {0.0f, 0.0f};
  if (j < a.g.vs_half) {
    constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    f2 W[18];
#pragma unroll
    for (int e = 0; e < 18; e++) W[e] = f2{0.0f, 0.0f};
#pragma unroll 1
    for (int mu = MU0; mu < 4; mu++) {
      f2 u[18];
      IO::load(a.links, a.g.vh, p, mu, i, u);
#pragma unroll
      for (int e = 0; e < 18; e++) W[e] = pair_add(W[e], u[e]);
      IO::load(a.links, a.g.vh, q, mu, cb_shift(a.g, c, mu, -1), u);
#pragma unroll
      for (int r = 0; r < 3; r++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) {  // K += U^dagger
          W[LGT_RE(r, cc)] = pair_add(W[LGT_RE(r, cc)], u[LGT_RE(cc, r)]);
          W[LGT_IM(r, cc)] = pair_add(W[LGT_IM(r, cc)], pair_neg(u[LGT_IM(cc, r)]));
        }
    }
    pair_violation(W, acc[0], acc[1]);
    uint4 draws = make_uint4(0, 0, 0, 0);
    if (ALGO == ALGO_SR) draws = sr_draws(a, c);
    Rot rot[3];
    pair_local_update<ALGO>(W, rot, (float)a.omega, a.sr_thr, draws);
    f2 d[18];
    pair_delta(rot, d);
    const int mu_lo = (GAUGE == GAUGE_COULOMB && a.transform_temporal) ? 0 : MU0;
#pragma unroll 1
    for (int mu = mu_lo; mu < 4; mu++) {
      const int nbm = cb_shift(a.g, c, mu, -1);
      f2 u[18];
      IO::load(a.links, a.g.vh, p, mu, i, u);
      pair_apply_left(u, d);
      IO::store(a.links, a.g.vh, p, mu, i, u);
      IO::load(a.links, a.g.vh, q, mu, nbm, u);
      pair_apply_right_dag(u, d);
      IO::store(a.links, a.g.vh, q, mu, nbm, u);
    }
  }
  fused_store<float>(a, p, t, bx, acc);
}

template <int GAUGE, int ALGO>
__global__ void __launch_bounds__(256) k_sweep_pair(SweepArgs a, int p) {
  sweep_body_pair<GAUGE, ALGO>(a, p, blockIdx.y, blockIdx.x, gridDim.x);
}

typedef void (*sweep_fn)(SweepArgs, int);

static sweep_fn pick_sweep(int fmt, int gauge, int algo) {
  if (fmt == FMT_PAIR) {
    if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_pair<GAUGE_LANDAU, ALGO_SR> : k_sweep_pair<GAUGE_LANDAU, ALGO_OR>;
    return algo == ALGO_SR ? k_sweep_pair<GAUGE_COULOMB, ALGO_SR> : k_sweep_pair<GAUGE_COULOMB, ALGO_OR>;
  }
#define LGT_PICK(F, G, A) \
  if (fmt == F && gauge == G && algo == A) return (F == FMT_F64) ? (sweep_fn)k_sweep_f64<G, A> : (sweep_fn)k_sweep_f32<(F == FMT_F64 ? FMT_F32_18 : F), G, A>;
  LGT_PICK(FMT_F64, GAUGE_LANDAU, ALGO_OR)
  LGT_PICK(FMT_F64, GAUGE_LANDAU, ALGO_SR)
  LGT_PICK(FMT_F64, GAUGE_COULOMB, ALGO_OR)
  LGT_PICK(FMT_F64, GAUGE_COULOMB, ALGO_SR)
  LGT_PICK(FMT_F32_18, GAUGE_LANDAU, ALGO_OR)
  LGT_PICK(FMT_F32_18, GAUGE_LANDAU, ALGO_SR)
  LGT_PICK(FMT_F32_18, GAUGE_COULOMB, ALGO_OR)
  LGT_PICK(FMT_F32_18, GAUGE_COULOMB, ALGO_SR)
  LGT_PICK(FMT_F32_12, GAUGE_LANDAU, ALGO_OR)
  LGT_PICK(FMT_F32_12, GAUGE_LANDAU, ALGO_SR)
  LGT_PICK(FMT_F32_12, GAUGE_COULOMB, ALGO_OR)
  LGT_PICK(FMT_F32_12, GAUGE_COULOMB, ALGO_SR)
#undef LGT_PICK
  return nullptr;
}

void fill_sweep_args(SweepArgs *a, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                     unsigned long long sweep, int reunit, int use_mask) {
  a->g = g;
  a->links = links;
  a->G = G;
  a->active = use_mask ? w.active : nullptr;
  a->warp_part = w.warp_part;
  a->wps = w.wps;
  a->omega = c.omega;
  a->sr_thr = c.sr_thr;
  a->seed = c.seed;
  a->sweep = sweep;
  a->transform_temporal = c.transform_temporal;
  a->reunit = reunit;
  a->reunit_every = 0;
  a->count_base = 0;
}

cudaError_t launch_half_sweep(int fmt, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                              int parity, unsigned long long sweep, int reunit, int use_mask, int block,
                              cudaStream_t st) {
  sweep_fn fn = pick_sweep(fmt, c.gauge, c.algo);
  if (!fn) return cudaErrorInvalidValue;
  SweepArgs a;
  fill_sweep_args(&a, g, links, G, w, c, sweep, reunit, use_mask);
  dim3 grid(ceil_div(g.vs_half, block), g.nt);
  fn<<<grid, block, 0, st>>>(a, parity & 1);
  return cudaGetLastError();
}

// ------------------------------------------------------------ measurement


template <int FMT>
struct LoadD {
  static __device__ __forceinline__ void run(const void *base, int vh, int p, int mu, int i, double m[18]) {
    typedef typename LinkIO<FMT>::real R;
    R r[18];
    LinkIO<FMT>::load(base, vh, p, mu, i, r);
#pragma unroll
    for (int k = 0; k < 18; k++) m[k] = (double)r[k];
  }
};

template <>
struct LoadD<FMT_PAIR> {
  static __device__ __forceinline__ void run(const void *base, int vh, int p, int mu, int i, double m[18]) {
    f2 r[18];
    LinkIO<FMT_PAIR>::load(base, vh, p, mu, i, r);
#pragma unroll
    for (int k = 0; k < 18; k++) m[k] = (double)r[k].hi + (double)r[k].lo;
  }
};

// a link of any storage format, widened to FP64
template <int FMT>
__device__ __forceinline__ void load_d(const void *base, int vh, int p, int mu, int i, double m[18]) {
  LoadD<FMT>::run(base, vh, p, mu, i, m);
}

// X += s * (U - U^dagger)
__device__ __forceinline__ void acc_antiherm(double X[18], const double u[18], double s) {
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      X[LGT_RE(a, b)] += s * (u[LGT_RE(a, b)] - u[LGT_RE(b, a)]);
      X[LGT_IM(a, b)] += s * (u[LGT_IM(a, b)] + u[LGT_IM(b, a)]);
    }
}

// tr[D D^dagger] for D = traceless part of X/(2i), X anti-Hermitian
__device__ __forceinline__ double traceless_norm(const double X[18]) {
  const double d0 = 0.5 * X[LGT_IM(0, 0)], d1 = 0.5 * X[LGT_IM(1, 1)], d2 = 0.5 * X[LGT_IM(2, 2)];
  const double tr3 = (d0 + d1 + d2) * (1.0 / 3.0);
  double s = (d0 - tr3) * (d0 - tr3) + (d1 - tr3) * (d1 - tr3) + (d2 - tr3) * (d2 - tr3);
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = a + 1; b < 3; b++) s += 0.5 * (X[LGT_RE(a, b)] * X[LGT_RE(a, b)] + X[LGT_IM(a, b)] * X[LGT_IM(a, b)]);
  return s;
}

template <int FMT>
__device__ __forceinline__ void measure_body(const MeasArgs &a, int t, int p, int bx, int nbx) {
  const int j = bx * blockDim.x + threadIdx.x;
  double v[MEAS_NV];
#pragma unroll
  for (int k = 0; k < MEAS_NV; k++) v[k] = 0.0;
  if (j < a.g.vs_half) {
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    double XL[18], XS[18];
    mat_zero(XL);
    mat_zero(XS);
    for (int mu = 0; mu < 4; mu++) {
      double u[18];
      load_d<FMT>(a.links, a.g.vh, p, mu, i, u);
      const double rt = u[LGT_RE(0, 0)] + u[LGT_RE(1, 1)] + u[LGT_RE(2, 2)];
      v[0] += rt;
      acc_antiherm(XL, u, 1.0);
      if (mu > 0) {
        v[1] += rt;
        acc_antiherm(XS, u, 1.0);
      }
      load_d<FMT>(a.links, a.g.vh, q, mu, cb_shift(a.g, c, mu, -1), u);
      acc_antiherm(XL, u, -1.0);
      if (mu > 0) acc_antiherm(XS, u, -1.0);
    }
    v[2] = traceless_norm(XL);
    v[3] = traceless_norm(XS);
    if (a.with_plaq) {
      for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) {
          double ua[18], ub[18], uc[18], ud[18], m1[18], m2[18];
          load_d<FMT>(a.links, a.g.vh, p, mu, i, ua);
          load_d<FMT>(a.links, a.g.vh, q, nu, cb_shift(a.g, c, mu, +1), ub);
          load_d<FMT>(a.links, a.g.vh, q, mu, cb_shift(a.g, c, nu, +1), uc);
          load_d<FMT>(a.links, a.g.vh, p, nu, i, ud);
          mat_mul(ua, ub, m1);       // U_mu(x) U_nu(x+mu)
          mat_mul(ud, uc, m2);       // U_nu(x) U_mu(x+nu)
          // Re tr[m1 m2^dagger] = sum_ab Re(m1_ab conj(m2_ab))
          double s = 0.0;
#pragma unroll
          for (int e = 0; e < 18; e++) s += m1[e] * m2[e];
          v[4] += s;
        }
    }
  }
  __shared__ double tot[MEAS_NV];
  __shared__ int am_last;
  block_sum<MEAS_NV, double>(v, tot);
  const int nblk = nbx * 2;  // blocks of this slice
  const int bidx = p * nbx + bx;
  if (threadIdx.x == 0) {
    double *dst = a.partial + ((size_t)t * nblk + bidx) * MEAS_NV;
#pragma unroll
    for (int k = 0; k < MEAS_NV; k++) dst[k] = tot[k];
    __threadfence();
    const unsigned prev = atomicAdd(&a.counter[t], 1u);
    am_last = (prev == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  // last block of slice t: fixed-order sum over the slice's blocks
  __threadfence();
#pragma unroll
  for (int k = 0; k < MEAS_NV; k++) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    const double *src = a.partial + ((size_t)t * nblk + b) * MEAS_NV;
#pragma unroll
    for (int k = 0; k < MEAS_NV; k++) v[k] += __ldcg(src + k);
  }
  block_sum<MEAS_NV, double>(v, tot);
  __shared__ int am_final;
  if (threadIdx.x == 0) {
    const double vs = 2.0 * (double)a.g.vs_half;
#pragma unroll
    for (int k = 0; k < MEAS_NV; k++) a.slice_sum[(size_t)t * MEAS_NV + k] = tot[k];
    const double ft = tot[1] / (9.0 * vs);
    const double tt = tot[3] / (3.0 * vs);
    a.slice_F[t] = ft;
    a.slice_theta[t] = tt;
    if (a.coulomb_target >= 0.0) a.active[t] = (tt >= a.coulomb_target) ? 1 : 0;
    a.counter[t] = 0u;
    __threadfence();
    const unsigned prev = atomicAdd(a.glob, 1u);
    am_final = (prev == (unsigned)a.g.nt - 1);
  }
  __syncthreads();
  if (!am_final || threadIdx.x != 0) return;
  // final block: totals over slices in slice order
  __threadfence();
  double s[MEAS_NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double fsum = 0.0, tmax = 0.0, tsum = 0.0;
  int nact = 0;
  for (int tt = 0; tt < a.g.nt; tt++) {
#pragma unroll
    for (int k = 0; k < MEAS_NV; k++) s[k] += __ldcg(a.slice_sum + (size_t)tt * MEAS_NV + k);
    const double th = __ldcg(a.slice_theta + tt);
    fsum += __ldcg(a.slice_F + tt);
    tsum += th;
    tmax = th > tmax ? th : tmax;
    nact += (int)(*(volatile uint8_t *)(a.active + tt));
  }
  const double vol = 2.0 * (double)a.g.vh;
  a.totals[TOT_F_LANDAU] = s[0] / (12.0 * vol);
  a.totals[TOT_THETA_LANDAU] = s[2] / (3.0 * vol);
  a.totals[TOT_PLAQ] = s[4] / (18.0 * vol);
  a.totals[TOT_F_COULOMB] = fsum / (double)a.g.nt;
  a.totals[TOT_THETA_COULOMB_MAX] = tmax;
  a.totals[TOT_THETA_COULOMB_MEAN] = tsum / (double)a.g.nt;
  a.totals[TOT_ACTIVE_SLICES] = (double)nact;
  *a.glob = 0u;
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
}

cudaError_t launch_measure(int fmt, const Geom &g, const void *links, const Workspace &w, int with_plaq,
                           double coulomb_target, int block, cudaStream_t st) {
  MeasArgs a;
  fill_meas_args(&a, g, links, w, with_plaq, coulomb_target);
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
    load_G_fp64(G, g.vh, p, i, gx);
    load_G_fp64(G, g.vh, p ^ 1, cb_shift(g, c, mu, +1), gy);
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
  k_apply_G<<<(unsigned)((n + blk - 1) / blk), blk, 0, st>>>(g, G, u64_in, u64_out, aos_out, skip_temporal);
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
void fill_fused_args(FusedArgs *a, const Geom &g, const Workspace &w, int gauge, int sweep_block,
                     double coulomb_target) {
  a->g = g;
  a->warp_part = w.warp_part;
  a->wps = w.wps;
  a->nw = ceil_div(g.vs_half, sweep_block) * (sweep_block / 32);
  a->gauge = gauge;
  a->slice = w.fused_slice;
  a->counter = w.fused_counter;
  a->totals = w.fused_totals;
  a->active = w.active;
  a->coulomb_target = coulomb_target;
}

// One block per timeslice: fixed-order sums of the slice's warp slots
// (parity-0 Re tr K; tr Delta^2 of both parities); the last block forms the
// totals in slice order.  Slices masked off (converged) keep their previous
// Re tr K sum and report zero violation.
__device__ __forceinline__ void fused_finish_body(const FusedArgs &a, int t) {
  __shared__ double tot[2];
  __shared__ int am_last;
  if (a.active[t]) {
    double v[2] = {0.0, 0.0};
    const double2 *p0 = a.warp_part + (size_t)t * a.wps;
    const double2 *p1 = a.warp_part + ((size_t)a.g.nt + t) * a.wps;
    for (int w = threadIdx.x; w < a.nw; w += blockDim.x) {
      const double2 x0 = p0[w], x1 = p1[w];
      v[0] += x0.x;
      v[1] += x0.y + x1.y;
    }
    block_sum<2, double>(v, tot);
    if (threadIdx.x == 0) {
      a.slice[2 * t] = tot[0];
      a.slice[2 * t + 1] = tot[1];
    }
  } else if (threadIdx.x == 0) {
    a.slice[2 * t + 1] = 0.0;  // converged and masked off: no new estimate
  }
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(a.counter, 1u) == (unsigned)a.g.nt - 1;
  }
  __syncthreads();
  if (!am_last || threadIdx.x != 0) return;
  __threadfence();
  const double vs = 2.0 * (double)a.g.vs_half, vol = 2.0 * (double)a.g.vh;
  const double nd = a.gauge == GAUGE_COULOMB ? 3.0 : 4.0;
  double fsum = 0.0, tsum = 0.0, tmax = 0.0, ftot = 0.0, ttot = 0.0;
  int nact = 0;
  for (int tt = 0; tt < a.g.nt; tt++) {
    const double rk = __ldcg(a.slice + 2 * tt), th2 = __ldcg(a.slice + 2 * tt + 1);
    ftot += rk;
    ttot += th2;
    const double ft = rk / (3.0 * nd * vs), th = th2 / (3.0 * vs);
    fsum += ft;
    tsum += th;
    tmax = th > tmax ? th : tmax;
    if (a.coulomb_target >= 0.0) a.active[tt] = th >= a.coulomb_target ? 1 : 0;
    nact += a.active[tt];
  }
  a.totals[TOT_F_LANDAU] = ftot / (3.0 * nd * vol);
  a.totals[TOT_THETA_LANDAU] = ttot / (3.0 * vol);
  a.totals[TOT_PLAQ] = 0.0;
  a.totals[TOT_F_COULOMB] = fsum / (double)a.g.nt;
  a.totals[TOT_THETA_COULOMB_MAX] = tmax;
  a.totals[TOT_THETA_COULOMB_MEAN] = tsum / (double)a.g.nt;
  a.totals[TOT_ACTIVE_SLICES] = (double)nact;
  *a.counter = 0u;
}

__global__ void __launch_bounds__(256) k_fused_finish(FusedArgs a) { fused_finish_body(a, blockIdx.x); }

cudaError_t launch_fused_finish(const Geom &g, const Workspace &w, int gauge, int sweep_block, double coulomb_target,
                                cudaStream_t st) {
  FusedArgs a;
  fill_fused_args(&a, g, w, gauge, sweep_block, coulomb_target);
  k_fused_finish<<<g.nt, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------- batched launches
// Block b of a batched grid belongs to the last row k with
// jobs[k].block_begin <= b (rows sorted by block_begin).
__device__ __forceinline__ int batch_row(const int *begins, int stride_bytes, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int beg = *reinterpret_cast<const int *>(reinterpret_cast<const char *>(begins) + (size_t)mid * stride_bytes);
    if (beg <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int FMT, int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_dispatch(const SweepArgs &a, int p, int t, int bx, int nbx) {
  if (FMT == FMT_F64) sweep_body_f64<GAUGE, ALGO>(a, p, t, bx, nbx);
  else if (FMT == FMT_PAIR) sweep_body_pair<GAUGE, ALGO>(a, p, t, bx, nbx);
  else sweep_body_f32<(FMT == FMT_F32_12 ? FMT_F32_12 : FMT_F32_18), GAUGE, ALGO>(a, p, t, bx, nbx);
}

template <int FMT, int GAUGE, int ALGO>
__global__ void __launch_bounds__(256) k_sweep_batch(const BatchSweep *jobs, int n, int p, int s) {
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchSweep), n, blockIdx.x);
  const BatchSweep &J = jobs[k];
  SweepArgs a = J.a;
  a.sweep += (unsigned long long)s;
  a.reunit = a.reunit_every > 0 && ((a.count_base + s + 1) % a.reunit_every) == 0;
  const int local = blockIdx.x - J.block_begin;
  const int t = local / J.nbx;
  sweep_dispatch<FMT, GAUGE, ALGO>(a, p, t, local - t * J.nbx, J.nbx);
}

template <int FMT>
__global__ void __launch_bounds__(256) k_measure_batch(const BatchMeas *jobs, int n) {
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchMeas), n, blockIdx.x);
  const BatchMeas &J = jobs[k];
  const int local = blockIdx.x - J.block_begin;
  const int per_t = 2 * J.nbx;
  const int t = local / per_t;
  const int rem = local - t * per_t;
  const int p = rem / J.nbx;
  measure_body<FMT>(J.a, t, p, rem - p * J.nbx, J.nbx);
}

typedef void (*batch_fn)(const BatchSweep *, int, int, int);

template <int FMT>
static batch_fn pick_batch_fmt(int gauge, int algo) {
  if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_batch<FMT, GAUGE_LANDAU, ALGO_SR> : k_sweep_batch<FMT, GAUGE_LANDAU, ALGO_OR>;
  return algo == ALGO_SR ? k_sweep_batch<FMT, GAUGE_COULOMB, ALGO_SR> : k_sweep_batch<FMT, GAUGE_COULOMB, ALGO_OR>;
}

cudaError_t launch_half_sweep_batch(int fmt, int gauge, int algo, const BatchSweep *jobs, int n, int total_blocks,
                                    int parity, int s, int block, cudaStream_t st) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  batch_fn fn = nullptr;
  if (fmt == FMT_F64) fn = pick_batch_fmt<FMT_F64>(gauge, algo);
  else if (fmt == FMT_F32_18) fn = pick_batch_fmt<FMT_F32_18>(gauge, algo);
  else if (fmt == FMT_F32_12) fn = pick_batch_fmt<FMT_F32_12>(gauge, algo);
  else if (fmt == FMT_PAIR) fn = pick_batch_fmt<FMT_PAIR>(gauge, algo);
  if (!fn) return cudaErrorInvalidValue;
  fn<<<total_blocks, block, 0, st>>>(jobs, n, parity & 1, s);
  return cudaGetLastError();
}

cudaError_t launch_measure_batch(int fmt, const BatchMeas *jobs, int n, int total_blocks, int block, cudaStream_t st) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  if (fmt == FMT_F64) k_measure_batch<FMT_F64><<<total_blocks, block, 0, st>>>(jobs, n);
  else if (fmt == FMT_F32_18) k_measure_batch<FMT_F32_18><<<total_blocks, block, 0, st>>>(jobs, n);
  else if (fmt == FMT_F32_12) k_measure_batch<FMT_F32_12><<<total_blocks, block, 0, st>>>(jobs, n);
  else if (fmt == FMT_PAIR) k_measure_batch<FMT_PAIR><<<total_blocks, block, 0, st>>>(jobs, n);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_fused_finish_batch(const BatchFused *jobs, int n) {
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchFused), n, blockIdx.x);
  fused_finish_body(jobs[k].a, blockIdx.x - jobs[k].block_begin);
}

cudaError_t launch_fused_finish_batch(const BatchFused *jobs, int n, int total_blocks, cudaStream_t st) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  k_fused_finish_batch<<<total_blocks, 256, 0, st>>>(jobs, n);
  return cudaGetLastError();
}

}  // namespace lgt
