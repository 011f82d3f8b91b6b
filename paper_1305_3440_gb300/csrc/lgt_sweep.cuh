// lgt_sweep.cuh -- the half-sweep bodies (Sec. 3 and Sec. 4 of Schroeck &
// Vogt): one thread per site of the active parity gathers K(x) from its 4
// forward links and the 4 backward links U_mu(x-mu) (sites of the other
// parity), runs the Cabibbo-Marinari local update and writes g U_mu(x) and
// U_mu(x-mu) g^dagger back in place.  Sites of one parity touch disjoint
// links, so a launch is race-free.  While K(x) is in registers each thread
// also adds Re tr K and tr[Delta Delta^dagger] to its warp's slot of the fused
// estimate.  The bodies take (timeslice, block in slice, blocks per slice) so
// the single-lattice and the batched multi-lattice kernels share them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lgt_device.cuh"
#include "lgt_internal.h"
#include "lgt_anchor.cuh"
#include "lgt_pair.cuh"

namespace lgt {



// The fused estimate: the sum of (Re tr K, tr Delta^2) over each group of
// LGT_FUSED_GROUP = 8 consecutive sites of a slice goes to the group's slot
// (xor butterfly: fixed order; no block barrier, no atomics), and
// k_fused_finish reduces the slots when an estimate is wanted.  STRIDE is the
// lane distance between consecutive sites (1: one thread per site, 4: four
// threads per site, the site's value on its thread 0).  The butterfly pairs
// the same sites in both layouts, so the slots do not depend on it.
template <typename T, int STRIDE>
__device__ __forceinline__ void fused_store(const SweepArgs &a, int p, int t, int bx, T acc[2]) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int off = 4 * STRIDE; off >= STRIDE; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  const int tid = bx * (int)blockDim.x + (int)threadIdx.x;  // thread index within the slice
  if ((threadIdx.x & (LGT_FUSED_GROUP * STRIDE - 1)) == 0) {
    const int slot = tid / (LGT_FUSED_GROUP * STRIDE);
    a.warp_part[((size_t)p * a.g.nt + t) * a.wps + slot] = make_double2((double)acc[0], (double)acc[1]);
  }
}

// The term of direction mu in K(x): U_mu(x) + U_mu(x - mu)^dagger (Sec. 3),
// formed from zero so that every site layout rounds it the same way.
template <typename R>
__device__ __forceinline__ void k_term(R k[18], const R uf[18], const R ub[18]) {
  mat_zero(k);
  acc_add(k, uf);
  acc_add_dag(k, ub);
}

// the heat-bath stream of one site update (simulated annealing)
__device__ __forceinline__ SaDraw sa_draw_of(const SweepArgs &a, const Coords &c) {
  SaDraw d;
  d.beta = a.beta;
  d.key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
  d.site = (uint32_t)((unsigned long long)c.x1 +
                      (unsigned long long)a.g.n1 *
                          ((unsigned long long)c.x2 +
                           (unsigned long long)a.g.n2 * ((unsigned long long)c.x3 + (unsigned long long)a.g.n3 * c.t)));
  d.sweep = (uint32_t)a.sweep;
  return d;
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

// A device loop's sweep kernels take the sweep number (SR counter) and the
// reunitarisation flag from the loop state (see LoopState).
__device__ __forceinline__ SweepArgs resolve_loop(const SweepArgs &in) {
  SweepArgs a = in;
  if (a.loop) {
    const unsigned long long off = a.sweep;
    a.sweep = a.loop->sweep + off;
    a.reunit = a.reunit_every > 0 && ((a.loop->count + (long long)off + 1) % a.reunit_every) == 0;
  }
  return a;
}

// The FP32 site update once the site's links are in registers (raw storage:
// 12-real links with row 2 zero): K(x), the fused estimate terms, the local
// update, the stores of the 8 links (and, for Coulomb gauge, the temporal
// links), and G(x) <- g G(x).  gpre: G(x) already loaded (row 2 rebuilt), or
// nullptr to load it here.
template <int FMT, int GAUGE, int ALGO>
__device__ __forceinline__ void site_update_f32(const SweepArgs &a, int p, const Coords &c, int i, const int nb[4],
                                                float uf[4][18], float ub[4][18], const float *gpre, float acc[2]) {
  typedef LinkIO<FMT> IO;
  constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
  const int q = p ^ 1;
  // K(x) = (k_0 + k_1) + (k_2 + k_3), k_mu the direction terms (k_0 = 0 for
  // Coulomb gauge): the order of the four-threads-per-site layout
  float W[18], k2[18];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    float ka[18], kb[18];
#pragma unroll
    for (int d = 0; d < 2; d++) {
      const int mu = 2 * h + d;
      float *k = d ? kb : ka;
      if (mu < MU0) {
        mat_zero(k);
      } else if (IO::kCompressed) {
        float ff[18], fb[18];
#pragma unroll
        for (int e = 0; e < 18; e++) {
          ff[e] = uf[mu][e];
          fb[e] = ub[mu][e];
        }
        rebuild_row2(ff);
        rebuild_row2(fb);
        k_term(k, ff, fb);
      } else {
        k_term(k, uf[mu], ub[mu]);
      }
    }
    float *dst = h ? k2 : W;
#pragma unroll
    for (int e = 0; e < 18; e++) dst[e] = ka[e] + kb[e];
  }
#pragma unroll
  for (int e = 0; e < 18; e++) W[e] = W[e] + k2[e];
  violation_of_K(W, acc[0], acc[1]);
  uint4 draws = make_uint4(0, 0, 0, 0);
  if (ALGO == ALGO_SR) draws = sr_draws(a, c);
  float gm[18];
  SaDraw sd;
  if (ALGO == ALGO_SA) sd = sa_draw_of(a, c);
  local_update<float, ALGO>(W, gm, (float)a.omega, a.sr_thr, draws, &sd);
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
    if (gpre) {
#pragma unroll
      for (int e = 0; e < 18; e++) gx[e] = gpre[e];
    } else {
      GIO::load(a.G, a.g.vh, p, i, gx);
    }
    mat_mul(gm, gx, r);
    if (a.reunit) reunitarise(r);
    GIO::store(a.G, a.g.vh, p, i, r);
  }
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
    site_update_f32<FMT, GAUGE, ALGO>(a, p, c, i, nb, uf, ub, nullptr, acc);
  }
  fused_store<float, 1>(a, p, t, bx, acc);
}

// FP32 link formats, lean: K(x) streamed (each link loaded, widened to 3 rows,
// added and dropped), the links loaded again for the write-back (L2 still
// holds them), so a thread keeps about a third of the registers of the
// all-in-registers body and more warps fit on an SM.
template <int FMT, int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_f32_lean(const SweepArgs &a, int p, int t, int bx) {
  typedef LinkIO<FMT> IO;
  if (a.active && !a.active[t]) return;
  const int j = bx * blockDim.x + threadIdx.x;
  float acc[2] = {0.0f, 0.0f};
  if (j < a.g.vs_half) {
    constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    // K(x) = (k_0 + k_1) + (k_2 + k_3), as the other layouts
    float W[18], k2[18];
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
      float ka[18], kb[18];
#pragma unroll
      for (int d = 0; d < 2; d++) {
        const int mu = 2 * h + d;
        float *k = d ? kb : ka;
        if (mu < MU0) {
          mat_zero(k);
        } else {
          float uf[18], ub[18];
          IO::load(a.links, a.g.vh, p, mu, i, uf);
          IO::load(a.links, a.g.vh, q, mu, cb_shift(a.g, c, mu, -1), ub);
          k_term(k, uf, ub);
        }
      }
      float *dst = h ? k2 : W;
#pragma unroll
      for (int e = 0; e < 18; e++) dst[e] = ka[e] + kb[e];
    }
#pragma unroll
    for (int e = 0; e < 18; e++) W[e] = W[e] + k2[e];
    violation_of_K(W, acc[0], acc[1]);
    uint4 draws = make_uint4(0, 0, 0, 0);
    if (ALGO == ALGO_SR) draws = sr_draws(a, c);
    float gm[18];
    local_update<float, ALGO>(W, gm, (float)a.omega, a.sr_thr, draws);
    const int mu_lo = (GAUGE == GAUGE_COULOMB && a.transform_temporal) ? 0 : MU0;
#pragma unroll 1
    for (int mu = mu_lo; mu < 4; mu++) {
      const int nb = cb_shift(a.g, c, mu, -1);
      float u[18], r[18];
      IO::load(a.links, a.g.vh, p, mu, i, u);
      mat_mul(gm, u, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, p, mu, i, r);
      IO::load_raw(a.links, a.g.vh, q, mu, nb, u);  // rows 0, 1 of U g^dagger need rows 0, 1 of U only
      mat_mul_dag(u, gm, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, q, mu, nb, r);
    }
    if (a.G) {
      float gx[18], r[18];
      GIO::load(a.G, a.g.vh, p, i, gx);
      mat_mul(gm, gx, r);
      if (a.reunit) reunitarise(r);
      GIO::store(a.G, a.g.vh, p, i, r);
    }
  }
  fused_store<float, 1>(a, p, t, bx, acc);
}

// 16-byte asynchronous copy global -> shared (cp.async, L1 bypassed) and its
// group bookkeeping
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// chunks of one site staged by the pipelined layout: 8 links x 3 (FP32-12) + G x 3
constexpr int LGT_PIPE_CHUNKS = 27;

// FP32-12, pipelined: persistent blocks walk the (slice, tile) list; while a
// thread updates its current site, the links and G of its next site are on the
// way into shared memory (cp.async), so each thread keeps a site's loads in
// flight through its compute phase.  A thread reads back only the chunks it
// staged itself (layout [buffer][chunk][thread]: conflict-free 16-byte reads),
// so no block barrier is needed; cp.async.wait_group orders each thread's own
// copies.  The site update is the one-thread body's, so results are the same.
template <int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_f32_pipe(const SweepArgs &a, int p, int tiles_x) {
  extern __shared__ float4 lgt_stage[];  // [2][LGT_PIPE_CHUNKS][blockDim.x]
  typedef LinkIO<FMT_F32_12> IO;
  constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
  const int T = (int)blockDim.x, tid = (int)threadIdx.x, q = p ^ 1;
  const int total = tiles_x * a.g.nt;
  const float4 *L = reinterpret_cast<const float4 *>(a.links);
  const float4 *Gs = reinterpret_cast<const float4 *>(a.G);
  auto issue = [&](int tile, int buf) {
    if (tile < total) {
      const int t = tile / tiles_x, j = (tile - t * tiles_x) * T + tid;
      if (!(a.active && !a.active[t]) && j < a.g.vs_half) {
        const Coords c = coords_in_slice(a.g, p, t, j);
        const int i = t * a.g.vs_half + j;
        float4 *st = lgt_stage + (size_t)buf * LGT_PIPE_CHUNKS * T + tid;
#pragma unroll
        for (int mu = MU0; mu < 4; mu++) {
          const int nb = cb_shift(a.g, c, mu, -1);
#pragma unroll
          for (int k = 0; k < 3; k++) {
            cp_async16(st + (mu * 6 + k) * T, L + (size_t)((p * 4 + mu) * 3 + k) * a.g.vh + i);
            cp_async16(st + (mu * 6 + 3 + k) * T, L + (size_t)((q * 4 + mu) * 3 + k) * a.g.vh + nb);
          }
        }
        if (Gs) {
#pragma unroll
          for (int k = 0; k < 3; k++) cp_async16(st + (24 + k) * T, Gs + (size_t)(p * 3 + k) * a.g.vh + i);
        }
      }
    }
    cp_async_commit();  // possibly empty: every iteration commits exactly one group
  };
  int tile = (int)blockIdx.x;
  issue(tile, 0);
  for (int it = 0; tile < total; it++, tile += (int)gridDim.x) {
    issue(tile + (int)gridDim.x, (it + 1) & 1);
    cp_async_wait<1>();  // this thread's copies of the current tile have landed
    const int t = tile / tiles_x, bx = tile - t * tiles_x;
    if (a.active && !a.active[t]) continue;  // the whole tile belongs to one slice
    const int j = bx * T + tid;
    float acc[2] = {0.0f, 0.0f};
    if (j < a.g.vs_half) {
      const Coords c = coords_in_slice(a.g, p, t, j);
      const int i = t * a.g.vs_half + j;
      const float4 *st = lgt_stage + (size_t)(it & 1) * LGT_PIPE_CHUNKS * T + tid;
      float uf[4][18], ub[4][18], gx[18];
      int nb[4];
#pragma unroll
      for (int mu = MU0; mu < 4; mu++) {
        nb[mu] = cb_shift(a.g, c, mu, -1);
#pragma unroll
        for (int k = 0; k < 3; k++) {
          const float4 f = st[(mu * 6 + k) * T], b = st[(mu * 6 + 3 + k) * T];
          uf[mu][4 * k] = f.x, uf[mu][4 * k + 1] = f.y, uf[mu][4 * k + 2] = f.z, uf[mu][4 * k + 3] = f.w;
          ub[mu][4 * k] = b.x, ub[mu][4 * k + 1] = b.y, ub[mu][4 * k + 2] = b.z, ub[mu][4 * k + 3] = b.w;
        }
#pragma unroll
        for (int e = 12; e < 18; e++) uf[mu][e] = ub[mu][e] = 0.0f;
      }
      if (Gs) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
          const float4 v = st[(24 + k) * T];
          gx[4 * k] = v.x, gx[4 * k + 1] = v.y, gx[4 * k + 2] = v.z, gx[4 * k + 3] = v.w;
        }
        rebuild_row2(gx);
      }
      site_update_f32<FMT_F32_12, GAUGE, ALGO>(a, p, c, i, nb, uf, ub, Gs ? gx : nullptr, acc);
    }
    fused_store<float, 1>(a, p, t, bx, acc);
  }
  cp_async_wait<0>();  // nothing of this thread's in flight at exit
}


// FP32 link formats, four threads per site: thread m of the site's quad owns
// direction m (for Coulomb gauge thread 0 owns the temporal links, which the
// transformation also moves).  Each thread loads its forward and backward
// link and forms its term k_m of K(x); two xor shuffles sum the terms as
// (k_0 + k_1) + (k_2 + k_3), the order of the one-thread layout, so all four
// threads hold the same K bit for bit and run the same local update; then
// each thread writes its own two links (thread 0 also G).  Per thread this
// holds a quarter of the links, which buys occupancy: more loads in flight.
template <int FMT, int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_f32_quad(const SweepArgs &a, int p, int t, int bx) {
  typedef LinkIO<FMT> IO;
  if (a.active && !a.active[t]) return;  // whole block belongs to one slice
  constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
  const int m = threadIdx.x & 3;
  const int j = bx * (int)(blockDim.x >> 2) + (int)(threadIdx.x >> 2);
  const bool valid = j < a.g.vs_half;  // the shuffles below need every lane
  const bool in_K = m >= MU0;
  const Coords c = coords_in_slice(a.g, p, t, valid ? j : 0);
  const int i = t * a.g.vs_half + (valid ? j : 0);
  const int q = p ^ 1;
  const int nb = cb_shift(a.g, c, m, -1);
  float uf[18], ub[18], W[18];
  mat_zero(W);
  if (valid && in_K) {
    IO::load_raw(a.links, a.g.vh, p, m, i, uf);
    IO::load_raw(a.links, a.g.vh, q, m, nb, ub);
    if (IO::kCompressed) {
      float fb[18];
#pragma unroll
      for (int e = 0; e < 18; e++) fb[e] = ub[e];
      rebuild_row2(uf);  // g U needs row 2 of U
      rebuild_row2(fb);
      k_term(W, uf, fb);
    } else {
      k_term(W, uf, ub);
    }
  }
#pragma unroll
  for (int e = 0; e < 18; e++) W[e] = W[e] + __shfl_xor_sync(0xffffffffu, W[e], 1);
#pragma unroll
  for (int e = 0; e < 18; e++) W[e] = W[e] + __shfl_xor_sync(0xffffffffu, W[e], 2);
  float acc[2] = {0.0f, 0.0f};
  {
    float vr, vd;
    violation_of_K(W, vr, vd);
    if (valid && m == 0) {
      acc[0] = vr;
      acc[1] = vd;
    }
  }
  uint4 draws = make_uint4(0, 0, 0, 0);
  if (ALGO == ALGO_SR) draws = sr_draws(a, c);
  float gm[18];
  local_update<float, ALGO>(W, gm, (float)a.omega, a.sr_thr, draws);
  if (valid && in_K) {
    float r[18];
    mat_mul(gm, uf, r);
    if (a.reunit) reunitarise(r);
    IO::store(a.links, a.g.vh, p, m, i, r);
    mat_mul_dag(ub, gm, r);  // rows 0, 1 of U g^dagger need rows 0, 1 of U only
    if (a.reunit) reunitarise(r);
    IO::store(a.links, a.g.vh, q, m, nb, r);
  }
  if (GAUGE == GAUGE_COULOMB && valid && m == 0 && a.transform_temporal) {
    float u[18], r[18];
    IO::load(a.links, a.g.vh, p, 0, i, u);
    mat_mul(gm, u, r);
    if (a.reunit) reunitarise(r);
    IO::store(a.links, a.g.vh, p, 0, i, r);
    IO::load(a.links, a.g.vh, q, 0, nb, u);
    mat_mul_dag(u, gm, r);
    if (a.reunit) reunitarise(r);
    IO::store(a.links, a.g.vh, q, 0, nb, r);
  }
  if (a.G && valid && m == 0) {
    float gx[18], r[18];
    GIO::load(a.G, a.g.vh, p, i, gx);
    mat_mul(gm, gx, r);
    if (a.reunit) reunitarise(r);
    GIO::store(a.G, a.g.vh, p, i, r);
  }
  fused_store<float, 4>(a, p, t, bx, acc);
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
    SaDraw sd;
    if (ALGO == ALGO_SA) sd = sa_draw_of(a, c);
    local_update<double, ALGO>(W, gm, a.omega, a.sr_thr, draws, &sd);
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
  fused_store<double, 1>(a, p, t, bx, acc);
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
    PairAcc K[18];
#pragma unroll
    for (int e = 0; e < 18; e++) K[e] = PairAcc{0.0f, 0.0f};
#pragma unroll 1
    for (int mu = MU0; mu < 4; mu++) {
      f2 u[18];
      IO::load(a.links, a.g.vh, p, mu, i, u);
#pragma unroll
      for (int e = 0; e < 18; e++) acc_add_pair(K[e], u[e]);
      IO::load(a.links, a.g.vh, q, mu, cb_shift(a.g, c, mu, -1), u);
#pragma unroll
      for (int r = 0; r < 3; r++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) {  // K += U^dagger
          acc_add_pair(K[LGT_RE(r, cc)], u[LGT_RE(cc, r)]);
          acc_add_pair(K[LGT_IM(r, cc)], pair_neg(u[LGT_IM(cc, r)]));
        }
    }
    f2 W[18];
#pragma unroll
    for (int e = 0; e < 18; e++) W[e] = acc_value(K[e]);
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
  fused_store<float, 1>(a, p, t, bx, acc);
}


// Anchored polishing sweep (lgt_anchor.cuh): a.links = FP32-12 copy of the
// anchor field U', a.G = D = G - 1 (pairs), a.aux = K0 (pairs).  One thread per
// site; only D(x) is written.  K(x) in pair precision; rotations, delta = g - 1
// and delta D in FP32; D accumulated as a pair.
template <int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_anchor(const SweepArgs &a, int p, int t, int bx, int nbx) {
  typedef LinkIO<FMT_F32_12> IO;
  if (a.active && !a.active[t]) return;
  const int j = bx * blockDim.x + threadIdx.x;
  float acc[2] = {0.0f, 0.0f};
  if (j < a.g.vs_half) {
    constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    // C(x) = sum_mu U'_mu(x) D(x+mu)^+ + U'_mu(x-mu)^+ D(x-mu)^+  (small; FP32)
    float C[18];
    mat_zero(C);
#pragma unroll 1
    for (int mu = MU0; mu < 4; mu++) {
      float u[18], dn[18];
      IO::load(a.links, a.g.vh, p, mu, i, u);
      DIO::load_hi(a.G, a.g.vh, q, cb_shift(a.g, c, mu, +1), dn);
      acc_mul_dag(u, dn, C);
      const int nb = cb_shift(a.g, c, mu, -1);
      IO::load(a.links, a.g.vh, q, mu, nb, u);
      DIO::load_hi(a.G, a.g.vh, q, nb, dn);
      acc_dag_mul_dag(u, dn, C);
    }
    // M = K0 + C, then K = M + D(x) M (the small product in FP32)
    f2 K[18];
    K0IO::load(a.aux, a.g.vh, p, i, K);
#pragma unroll
    for (int e = 0; e < 18; e++) K[e] = pair_add(K[e], f2{C[e], 0.0f});
    float dh[18];  // D(x), high parts, row 2 rebuilt
    DIO::load_hi(a.G, a.g.vh, p, i, dh);
    {
      float mh[18], dm[18];
#pragma unroll
      for (int e = 0; e < 18; e++) mh[e] = K[e].hi;
      mat_mul(dh, mh, dm);
#pragma unroll
      for (int e = 0; e < 18; e++) K[e] = pair_add(K[e], f2{dm[e], 0.0f});
    }
    pair_violation(K, acc[0], acc[1]);
    uint4 draws = make_uint4(0, 0, 0, 0);
    if (ALGO == ALGO_SR) draws = sr_draws(a, c);
    RotF rf[3];
    anchor_local_update<ALGO>(K, rf, (float)a.omega, a.sr_thr, draws);
    float d[18];
    float_delta(rf, d);
    f2 D[18];
    DIO::load_pair_rows(a.G, a.g.vh, p, i, D);
    d_update_lite(D, dh, d);
    DIO::store_pair(a.G, a.g.vh, p, i, D);
  }
  fused_store<float, 1>(a, p, t, bx, acc);
}


template <int FMT, int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_dispatch(const SweepArgs &a, int p, int t, int bx, int nbx) {
  if (FMT == FMT_F64) sweep_body_f64<GAUGE, ALGO>(a, p, t, bx, nbx);
  else if (FMT == FMT_PAIR) sweep_body_pair<GAUGE, ALGO>(a, p, t, bx, nbx);
  else if (FMT == FMT_ANCHOR) sweep_body_anchor<GAUGE, ALGO>(a, p, t, bx, nbx);
  else sweep_body_f32<(FMT == FMT_F32_12 ? FMT_F32_12 : FMT_F32_18), GAUGE, ALGO>(a, p, t, bx, nbx);
}

}  // namespace lgt
