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
                           (unsigned long long)a.g.n2 *
                               ((unsigned long long)c.x3 + (unsigned long long)a.g.n3 * (long long)(c.t + a.t_offset))));
  d.sweep = (uint32_t)a.sweep;
  return d;
}

__device__ __forceinline__ uint4 sr_draws(const SweepArgs &a, const Coords &c) {
  const unsigned long long lex =
      (unsigned long long)c.x1 +
      (unsigned long long)a.g.n1 * ((unsigned long long)c.x2 +
                                    (unsigned long long)a.g.n2 * ((unsigned long long)c.x3 +
                                                                  (unsigned long long)a.g.n3 *
                                                                      (unsigned long long)(c.t + a.t_offset)));
  const uint4 ctr = make_uint4((uint32_t)lex, (uint32_t)(lex >> 32), (uint32_t)a.sweep, LGT_SR_TAG);
  const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
  return philox4x32_10(ctr, key);
}

// Programmatic dependent launch: a sweep kernel may be scheduled while the
// kernel before it in the stream drains.  Its first act is griddepcontrol.wait,
// which returns once that kernel has completed and its writes are visible, so
// nothing of the field, the loop state or the estimate slots is touched before;
// then it lets its own successor be scheduled.  Both are no-ops in a plain launch.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Snake order.  Blocks are dispatched in increasing linear index, so a launch
// walks the lattice slice by slice and the lines it touched last are the ones
// still in L2 when it ends.  A half-sweep of parity 1 therefore visits the
// (slice, tile) list from its end: it starts on the slices the parity-0
// half-sweep finished last, reads most of their links from L2 and overwrites
// those dirty lines before they are written back, and the next parity-0
// half-sweep starts where it ended.  Sites of one parity touch disjoint links,
// so the order changes no result; the estimate slots follow the logical tile.
__device__ __forceinline__ bool sweep_reversed(const SweepArgs &a, int p) { return a.snake && (p & 1); }
// (slice, tile) of this block in a (tiles per slice, slices) grid
__device__ __forceinline__ void sweep_block_tile(const SweepArgs &a, int p, int &t, int &bx) {
  if (sweep_reversed(a, p)) {
    t = a.t_first + (int)gridDim.y - 1 - (int)blockIdx.y;
    bx = (int)gridDim.x - 1 - (int)blockIdx.x;
  } else {
    t = a.t_first + (int)blockIdx.y;
    bx = (int)blockIdx.x;
  }
}

// A device loop's sweep kernels take the sweep number (SR counter), the OR
// parameter (omega schedule) and the reunitarisation flag from the loop state
// (see LoopState).
__device__ __forceinline__ SweepArgs resolve_loop(const SweepArgs &in) {
  SweepArgs a = in;
  if (a.loop) {
    const unsigned long long off = a.sweep;
    a.omega = a.loop->omega;
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
    // K(x) = sum_mu U_mu(x) + U_mu(x - mu)^dagger accumulated link by link: one
    // link in registers at a time (the other layouts' pairwise order needs three
    // matrices live; the sums differ only in FP32 rounding)
    float W[18];
    mat_zero(W);
#pragma unroll 1
    for (int mu = MU0; mu < 4; mu++) {
      float u[18];
      IO::load(a.links, a.g.vh, p, mu, i, u);
      acc_add(W, u);
      IO::load(a.links, a.g.vh, q, mu, cb_shift(a.g, c, mu, -1), u);
      acc_add_dag(W, u);
    }
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
  const int total = tiles_x * a.t_count;  // tiles of the launch's slices t_first ...
  const float4 *L = reinterpret_cast<const float4 *>(a.links);
  const float4 *Gs = reinterpret_cast<const float4 *>(a.G);
  const bool rev = sweep_reversed(a, p);
  auto issue = [&](int slot, int buf) {
    if (slot < total) {
      const int tile = rev ? total - 1 - slot : slot;
      const int t = a.t_first + tile / tiles_x, j = (tile - (t - a.t_first) * tiles_x) * T + tid;
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
  int slot = (int)blockIdx.x;  // position in the visiting order
  issue(slot, 0);
  for (int it = 0; slot < total; it++, slot += (int)gridDim.x) {
    issue(slot + (int)gridDim.x, (it + 1) & 1);
    cp_async_wait<1>();  // this thread's copies of the current tile have landed
    const int tile = rev ? total - 1 - slot : slot;
    const int t = a.t_first + tile / tiles_x, bx = tile - (t - a.t_first) * tiles_x;
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


// FP32-12, staged: one batch of cp.async copies brings the site's links (the 8
// of K(x), plus the temporal pair of a Coulomb update that transforms U_0) and
// G(x) into the thread's own shared-memory slots, so the site waits for memory
// once instead of once per direction and once more per reload; the update then
// runs as the lean body's (K summed link by link, same arithmetic), reading its
// operands from shared memory.  Slots [chunk][thread] as in the pipelined
// layout: a thread reads back only what it staged, so no block barrier is
// needed; 432 B per thread bound the blocks per SM (4 of 128 threads).  With
// STAGE_G false only the links are staged (384 B per thread, 9 blocks of 64
// threads per SM) and G(x) comes into registers by plain loads issued beside
// the copies.
template <int GAUGE, int ALGO, bool STAGE_G = true>
__device__ __forceinline__ void sweep_body_f32_staged(const SweepArgs &a, int p, int t, int bx) {
  extern __shared__ float4 lgt_stage[];  // [LGT_PIPE_CHUNKS][blockDim.x]
  typedef LinkIO<FMT_F32_12> IO;
  if (a.active && !a.active[t]) return;  // whole block belongs to one slice
  const int T = (int)blockDim.x, tid = (int)threadIdx.x;
  const int j = bx * T + tid;
  float acc[2] = {0.0f, 0.0f};
  if (j < a.g.vs_half) {
    constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
    const int mu_lo = (GAUGE == GAUGE_COULOMB && a.transform_temporal) ? 0 : MU0;
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    const float4 *L = reinterpret_cast<const float4 *>(a.links);
    const float4 *Gs = reinterpret_cast<const float4 *>(a.G);
    float4 *slot = lgt_stage + tid;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      if (mu < mu_lo) continue;
      const int nb = cb_shift(a.g, c, mu, -1);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        cp_async16(slot + (mu * 6 + k) * T, L + (size_t)((p * 4 + mu) * 3 + k) * a.g.vh + i);
        cp_async16(slot + (mu * 6 + 3 + k) * T, L + (size_t)((q * 4 + mu) * 3 + k) * a.g.vh + nb);
      }
    }
    float4 gq[3];  // !STAGE_G: rows 0, 1 of G(x), in flight beside the copies
    if (Gs) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        if constexpr (STAGE_G) cp_async16(slot + (24 + k) * T, Gs + (size_t)(p * 3 + k) * a.g.vh + i);
        else gq[k] = __ldg(Gs + (size_t)(p * 3 + k) * a.g.vh + i);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();  // this thread's copies have landed
    // rows 0, 1 of the staged matrix at chunk c0 (row 2 zero)
    auto staged = [&](int c0, float m[18]) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const float4 v = slot[(c0 + k) * T];
        m[4 * k] = v.x, m[4 * k + 1] = v.y, m[4 * k + 2] = v.z, m[4 * k + 3] = v.w;
      }
#pragma unroll
      for (int e = 12; e < 18; e++) m[e] = 0.0f;
    };
    float W[18];
    mat_zero(W);
#pragma unroll 1
    for (int mu = MU0; mu < 4; mu++) {
      float u[18];
      staged(mu * 6, u);
      rebuild_row2(u);
      acc_add(W, u);
      staged(mu * 6 + 3, u);
      rebuild_row2(u);
      acc_add_dag(W, u);
    }
    violation_of_K(W, acc[0], acc[1]);
    uint4 draws = make_uint4(0, 0, 0, 0);
    if (ALGO == ALGO_SR) draws = sr_draws(a, c);
    float gm[18];
    local_update<float, ALGO>(W, gm, (float)a.omega, a.sr_thr, draws);
#pragma unroll 1
    for (int mu = mu_lo; mu < 4; mu++) {
      const int nb = cb_shift(a.g, c, mu, -1);
      float u[18], r[18];
      staged(mu * 6, u);
      rebuild_row2(u);
      mat_mul(gm, u, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, p, mu, i, r);
      staged(mu * 6 + 3, u);  // rows 0, 1 of U g^dagger need rows 0, 1 of U only
      mat_mul_dag(u, gm, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, q, mu, nb, r);
    }
    if (Gs) {
      float gx[18], r[18];
      if constexpr (STAGE_G) {
        staged(24, gx);
      } else {
#pragma unroll
        for (int k = 0; k < 3; k++) {
          gx[4 * k] = gq[k].x, gx[4 * k + 1] = gq[k].y, gx[4 * k + 2] = gq[k].z, gx[4 * k + 3] = gq[k].w;
        }
#pragma unroll
        for (int e = 12; e < 18; e++) gx[e] = 0.0f;
      }
      rebuild_row2(gx);
      mat_mul(gm, gx, r);
      if (a.reunit) reunitarise(r);
      GIO::store(a.G, a.g.vh, p, i, r);
    }
  }
  fused_store<float, 1>(a, p, t, bx, acc);
}


// ---------------------------------------------------------------- streaming
// Several half-sweeps in one persistent launch.  Item n of the launch is
// (half-sweep h, position k, group bx of up to stream_tiles tiles); half-sweep
// h visits slice t = (h S + k) mod nt at position k.  A site of slice t touches
// links stored in slices t and t - 1 only (the temporal backward link), so
// half-sweep h may update slice t once half-sweep h - 1 has finished slices
// t - 1, t and t + 1.  Configuration 10 takes the half-sweeps one after the
// other (n = (h nt + k) items_x + bx, S = 1): the slices item (h, k) needs are
// the first positions of half-sweep h - 1 after k, long finished when it comes
// up, and the pipeline streams across half-sweep boundaries.  Configuration 12
// takes them in a rolling band (stream_band_rank: half-sweep h starts D waves
// after h - 1 and S = D - G slices further on), so about nt / D half-sweeps
// sweep the lattice together, G slices apart, and a slice's links come back to
// the next half-sweep a few slices of work after the last one wrote them, from
// L2; only the S slices each half-sweep skips at its start wait for its end.  done[t] counts the finished items of slice t over the
// launch: it reaches h * items_x only when every item of slice t in half-sweeps
// before h has finished, because each such item waited for the ones before it.
// Blocks take items from a ticket counter, in order, and wait only for items
// of smaller tickets, which running blocks hold; a block waits only while it
// holds no unfinished item of its own, so the launch cannot deadlock, however
// many of its blocks are resident.  Every wait is bounded in time: after
// stream_wait_ns (LGT_STREAM_WAIT_NS unless a test sets it) the block raises
// the abort flag and bit 1 of the error word, and every block ends.
__device__ __forceinline__ unsigned long long lgt_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned lgt_ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Publication: after a block barrier, one thread's release-add makes the whole
// block's earlier writes visible to a thread whose acquire-load reads the sum
// (release is cumulative over what the barrier ordered before it); that thread
// passes them on to its block through the next barrier.
__device__ __forceinline__ void lgt_red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct StreamItem {
  int h, t, bx;
};
// item n: slot n / items_x of the launch's order -- (h, k) = (slot / nt, slot
// mod nt) half-sweep after half-sweep, or the rolling band's table -- and group
// n mod items_x of slice h * shift + k (mod nt)
__device__ __forceinline__ StreamItem stream_item(unsigned n, int items_x, int nt, const unsigned *order, int shift) {
  StreamItem it;
  const unsigned slot = n / (unsigned)items_x;
  it.bx = (int)(n - slot * (unsigned)items_x);
  int k;
  if (order) {
    const unsigned e = __ldg(order + slot);
    it.h = (int)(e >> 16);
    k = (int)(e & 0xffffu);
  } else {
    it.h = (int)(slot / (unsigned)nt);
    k = (int)(slot - (unsigned)it.h * (unsigned)nt);
  }
  it.t = (int)(((long long)it.h * shift + k) % nt);
  return it;
}
// whether half-sweep it.h - 1 has finished slices t - 1, t, t + 1 (one look)
__device__ __forceinline__ bool stream_ready(const unsigned *done, const StreamItem &it, int items_x, int nt) {
  if (it.h == 0) return true;
  const unsigned need = (unsigned)it.h * (unsigned)items_x;
  const int tm = it.t == 0 ? nt - 1 : it.t - 1, tp = it.t == nt - 1 ? 0 : it.t + 1;
  const unsigned a = lgt_ld_acquire(done + tm), b = lgt_ld_acquire(done + it.t), c = lgt_ld_acquire(done + tp);
  return a >= need && b >= need && c >= need;
}
// bounded wait for stream_ready (thread 0 of a block); false: the launch gives up
__device__ __forceinline__ bool stream_wait(unsigned *ctr, int *err, const StreamItem &it, int items_x, int nt,
                                            unsigned long long limit_ns) {
  const unsigned long long t0 = lgt_clock_ns();
  for (unsigned k = 0; k < (1u << 26); k++) {
    if (stream_ready(ctr + 2, it, items_x, nt)) return true;
    if (lgt_ld_acquire(ctr + 1)) return false;  // another block gave up
    if (lgt_clock_ns() - t0 > limit_ns) break;
    __nanosleep(128);
  }
  atomicExch(ctr + 1, 1u);
  atomicOr(err, LGT_ERR_STREAM_WAIT);
  return false;
}

template <int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_body_f32_stream(const SweepArgs &in, int p0, int tiles_x) {
  extern __shared__ float4 lgt_stage[];  // [2][LGT_PIPE_CHUNKS][blockDim.x]
  __shared__ unsigned s_next;            // the next item's ticket
  __shared__ int s_ready, s_go;          // its slices were ready when looked at; the current item may start
  typedef LinkIO<FMT_F32_12> IO;
  constexpr int MU0 = GAUGE == GAUGE_COULOMB ? 1 : 0;
  const int T = (int)blockDim.x, tid = (int)threadIdx.x, nt = in.g.nt;
  const int per_item = in.stream_tiles;                    // tiles per item
  const int items_x = (tiles_x + per_item - 1) / per_item;  // items per slice
  const unsigned total = (unsigned)items_x * (unsigned)nt * (unsigned)in.n_half;
  unsigned *ctr = in.stream;
  const float4 *L = reinterpret_cast<const float4 *>(in.links);
  const float4 *Gs = reinterpret_cast<const float4 *>(in.G);
  // sweep numbers and the reunitarisation schedule of the launch's sweeps
  // (with a device loop, in.sweep is the launch's offset in the chunk)
  unsigned long long sweep0 = in.sweep;
  long long count0 = in.count_base;
  double omega = in.omega;
  if (in.loop) {
    sweep0 = in.loop->sweep + in.sweep;
    count0 = in.loop->count + (long long)in.sweep;
    omega = in.loop->omega;
  }
  // stage tile `tile` of slice it.t in half-sweep it.h
  auto issue = [&](const StreamItem &it, int tile, int buf) {
    const int p = (p0 + it.h) & 1, q = p ^ 1;
    const int j = tile * T + tid;
    if (!(in.active && !in.active[it.t]) && j < in.g.vs_half) {
      const Coords c = coords_in_slice(in.g, p, it.t, j);
      const int i = it.t * in.g.vs_half + j;
      float4 *st = lgt_stage + (size_t)buf * LGT_PIPE_CHUNKS * T + tid;
#pragma unroll
      for (int mu = MU0; mu < 4; mu++) {
        const int nb = cb_shift(in.g, c, mu, -1);
#pragma unroll
        for (int k = 0; k < 3; k++) {
          cp_async16(st + (mu * 6 + k) * T, L + (size_t)((p * 4 + mu) * 3 + k) * in.g.vh + i);
          cp_async16(st + (mu * 6 + 3 + k) * T, L + (size_t)((q * 4 + mu) * 3 + k) * in.g.vh + nb);
        }
      }
      if (Gs) {
#pragma unroll
        for (int k = 0; k < 3; k++) cp_async16(st + (24 + k) * T, Gs + (size_t)(p * 3 + k) * in.g.vh + i);
      }
    }
  };
  // thread 0 looks (without waiting: the item may depend on this block's
  // current one) whether ticket n's slices are ready, and shares n
  auto share = [&](unsigned n) {
    if (tid == 0) {
      int ready = 0;
      if (n < total && !lgt_ld_acquire(ctr + 1)) {
        ready = stream_ready(ctr + 2, stream_item(n, items_x, nt, in.stream_order, in.stream_shift), items_x, nt) ? 1 : 0;
      }
      s_next = n;
      s_ready = ready;
    }
    __syncthreads();
  };
  share(tid == 0 ? atomicAdd(ctr, 1u) + in.stream_skip : 0u);
  unsigned cur = s_next;
  int staged = s_ready, buf = 0;  // staged: the current tile's loads are issued
  if (cur < total && staged) {
    const StreamItem it = stream_item(cur, items_x, nt, in.stream_order, in.stream_shift);
    issue(it, it.bx * per_item, 0);
  }
  cp_async_commit();
  bool abort = false;
  while (cur < total && !abort) {
    const StreamItem it = stream_item(cur, items_x, nt, in.stream_order, in.stream_shift);  // it.bx: the item's index in its slice
    const int first = it.bx * per_item;
    const int ntl = tiles_x - first < per_item ? tiles_x - first : per_item;
    const int p = (p0 + it.h) & 1;
    const int sw = (p0 + it.h) >> 1;  // sweep of the launch
    SweepArgs a = in;
    a.omega = omega;
    a.sweep = sweep0 + (unsigned long long)sw;
    a.reunit = in.reunit_every > 0 ? (int)(((count0 + sw + 1) % in.reunit_every) == 0) : in.reunit;
    const bool on = !(in.active && !in.active[it.t]);
    unsigned ticket = 0;
    if (tid == 0) ticket = atomicAdd(ctr, 1u) + in.stream_skip;  // the next item's ticket, used at the last tile
    unsigned nxt = 0;
    int nxt_ready = 0;
    // one copy of the site update: unrolled, the body would outgrow the instruction cache
#pragma unroll 1
    for (int u = 0; u < ntl; u++) {
      if (!staged) {  // first tile of an item that was not ready: wait, then load it
        if (tid == 0) s_go = stream_wait(ctr, in.err, it, items_x, nt, in.stream_wait_ns) ? 1 : 0;
        __syncthreads();
        if (!s_go) {  // uniform: every thread read the same flag
          abort = true;
          break;
        }
        issue(it, first + u, buf);
        cp_async_commit();
      }
      // stage the tile after this one (the item's slices are ready now): the
      // item's next tile, or the next item's first if its slices are ready
      if (u + 1 < ntl) {
        issue(it, first + u + 1, buf ^ 1);
      } else {
        share(ticket);
        nxt = s_next;
        nxt_ready = s_ready;
        if (nxt < total && nxt_ready) {
          const StreamItem in2 = stream_item(nxt, items_x, nt, in.stream_order, in.stream_shift);
          issue(in2, in2.bx * per_item, buf ^ 1);
        }
      }
      cp_async_commit();   // possibly empty: every tile commits exactly one group here
      cp_async_wait<1>();  // all but that group: this thread's copies of the current tile have landed
      if (on) {  // the whole tile belongs to one slice
        const int tile = first + u;
        const int j = tile * T + tid;
        float acc[2] = {0.0f, 0.0f};
        if (j < in.g.vs_half) {
          const Coords c = coords_in_slice(in.g, p, it.t, j);
          const int i = it.t * in.g.vs_half + j;
          const float4 *st = lgt_stage + (size_t)buf * LGT_PIPE_CHUNKS * T + tid;
          float uf[4][18], ub[4][18], gx[18];
          int nb[4];
#pragma unroll
          for (int mu = MU0; mu < 4; mu++) {
            nb[mu] = cb_shift(in.g, c, mu, -1);
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
        fused_store<float, 1>(a, p, it.t, tile, acc);
      }
      buf ^= 1;
      staged = 1;  // the item's next tile was issued above
    }
    if (abort) break;
    // the item is finished once every thread's stores are: publish it
    __syncthreads();
    if (tid == 0) lgt_red_release_add(ctr + 2 + it.t, 1u);
    cur = nxt;
    staged = nxt_ready;
  }
  cp_async_wait<0>();  // nothing of this thread's in flight at exit
}

// ------------------------------------------------ maximally Abelian gauge
// Complex arithmetic of the subgroup steps (a value per (re, im) pair).
template <typename R>
struct Cx {
  R re, im;
};
template <typename R>
__device__ __forceinline__ Cx<R> cx_at(const R m[18], int a, int b) {
  return Cx<R>{m[LGT_RE(a, b)], m[LGT_IM(a, b)]};
}
template <typename R>
__device__ __forceinline__ Cx<R> cx_mul(Cx<R> x, Cx<R> y) {
  return Cx<R>{x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> cx_mul_conj(Cx<R> x, Cx<R> y) {  // x conj(y)
  return Cx<R>{x.re * y.re + x.im * y.im, x.im * y.re - x.re * y.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> cx_add(Cx<R> x, Cx<R> y) {
  return Cx<R>{x.re + y.re, x.im + y.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> cx_conj(Cx<R> x) {
  return Cx<R>{x.re, -x.im};
}

// The 2x2 blocks a subgroup step needs: F = (g U)_{ab} and B = (U g^dagger)_{ab}
// for a, b in (I, J), with the rows I, J of the running g given as complex
// 3-vectors; the s-terms of the step's vector v (see mag_s above).
template <typename R>
__device__ __forceinline__ void mag_terms(Cx<R> f_ii, Cx<R> f_ij, Cx<R> f_ji, Cx<R> f_jj, Cx<R> b_ii, Cx<R> b_ij,
                                          Cx<R> b_ji, Cx<R> b_jj, R v[3]) {
  mag_s<R>(f_ii.re, f_ii.im, f_ji.re, f_ji.im, R(1), v);    // s((gU)_II, (gU)_JI)
  mag_s<R>(f_ij.re, f_ij.im, f_jj.re, f_jj.im, R(-1), v);   // - s((gU)_IJ, (gU)_JJ)
  mag_s<R>(b_ii.re, -b_ii.im, b_ij.re, -b_ij.im, R(1), v);  // s(conj B_II, conj B_IJ)
  mag_s<R>(b_ji.re, -b_ji.im, b_jj.re, -b_jj.im, R(-1), v); // - s(conj B_JI, conj B_JJ)
}

// A subgroup element as the complex pair (a, b) of [[a, b], [-conj b, conj a]]
// (a = r0 + i r3, b = r2 + i r1): the maximum of v, overrelaxed (Sec. 3.1) or
// squared with probability p (Sec. 3.2).
template <typename R, int ALGO>
__device__ __forceinline__ void mag_element(const R v[3], R omega, uint64_t sr_thr, uint32_t draw, Cx<R> &ea,
                                            Cx<R> &eb) {
  R r0, r1, r2, r3;
  mag_maximum<R>(v, r0, r1, r2, r3);
  if (ALGO == ALGO_OR) {
    r0 = (R(1) - omega) + omega * r0;
    r1 *= omega;
    r2 *= omega;
    r3 *= omega;
    const R inv = rsqrt_t(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    r0 *= inv;
    r1 *= inv;
    r2 *= inv;
    r3 *= inv;
  } else if ((uint64_t)draw < sr_thr) {
    const R a0 = r0 * r0 - (r1 * r1 + r2 * r2 + r3 * r3);
    const R two_r0 = R(2) * r0;
    r1 *= two_r0;
    r2 *= two_r0;
    r3 *= two_r0;
    r0 = a0;
  }
  ea = Cx<R>{r0, r3};
  eb = Cx<R>{r2, r1};
}

// The half-sweep of the maximally Abelian gauge (one thread per site, any
// link format; R = float for the FP32 formats, double for FP64).  The site
// functional is quadratic in g, so K(x) does not suffice: each subgroup step
// needs the (I, J) blocks of g U and U g^dagger of the site's 8 links under the
// running g = R_{s-1} ... R_0.  That g is sparse in a known way -- after step
// (0,1) row 2 is e_2, after step (0,2) row 1 still has no third entry -- so
// the blocks are formed from the links with 2- and 3-term products instead of
// full ones (the links are loaded again for each step: L1/L2 hits, or, with
// STAGED (FP32-12, launch configurations 13 and 14), from the thread's
// shared-memory slots, filled by one batch of cp.async copies as in the staged
// relaxation body).  The first pass also forms X(x) and the estimate:
// sum_a |U_aa|^2 over the 8 links (the parity-0 sums give F_MAG, every link
// counted once) and tr Delta_MAG^2.
template <int FMT, typename R, int ALGO, bool STAGED = false>
__device__ __forceinline__ void sweep_body_mag(const SweepArgs &a, int p, int t, int bx) {
  typedef LinkIO<FMT> IO;
  static_assert(!STAGED || FMT == FMT_F32_12, "the staged layout holds 12-real FP32 links");
  extern __shared__ float4 lgt_stage[];  // STAGED: [LGT_PIPE_CHUNKS][blockDim.x]
  if (a.active && !a.active[t]) return;
  const int j = bx * blockDim.x + threadIdx.x;
  R acc[2] = {R(0), R(0)};
  if (j < a.g.vs_half) {
    const Coords c = coords_in_slice(a.g, p, t, j);
    const int i = t * a.g.vs_half + j;
    const int q = p ^ 1;
    const int T = (int)blockDim.x;
    float4 *slot = lgt_stage + threadIdx.x;
    if constexpr (STAGED) {  // the site's 8 links and G, one wait for memory
      const float4 *L = reinterpret_cast<const float4 *>(a.links);
      const float4 *Gs = reinterpret_cast<const float4 *>(a.G);
#pragma unroll
      for (int mu = 0; mu < 4; mu++) {
        const int nb = cb_shift(a.g, c, mu, -1);
#pragma unroll
        for (int k = 0; k < 3; k++) {
          cp_async16(slot + (mu * 6 + k) * T, L + (size_t)((p * 4 + mu) * 3 + k) * a.g.vh + i);
          cp_async16(slot + (mu * 6 + 3 + k) * T, L + (size_t)((q * 4 + mu) * 3 + k) * a.g.vh + nb);
        }
      }
      if (Gs) {
#pragma unroll
        for (int k = 0; k < 3; k++) cp_async16(slot + (24 + k) * T, Gs + (size_t)(p * 3 + k) * a.g.vh + i);
      }
      cp_async_commit();
      cp_async_wait<0>();
    }
    // the matrix at staged chunk c0 (row 2 rebuilt)
    auto staged = [&](int c0, R m[18]) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const float4 v4 = slot[(c0 + k) * T];
        m[4 * k] = v4.x, m[4 * k + 1] = v4.y, m[4 * k + 2] = v4.z, m[4 * k + 3] = v4.w;
      }
#pragma unroll
      for (int e = 12; e < 18; e++) m[e] = R(0);
      rebuild_row2(m);
    };
    // U_mu(x) and U_mu(x - mu)
    auto load_fwd = [&](int mu, R m[18]) {
      if constexpr (STAGED) staged(mu * 6, m);
      else IO::load(a.links, a.g.vh, p, mu, i, m);
    };
    auto load_bwd = [&](int mu, R m[18]) {
      if constexpr (STAGED) staged(mu * 6 + 3, m);
      else IO::load(a.links, a.g.vh, q, mu, cb_shift(a.g, c, mu, -1), m);
    };
    uint4 draws = make_uint4(0, 0, 0, 0);
    if (ALGO == ALGO_SR) draws = sr_draws(a, c);
    const R omega = (R)a.omega;
    // pass 1: X(x), the estimate, and step (0,1) with g = 1
    R X[18], v[3] = {R(0), R(0), R(0)};
    mat_zero(X);
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
      R u[18];
      load_fwd(mu, u);
      // X += U D^dagger: X_ab += U_ab conj(U_bb)
#pragma unroll
      for (int x = 0; x < 3; x++)
#pragma unroll
        for (int y = 0; y < 3; y++) {
          X[LGT_RE(x, y)] += u[LGT_RE(x, y)] * u[LGT_RE(y, y)] + u[LGT_IM(x, y)] * u[LGT_IM(y, y)];
          X[LGT_IM(x, y)] += u[LGT_IM(x, y)] * u[LGT_RE(y, y)] - u[LGT_RE(x, y)] * u[LGT_IM(y, y)];
        }
#pragma unroll
      for (int x = 0; x < 3; x++) acc[0] += u[LGT_RE(x, x)] * u[LGT_RE(x, x)] + u[LGT_IM(x, x)] * u[LGT_IM(x, x)];
      R w[18];
      load_bwd(mu, w);
      // X -= D^dagger U: X_ab -= conj(U_aa) U_ab
#pragma unroll
      for (int x = 0; x < 3; x++)
#pragma unroll
        for (int y = 0; y < 3; y++) {
          X[LGT_RE(x, y)] -= w[LGT_RE(x, x)] * w[LGT_RE(x, y)] + w[LGT_IM(x, x)] * w[LGT_IM(x, y)];
          X[LGT_IM(x, y)] -= w[LGT_RE(x, x)] * w[LGT_IM(x, y)] - w[LGT_IM(x, x)] * w[LGT_RE(x, y)];
        }
#pragma unroll
      for (int x = 0; x < 3; x++) acc[0] += w[LGT_RE(x, x)] * w[LGT_RE(x, x)] + w[LGT_IM(x, x)] * w[LGT_IM(x, x)];
      mag_terms<R>(cx_at(u, 0, 0), cx_at(u, 0, 1), cx_at(u, 1, 0), cx_at(u, 1, 1), cx_at(w, 0, 0), cx_at(w, 0, 1),
                   cx_at(w, 1, 0), cx_at(w, 1, 1), v);
    }
    R unused;
    violation_of_K(X, unused, acc[1]);  // Delta: traceless part of (X - X^dagger)/(2i)
    Cx<R> a0, b0;
    mag_element<R, ALGO>(v, omega, a.sr_thr, draws.x, a0, b0);
    // pass 2: step (0,2); rows 0 and 2 of g = R_0: (a0, b0, 0) and e_2
    v[0] = v[1] = v[2] = R(0);
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
      R u[18], w[18];
      load_fwd(mu, u);
      load_bwd(mu, w);
      const Cx<R> f00 = cx_add(cx_mul(a0, cx_at(u, 0, 0)), cx_mul(b0, cx_at(u, 1, 0)));
      const Cx<R> f02 = cx_add(cx_mul(a0, cx_at(u, 0, 2)), cx_mul(b0, cx_at(u, 1, 2)));
      // (U g^dagger)_{x0} = U_x0 conj(a0) + U_x1 conj(b0), (U g^dagger)_{x2} = U_x2
      const Cx<R> b00 = cx_add(cx_mul_conj(cx_at(w, 0, 0), a0), cx_mul_conj(cx_at(w, 0, 1), b0));
      const Cx<R> b20 = cx_add(cx_mul_conj(cx_at(w, 2, 0), a0), cx_mul_conj(cx_at(w, 2, 1), b0));
      mag_terms<R>(f00, f02, cx_at(u, 2, 0), cx_at(u, 2, 2), b00, cx_at(w, 0, 2), b20, cx_at(w, 2, 2), v);
    }
    Cx<R> a1, b1;
    mag_element<R, ALGO>(v, omega, a.sr_thr, draws.y, a1, b1);
    // pass 3: step (1,2); row 1 of g = (-conj b0, conj a0, 0), row 2 = (-conj b1 a0, -conj b1 b0, conj a1)
    const Cx<R> g10 = Cx<R>{-b0.re, b0.im}, g11 = cx_conj(a0);
    const Cx<R> nb1 = Cx<R>{-b1.re, b1.im};  // -conj b1
    const Cx<R> g20 = cx_mul(nb1, a0), g21 = cx_mul(nb1, b0), g22 = cx_conj(a1);
    v[0] = v[1] = v[2] = R(0);
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
      R u[18], w[18];
      load_fwd(mu, u);
      load_bwd(mu, w);
      Cx<R> f[2][2], b[2][2];
#pragma unroll
      for (int y = 0; y < 2; y++) {
        const int col = 1 + y;
        f[0][y] = cx_add(cx_mul(g10, cx_at(u, 0, col)), cx_mul(g11, cx_at(u, 1, col)));
        f[1][y] = cx_add(cx_add(cx_mul(g20, cx_at(u, 0, col)), cx_mul(g21, cx_at(u, 1, col))),
                         cx_mul(g22, cx_at(u, 2, col)));
        const int row = 1 + y;
        b[y][0] = cx_add(cx_mul_conj(cx_at(w, row, 0), g10), cx_mul_conj(cx_at(w, row, 1), g11));
        b[y][1] = cx_add(cx_add(cx_mul_conj(cx_at(w, row, 0), g20), cx_mul_conj(cx_at(w, row, 1), g21)),
                         cx_mul_conj(cx_at(w, row, 2), g22));
      }
      mag_terms<R>(f[0][0], f[0][1], f[1][0], f[1][1], b[0][0], b[0][1], b[1][0], b[1][1], v);
    }
    Cx<R> a2, b2;
    mag_element<R, ALGO>(v, omega, a.sr_thr, draws.z, a2, b2);
    // g = R_2 R_1 R_0: rows 0 = a1 (a0, b0, 0) + b1 e_2 and rows 1, 2 from step (1,2)
    R g[18];
    {
      const Cx<R> r0c[3] = {cx_mul(a1, a0), cx_mul(a1, b0), b1};
      const Cx<R> r1c[3] = {g10, g11, Cx<R>{R(0), R(0)}};
      const Cx<R> r2c[3] = {g20, g21, g22};
      const Cx<R> nb2 = Cx<R>{-b2.re, b2.im}, ca2 = cx_conj(a2);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const Cx<R> n1 = cx_add(cx_mul(a2, r1c[k]), cx_mul(b2, r2c[k]));
        const Cx<R> n2 = cx_add(cx_mul(nb2, r1c[k]), cx_mul(ca2, r2c[k]));
        g[LGT_RE(0, k)] = r0c[k].re, g[LGT_IM(0, k)] = r0c[k].im;
        g[LGT_RE(1, k)] = n1.re, g[LGT_IM(1, k)] = n1.im;
        g[LGT_RE(2, k)] = n2.re, g[LGT_IM(2, k)] = n2.im;
      }
    }
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
      const int nb = cb_shift(a.g, c, mu, -1);
      R u[18], r[18];
      load_fwd(mu, u);
      mat_mul(g, u, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, p, mu, i, r);
      load_bwd(mu, u);
      mat_mul_dag(u, g, r);
      if (a.reunit) reunitarise(r);
      IO::store(a.links, a.g.vh, q, mu, nb, r);
    }
    if constexpr (sizeof(R) == sizeof(float)) {
      if (a.G) {
        float gx[18], r[18];
        if constexpr (STAGED) staged(24, gx);
        else GIO::load(a.G, a.g.vh, p, i, gx);
        mat_mul(g, gx, r);
        if (a.reunit) reunitarise(r);
        GIO::store(a.G, a.g.vh, p, i, r);
      }
    }
  }
  fused_store<R, 1>(a, p, t, bx, acc);
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
