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
#include "lgt_pair.cuh"

namespace lgt {



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
  fused_store<float>(a, p, t, bx, acc);
}


template <int FMT, int GAUGE, int ALGO>
__device__ __forceinline__ void sweep_dispatch(const SweepArgs &a, int p, int t, int bx, int nbx) {
  if (FMT == FMT_F64) sweep_body_f64<GAUGE, ALGO>(a, p, t, bx, nbx);
  else if (FMT == FMT_PAIR) sweep_body_pair<GAUGE, ALGO>(a, p, t, bx, nbx);
  else sweep_body_f32<(FMT == FMT_F32_12 ? FMT_F32_12 : FMT_F32_18), GAUGE, ALGO>(a, p, t, bx, nbx);
}

}  // namespace lgt
