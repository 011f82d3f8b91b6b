// lgt_measure.cuh -- bodies of the exact measurement (Sec. 2: F, theta,
// plaquette, per-slice F_t and theta_t) and of the fused estimate's finishing
// reduction, shared by the single-lattice and the batched kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lgt_device.cuh"
#include "lgt_internal.h"
#include "lgt_pair.cuh"

namespace lgt {



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
    if (a.mag) {  // maximally Abelian gauge: sum_a |U_aa|^2 and X(x) (see lgt_device.cuh)
      for (int mu = 0; mu < 4; mu++) {
        double u[18], y[18];
        load_d<FMT>(a.links, a.g.vh, p, mu, i, u);
#pragma unroll
        for (int x = 0; x < 3; x++) {
          v[0] += u[LGT_RE(x, x)] * u[LGT_RE(x, x)] + u[LGT_IM(x, x)] * u[LGT_IM(x, x)];
#pragma unroll
          for (int z = 0; z < 3; z++) {  // y = U D^dagger
            y[LGT_RE(x, z)] = u[LGT_RE(x, z)] * u[LGT_RE(z, z)] + u[LGT_IM(x, z)] * u[LGT_IM(z, z)];
            y[LGT_IM(x, z)] = u[LGT_IM(x, z)] * u[LGT_RE(z, z)] - u[LGT_RE(x, z)] * u[LGT_IM(z, z)];
          }
        }
        acc_antiherm(XL, y, 1.0);
        load_d<FMT>(a.links, a.g.vh, q, mu, cb_shift(a.g, c, mu, -1), u);
#pragma unroll
        for (int x = 0; x < 3; x++)
#pragma unroll
          for (int z = 0; z < 3; z++) {  // y = D^dagger U
            y[LGT_RE(x, z)] = u[LGT_RE(x, x)] * u[LGT_RE(x, z)] + u[LGT_IM(x, x)] * u[LGT_IM(x, z)];
            y[LGT_IM(x, z)] = u[LGT_RE(x, x)] * u[LGT_IM(x, z)] - u[LGT_IM(x, x)] * u[LGT_RE(x, z)];
          }
        acc_antiherm(XL, y, -1.0);
      }
      v[2] = traceless_norm(XL);
    }
    for (int mu = 0; mu < 4 && !a.mag; mu++) {
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
    if (!a.mag) {
      v[2] = traceless_norm(XL);
      v[3] = traceless_norm(XS);
    }
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
    // Each thread adds the slots w, w + blockDim.x, ... in that order.  The slots
    // sit in L2 (half of them on the other die), so the loads of eight
    // consecutive terms are issued before any of them is added.
    const int bd = (int)blockDim.x;
    int w = threadIdx.x;
    for (; w + 7 * bd < a.nw; w += 8 * bd) {
      double2 x0[8], x1[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        x0[u] = __ldcg(p0 + w + u * bd);
        x1[u] = __ldcg(p1 + w + u * bd);
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        v[0] += x0[u].x;
        v[1] += x0[u].y + x1[u].y;
      }
    }
    for (; w < a.nw; w += bd) {
      const double2 x0 = __ldcg(p0 + w), x1 = __ldcg(p1 + w);
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
  if (!am_last) return;
  __threadfence();
  // The last block forms the totals in slice order.  Its threads first load
  // the slices' sums and form each slice's F_t and theta_t side by side (one L2
  // round trip and one FP64 division latency instead of one per slice), then
  // thread 0 adds them in slice order: the same sums as a serial loop over the
  // slices, bit for bit.
  constexpr int CH = 256;
  __shared__ double sl[4 * CH];
  __shared__ uint8_t act[CH];
  const double vs = 2.0 * (double)a.g.vs_half, vol = 2.0 * (double)a.g.vh;
  const double nd = a.gauge == GAUGE_COULOMB ? 3.0 : 4.0;
  double fsum = 0.0, tsum = 0.0, tmax = 0.0, ftot = 0.0, ttot = 0.0;
  int nact = 0;
  for (int t0 = 0; t0 < a.g.nt; t0 += CH) {
    const int n = a.g.nt - t0 < CH ? a.g.nt - t0 : CH;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const double rk = __ldcg(a.slice + 2 * (t0 + k)), th2 = __ldcg(a.slice + 2 * (t0 + k) + 1);
      const double th = th2 / (3.0 * vs);
      sl[4 * k] = rk;
      sl[4 * k + 1] = th2;
      sl[4 * k + 2] = rk / (3.0 * nd * vs);
      sl[4 * k + 3] = th;
      if (a.coulomb_target >= 0.0) a.active[t0 + k] = th >= a.coulomb_target ? 1 : 0;
      act[k] = a.active[t0 + k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 0; k < n; k++) {
        ftot += sl[4 * k];
        ttot += sl[4 * k + 1];
        fsum += sl[4 * k + 2];
        const double th = sl[4 * k + 3];
        tsum += th;
        tmax = th > tmax ? th : tmax;
        nact += act[k];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  a.totals[TOT_F_LANDAU] = ftot / (3.0 * nd * vol);
  a.totals[TOT_THETA_LANDAU] = ttot / (3.0 * vol);
  a.totals[TOT_PLAQ] = 0.0;
  a.totals[TOT_F_COULOMB] = fsum / (double)a.g.nt;
  a.totals[TOT_THETA_COULOMB_MAX] = tmax;
  a.totals[TOT_THETA_COULOMB_MEAN] = tsum / (double)a.g.nt;
  a.totals[TOT_ACTIVE_SLICES] = (double)nact;
  *a.counter = 0u;
}

}  // namespace lgt
