// lgt_anchor.cuh -- the anchored polishing sweeps.
//
// After promotion the field U' (FP64) is already close to the gauge-fixed
// field.  The anchored polish keeps U' fixed and relaxes the gauge
// transformation G(x) = 1 + D(x) alone.  With every other G fixed, the local
// maximisation at x sees
//     K(x) = G(x) M(x),   M(x) = sum_mu U'_mu(x) G(x+mu)^+ + U'_mu(x-mu)^+ G(x-mu)^+,
// which is exactly the K(x) that the relaxation sweep of Sec. 3 would gather
// from the transformed links G U' G^+; the update G(x) <- g(x) G(x) is the
// update U_mu(x) <- g U_mu(x), U_mu(x-mu) <- U_mu(x-mu) g^+ of those links.  So
// these are the paper's sweeps with the transformation kept apart from the
// links, which allows each term to be stored at the precision it needs:
//   * M = K0 + C with the constant K0(x) = sum_mu U'_mu(x) + U'_mu(x-mu)^+,
//     formed once in FP64 and stored as FP32 pairs, and the small
//     C(x) = sum_mu U'_mu(x) D(x+mu)^+ + U'_mu(x-mu)^+ D(x-mu)^+, which FP32
//     resolves to |D| 2^-24 from FP32 copies of U' and the high parts of D;
//   * K = M + D(x) M with the small product in FP32;
//   * the rotation angles in FP32 from the pair-precision K, each SU(2)
//     element in FP32 near-identity form (unit to ~|r|^2 2^-24) and
//     delta = g - 1 in FP32 from the small quantities (error ~|delta| 2^-24);
//   * D <- D + delta + delta D accumulated as an FP32 pair, so G stays unitary
//     to ~1e-10 over a polish (what its rounding per update sums to), far below
//     the ~1e-7 violations that theta < 1e-14 resolves; the field is formed as
//     G U' G^+ in FP64 with G orthonormalised in FP64, an exact gauge transform
//     of the input whatever G's rounding.
// Per site update the sweep reads K0 (144 B), 8 FP32 links (384 B), the high
// parts of 8 neighbours' D (384 B, each neighbour's read by 8 sites, so 48 B
// of compulsory traffic) and its own D (96 B), and writes its own D (96 B):
// 768 B of compulsory traffic; no link is written.
#pragma once

#include "lgt_device.cuh"
#include "lgt_pair.cuh"

namespace lgt {

// Row 2 of G = 1 + D from rows 0 and 1 (G in SU(3)): G_2 = conj(G_0 x G_1)
// with G_0 = e_0 + D_0 and G_1 = e_1 + D_1, hence
//   D_2 = conj(e_0 x D_1 + D_0 x e_1 + D_0 x D_1)
//       = conj((-D_02, -D_12, D_00 + D_11) + D_0 x D_1),
// formed from the small entries only (error relative to |D|).
__device__ __forceinline__ void small_row2(float d[18]) {
  float cre[3], cim[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    const float ar1 = d[LGT_RE(0, k1)], ai1 = d[LGT_IM(0, k1)], ar2 = d[LGT_RE(0, k2)], ai2 = d[LGT_IM(0, k2)];
    const float br1 = d[LGT_RE(1, k1)], bi1 = d[LGT_IM(1, k1)], br2 = d[LGT_RE(1, k2)], bi2 = d[LGT_IM(1, k2)];
    cre[k] = (ar1 * br2 - ai1 * bi2) - (ar2 * br1 - ai2 * bi1);
    cim[k] = (ar1 * bi2 + ai1 * br2) - (ar2 * bi1 + ai2 * br1);
  }
  const float lre[3] = {-d[LGT_RE(0, 2)], -d[LGT_RE(1, 2)], d[LGT_RE(0, 0)] + d[LGT_RE(1, 1)]};
  const float lim[3] = {-d[LGT_IM(0, 2)], -d[LGT_IM(1, 2)], d[LGT_IM(0, 0)] + d[LGT_IM(1, 1)]};
#pragma unroll
  for (int k = 0; k < 3; k++) {
    d[LGT_RE(2, k)] = lre[k] + cre[k];
    d[LGT_IM(2, k)] = -(lim[k] + cim[k]);
  }
}

// The same in pair arithmetic (D need not be small: a context may be promoted
// far from convergence).
__device__ __forceinline__ void small_row2_pair(f2 d[18]) {
  f2 cre[3], cim[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    const f2 ar1 = d[LGT_RE(0, k1)], ai1 = d[LGT_IM(0, k1)], ar2 = d[LGT_RE(0, k2)], ai2 = d[LGT_IM(0, k2)];
    const f2 br1 = d[LGT_RE(1, k1)], bi1 = d[LGT_IM(1, k1)], br2 = d[LGT_RE(1, k2)], bi2 = d[LGT_IM(1, k2)];
    // a_k1 b_k2 - a_k2 b_k1
    cre[k] = pair_dot4(ar1, br2, pair_neg(ai1), bi2, pair_neg(ar2), br1, ai2, bi1);
    cim[k] = pair_dot4(ar1, bi2, ai1, br2, pair_neg(ar2), bi1, pair_neg(ai2), br1);
  }
  const f2 lre[3] = {pair_neg(d[LGT_RE(0, 2)]), pair_neg(d[LGT_RE(1, 2)]), pair_add(d[LGT_RE(0, 0)], d[LGT_RE(1, 1)])};
  const f2 lim[3] = {pair_neg(d[LGT_IM(0, 2)]), pair_neg(d[LGT_IM(1, 2)]), pair_add(d[LGT_IM(0, 0)], d[LGT_IM(1, 1)])};
#pragma unroll
  for (int k = 0; k < 3; k++) {
    d[LGT_RE(2, k)] = pair_add(lre[k], cre[k]);
    d[LGT_IM(2, k)] = pair_neg(pair_add(lim[k], cim[k]));
  }
}

// D = G - 1: rows 0 and 1 as FP32 pairs; the high parts in one array and the
// low parts in a second, each laid out as the G of the bulk phase (chunk k of
// parity p at (p * 3 + k) * vh + i), so a neighbour's term reads 48 B.
struct DIO {
  static __device__ __forceinline__ size_t lo_offset(int vh) { return (size_t)6 * vh; }
  static __device__ __forceinline__ void load_hi(const void *base, int vh, int p, int i, float d[18]) {
    const float4 *b4 = reinterpret_cast<const float4 *>(base) + (size_t)(p * 3) * vh + i;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const float4 v = __ldg(b4 + (size_t)k * vh);
      d[4 * k] = v.x;
      d[4 * k + 1] = v.y;
      d[4 * k + 2] = v.z;
      d[4 * k + 3] = v.w;
    }
    small_row2(d);
  }
  static __device__ __forceinline__ void load_pair(const void *base, int vh, int p, int i, f2 d[18]) {
    const float4 *h4 = reinterpret_cast<const float4 *>(base) + (size_t)(p * 3) * vh + i;
    const float4 *l4 = h4 + lo_offset(vh);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const float4 h = __ldg(h4 + (size_t)k * vh), l = __ldg(l4 + (size_t)k * vh);
      d[4 * k] = {h.x, l.x};
      d[4 * k + 1] = {h.y, l.y};
      d[4 * k + 2] = {h.z, l.z};
      d[4 * k + 3] = {h.w, l.w};
    }
    small_row2_pair(d);
  }
  // rows 0, 1 as pairs only (row 2 left unset)
  static __device__ __forceinline__ void load_pair_rows(const void *base, int vh, int p, int i, f2 d[12]) {
    const float4 *h4 = reinterpret_cast<const float4 *>(base) + (size_t)(p * 3) * vh + i;
    const float4 *l4 = h4 + lo_offset(vh);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const float4 h = __ldg(h4 + (size_t)k * vh), l = __ldg(l4 + (size_t)k * vh);
      d[4 * k] = {h.x, l.x};
      d[4 * k + 1] = {h.y, l.y};
      d[4 * k + 2] = {h.z, l.z};
      d[4 * k + 3] = {h.w, l.w};
    }
  }
  static __device__ __forceinline__ void store_pair(void *base, int vh, int p, int i, const f2 d[18]) {
    float4 *h4 = reinterpret_cast<float4 *>(base) + (size_t)(p * 3) * vh + i;
    float4 *l4 = h4 + lo_offset(vh);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      h4[(size_t)k * vh] = make_float4(d[4 * k].hi, d[4 * k + 1].hi, d[4 * k + 2].hi, d[4 * k + 3].hi);
      l4[(size_t)k * vh] = make_float4(d[4 * k].lo, d[4 * k + 1].lo, d[4 * k + 2].lo, d[4 * k + 3].lo);
    }
  }
};

// K0(x): one 3x3 complex matrix per site as FP32 pairs, 9 float4 chunks
// (chunk c of parity p at (p * 9 + c) * vh + i).
struct K0IO {
  static __device__ __forceinline__ void load(const void *base, int vh, int p, int i, f2 m[18]) {
    const float4 *b = reinterpret_cast<const float4 *>(base) + (size_t)(p * 9) * vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const float4 v = __ldg(b + (size_t)c * vh);
      m[2 * c] = {v.x, v.y};
      m[2 * c + 1] = {v.z, v.w};
    }
  }
  static __device__ __forceinline__ void store(void *base, int vh, int p, int i, const f2 m[18]) {
    float4 *b = reinterpret_cast<float4 *>(base) + (size_t)(p * 9) * vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++)
      b[(size_t)c * vh] = make_float4(m[2 * c].hi, m[2 * c].lo, m[2 * c + 1].hi, m[2 * c + 1].lo);
  }
};

// c += a b^+
__device__ __forceinline__ void acc_mul_dag(const float a[18], const float b[18], float c[18]) {
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      float re = c[LGT_RE(i, j)], im = c[LGT_IM(i, j)];
#pragma unroll
      for (int k = 0; k < 3; k++) {  // a_ik conj(b_jk)
        re += a[LGT_RE(i, k)] * b[LGT_RE(j, k)] + a[LGT_IM(i, k)] * b[LGT_IM(j, k)];
        im += a[LGT_IM(i, k)] * b[LGT_RE(j, k)] - a[LGT_RE(i, k)] * b[LGT_IM(j, k)];
      }
      c[LGT_RE(i, j)] = re;
      c[LGT_IM(i, j)] = im;
    }
}

// c += a^+ b^+ = (b a)^+
__device__ __forceinline__ void acc_dag_mul_dag(const float a[18], const float b[18], float c[18]) {
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      float re = c[LGT_RE(i, j)], im = c[LGT_IM(i, j)];
#pragma unroll
      for (int k = 0; k < 3; k++) {  // conj(a_ki) conj(b_jk) = conj(b_jk a_ki)
        re += b[LGT_RE(j, k)] * a[LGT_RE(k, i)] - b[LGT_IM(j, k)] * a[LGT_IM(k, i)];
        im -= b[LGT_RE(j, k)] * a[LGT_IM(k, i)] + b[LGT_IM(j, k)] * a[LGT_RE(k, i)];
      }
      c[LGT_RE(i, j)] = re;
      c[LGT_IM(i, j)] = im;
    }
}

// Sec. 3 local update for the anchored polish: the block projections from the
// pair-precision K (no cancellation loss near convergence), the rotation
// angles and each subgroup element in FP32 near-identity form (1 + e0, r):
// unit to ~|r|^2 2^-24, i.e. ~1e-15 for the |r| <~ 1e-4 of polishing (only G's
// unitarity depends on it, and G is orthonormalised in FP64 when the field is
// formed).  W is steered between subgroups in FP32 as in the pair polish.
template <int ALGO>
__device__ __forceinline__ void anchor_local_update(f2 W[18], RotF rf[3], float omega, uint64_t sr_thr, uint4 draws) {
#pragma unroll
  for (int s = 0; s < 3; s++) {
    const int i = (s == 2) ? 1 : 0;
    const int j = (s == 0) ? 1 : 2;
    const float q0 = pair_to_float(pair_add(W[LGT_RE(i, i)], W[LGT_RE(j, j)]));
    const float q1 = pair_to_float(pair_add(W[LGT_IM(i, j)], W[LGT_IM(j, i)]));
    const float q2 = pair_to_float(pair_add(W[LGT_RE(i, j)], pair_neg(W[LGT_RE(j, i)])));
    const float q3 = pair_to_float(pair_add(W[LGT_IM(i, i)], pair_neg(W[LGT_IM(j, j)])));
    const uint32_t d = s == 0 ? draws.x : (s == 1 ? draws.y : draws.z);
    rf[s] = subgroup_rotation<ALGO>(q0, q1, q2, q3, omega, (uint64_t)d < sr_thr);
    if (s == 0) steer_rows<0, 1>(W, rf[s]);
    if (s == 1) steer_rows<0, 2>(W, rf[s]);
  }
}

// delta = g - 1 for g = R2 R1 R0 from FP32 near-identity elements, written with
// the small quantities only (the structure of pair_delta, in FP32): error
// ~|delta| 2^-24.
__device__ __forceinline__ void float_delta(const RotF rf[3], float d[18]) {
  // deviation blocks of element s: a = e0 + i r3, B = r2 + i r1, C = -r2 + i r1, d = e0 - i r3
  float ar[3], ai[3], br[3], bi[3], cr[3], ci[3], dr[3], di[3];
#pragma unroll
  for (int s = 0; s < 3; s++) {
    ar[s] = rf[s].e0, ai[s] = rf[s].r3;
    br[s] = rf[s].r2, bi[s] = rf[s].r1;
    cr[s] = -rf[s].r2, ci[s] = rf[s].r1;
    dr[s] = rf[s].e0, di[s] = -rf[s].r3;
  }
  auto mul = [](float xr, float xi, float yr, float yi, float &zr, float &zi) {
    zr = xr * yr - xi * yi;
    zi = xr * yi + xi * yr;
  };
  float t0r, t0i, t1r, t1i;
  // C1 A0 = C1 + C1 a0, C1 B0
  mul(cr[1], ci[1], ar[0], ai[0], t0r, t0i);
  const float c1a0r = cr[1] + t0r, c1a0i = ci[1] + t0i;
  float c1b0r, c1b0i;
  mul(cr[1], ci[1], br[0], bi[0], c1b0r, c1b0i);
  // row 0: A1 A0 - 1, A1 B0, B1
  mul(ar[1], ai[1], ar[0], ai[0], t0r, t0i);
  d[LGT_RE(0, 0)] = (ar[1] + ar[0]) + t0r, d[LGT_IM(0, 0)] = (ai[1] + ai[0]) + t0i;
  mul(ar[1], ai[1], br[0], bi[0], t0r, t0i);
  d[LGT_RE(0, 1)] = br[0] + t0r, d[LGT_IM(0, 1)] = bi[0] + t0i;
  d[LGT_RE(0, 2)] = br[1], d[LGT_IM(0, 2)] = bi[1];
  // row 1: A2 C0 + B2 C1 A0, A2 D0 + B2 C1 B0 - 1, B2 D1
  mul(ar[2], ai[2], cr[0], ci[0], t0r, t0i);
  mul(br[2], bi[2], c1a0r, c1a0i, t1r, t1i);
  d[LGT_RE(1, 0)] = (cr[0] + t0r) + t1r, d[LGT_IM(1, 0)] = (ci[0] + t0i) + t1i;
  mul(ar[2], ai[2], dr[0], di[0], t0r, t0i);
  mul(br[2], bi[2], c1b0r, c1b0i, t1r, t1i);
  d[LGT_RE(1, 1)] = ((ar[2] + dr[0]) + t0r) + t1r, d[LGT_IM(1, 1)] = ((ai[2] + di[0]) + t0i) + t1i;
  mul(br[2], bi[2], dr[1], di[1], t0r, t0i);
  d[LGT_RE(1, 2)] = br[2] + t0r, d[LGT_IM(1, 2)] = bi[2] + t0i;
  // row 2: C2 C0 + D2 C1 A0, C2 D0 + D2 C1 B0, D2 D1 - 1
  mul(cr[2], ci[2], cr[0], ci[0], t0r, t0i);
  mul(dr[2], di[2], c1a0r, c1a0i, t1r, t1i);
  d[LGT_RE(2, 0)] = (t0r + c1a0r) + t1r, d[LGT_IM(2, 0)] = (t0i + c1a0i) + t1i;
  mul(cr[2], ci[2], dr[0], di[0], t0r, t0i);
  mul(dr[2], di[2], c1b0r, c1b0i, t1r, t1i);
  d[LGT_RE(2, 1)] = (cr[2] + t0r) + (c1b0r + t1r), d[LGT_IM(2, 1)] = (ci[2] + t0i) + (c1b0i + t1i);
  mul(dr[2], di[2], dr[1], di[1], t0r, t0i);
  d[LGT_RE(2, 2)] = (dr[2] + dr[1]) + t0r, d[LGT_IM(2, 2)] = (di[2] + di[1]) + t0i;
}

// G <- g G on rows 0 and 1: D <- D + delta + delta D, D a pair (rows 0, 1),
// delta and the small product delta D in FP32 (dh: D's high parts with row 2)
__device__ __forceinline__ void d_update_lite(f2 D[12], const float dh[18], const float d[18]) {
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      float re = 0.0f, im = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        re += d[LGT_RE(i, k)] * dh[LGT_RE(k, j)] - d[LGT_IM(i, k)] * dh[LGT_IM(k, j)];
        im += d[LGT_RE(i, k)] * dh[LGT_IM(k, j)] + d[LGT_IM(i, k)] * dh[LGT_RE(k, j)];
      }
      D[LGT_RE(i, j)] = pair_add(pair_add(D[LGT_RE(i, j)], f2{d[LGT_RE(i, j)], 0.0f}), f2{re, 0.0f});
      D[LGT_IM(i, j)] = pair_add(pair_add(D[LGT_IM(i, j)], f2{d[LGT_IM(i, j)], 0.0f}), f2{im, 0.0f});
    }
}

}  // namespace lgt
