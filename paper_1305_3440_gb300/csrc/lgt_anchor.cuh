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
//   * g from the pair-precision K as in the pair polish (FP32 angles, each SU(2)
//     element unit to ~2^-48, delta = g - 1 in pair precision);
//   * D <- D + delta + delta D in pair arithmetic, so G stays unitary to
//     ~2^-48 and the final U = G U' G^+ (formed in FP64) is a gauge transform
//     of the input.
// Per site update the sweep reads K0 (144 B), 8 FP32 links (384 B), the high
// parts of 8 neighbours' D (384 B) and its own D (96 B), and writes its own D
// (96 B): 1104 B, no link is written.
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

// D <- D + delta + delta D on rows 0 and 1 (G <- g G), pair arithmetic
__device__ __forceinline__ void d_update(f2 D[18], const f2 d[18]) {
  f2 r[12];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      f2 c[6], x[6];
#pragma unroll
      for (int k = 0; k < 3; k++) {  // re: d_re D_re - d_im D_im
        c[2 * k] = d[LGT_RE(i, k)];
        x[2 * k] = D[LGT_RE(k, j)];
        c[2 * k + 1] = pair_neg(d[LGT_IM(i, k)]);
        x[2 * k + 1] = D[LGT_IM(k, j)];
      }
      r[LGT_RE(i, j)] = pair_axpy6(pair_add(D[LGT_RE(i, j)], d[LGT_RE(i, j)]), c, x);
#pragma unroll
      for (int k = 0; k < 3; k++) {  // im: d_re D_im + d_im D_re
        c[2 * k] = d[LGT_RE(i, k)];
        x[2 * k] = D[LGT_IM(k, j)];
        c[2 * k + 1] = d[LGT_IM(i, k)];
        x[2 * k + 1] = D[LGT_RE(k, j)];
      }
      r[LGT_IM(i, j)] = pair_axpy6(pair_add(D[LGT_IM(i, j)], d[LGT_IM(i, j)]), c, x);
    }
#pragma unroll
  for (int e = 0; e < 12; e++) D[e] = r[e];
}

}  // namespace lgt
