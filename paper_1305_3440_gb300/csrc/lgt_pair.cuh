// lgt_pair.cuh -- FP32-pair ("double-float") arithmetic and the pair-precision
// local update used by the polishing sweeps.
//
// A real is held as the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2 (Dekker 1971, Knuth TAOCP vol. 2: the error-free
// transformations TwoSum and, with a fused multiply-add, TwoProd), which gives a
// ~48-bit significand using only the FP32 pipe.  On this part FP64 arithmetic
// and FP64<->FP32 conversion both run at ~2 operations/clock/SM against ~128
// for FP32, so pair arithmetic is the fast way to carry more than FP32
// precision.
//
// The polishing update keeps two concerns apart:
//   * the rotation angles (which SU(2) element to apply) are chosen in FP32
//     from the pair-precision K(x); a slightly suboptimal angle is still a
//     gauge transformation and only costs optimality;
//   * every SU(2) element is the FP32 quaternion rescaled to unit length in
//     pair arithmetic, so it is unitary to ~2^-48 at any rotation size, and it
//     is applied to the links as R = 1 + rho in pair arithmetic.  The field
//     therefore stays an exact (to ~2^-48) gauge transform of its input.
#pragma once

#include "lgt_device.cuh"

namespace lgt {

struct f2 {
  float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ f2 quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// a + b in pair arithmetic (absolute error ~2^-48 max(|a|, |b|))
__device__ __forceinline__ f2 pair_add(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, e);
}

__device__ __forceinline__ f2 pair_neg(f2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ float pair_to_float(f2 a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ f2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ f2 pair_mul(f2 a, f2 b) {
  f2 p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}

// 1/sqrt of a positive pair: correctly rounded FP32 root, one Newton step in pairs
__device__ __forceinline__ f2 pair_rsqrt(f2 x) {
  const float y = __frsqrt_rn(x.hi);
  const f2 yy = two_prod(y, y);
  const f2 r = pair_add(f2{1.0f, 0.0f}, pair_neg(pair_mul(x, yy)));  // 1 - x y^2
  return quick_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), pair_to_float(r)));
}

// sum_k c[k] * x[k] for pair coefficients and pair values: exact products of
// the high parts (TwoProd via fma), the low-part products folded in with one
// rounding each
__device__ __forceinline__ f2 pair_dot4(f2 c0, f2 x0, f2 c1, f2 x1, f2 c2, f2 x2, f2 c3, f2 x3) {
  const float p0 = __fmul_rn(c0.hi, x0.hi), p1 = __fmul_rn(c1.hi, x1.hi);
  const float p2 = __fmul_rn(c2.hi, x2.hi), p3 = __fmul_rn(c3.hi, x3.hi);
  float e = __fmaf_rn(c0.hi, x0.hi, -p0);
  e = __fadd_rn(e, __fmaf_rn(c1.hi, x1.hi, -p1));
  e = __fadd_rn(e, __fmaf_rn(c2.hi, x2.hi, -p2));
  e = __fadd_rn(e, __fmaf_rn(c3.hi, x3.hi, -p3));
  e = __fmaf_rn(c0.hi, x0.lo, e);
  e = __fmaf_rn(c1.hi, x1.lo, e);
  e = __fmaf_rn(c2.hi, x2.lo, e);
  e = __fmaf_rn(c3.hi, x3.lo, e);
  e = __fmaf_rn(c0.lo, x0.hi, e);
  e = __fmaf_rn(c1.lo, x1.hi, e);
  e = __fmaf_rn(c2.lo, x2.hi, e);
  e = __fmaf_rn(c3.lo, x3.hi, e);
  f2 s = two_sum(p0, p1);
  e = __fadd_rn(e, s.lo);
  s = two_sum(s.hi, p2);
  e = __fadd_rn(e, s.lo);
  s = two_sum(s.hi, p3);
  e = __fadd_rn(e, s.lo);
  return quick_two_sum(s.hi, e);
}

// base + sum of six products of pairs, in one compensated chain
__device__ __forceinline__ f2 pair_axpy6(f2 base, const f2 c[6], const f2 x[6]) {
  float s = base.hi, e = base.lo;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const float p = __fmul_rn(c[k].hi, x[k].hi);
    e = __fadd_rn(e, __fmaf_rn(c[k].hi, x[k].hi, -p));
    e = __fmaf_rn(c[k].hi, x[k].lo, e);
    e = __fmaf_rn(c[k].lo, x[k].hi, e);
    const f2 t = two_sum(s, p);
    s = t.hi;
    e = __fadd_rn(e, t.lo);
  }
  return quick_two_sum(s, e);
}

// Running pair sum with the normalisation deferred to the end.
struct PairAcc {
  float s, e;
};

__device__ __forceinline__ void acc_add_pair(PairAcc &a, f2 x) {
  const f2 t = two_sum(a.s, x.hi);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, x.lo));
}

__device__ __forceinline__ f2 acc_value(const PairAcc &a) { return quick_two_sum(a.s, a.e); }

template <>
struct LinkIO<FMT_PAIR> {
  static __device__ __forceinline__ void load(const void *base, int vh, int p, int mu, int i, f2 m[18]) {
    const float4 *b = reinterpret_cast<const float4 *>(base) + (size_t)((p * 4 + mu) * 9) * vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const float4 v = __ldg(b + (size_t)c * vh);
      m[2 * c] = {v.x, v.y};
      m[2 * c + 1] = {v.z, v.w};
    }
  }
  static __device__ __forceinline__ void store(void *base, int vh, int p, int mu, int i, const f2 m[18]) {
    float4 *b = reinterpret_cast<float4 *>(base) + (size_t)((p * 4 + mu) * 9) * vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) b[(size_t)c * vh] = make_float4(m[2 * c].hi, m[2 * c].lo, m[2 * c + 1].hi, m[2 * c + 1].lo);
  }
};

// One subgroup element (r0, r1, r2, r3) in pair precision, r0 = 1 + e0: the
// FP32 quaternion rescaled to unit length in pair arithmetic, so the element is
// unitary to ~2^-48 at any rotation size (well conditioned even at r0 ~ 0).
struct Rot {
  f2 e0, r1, r2, r3;
};

// FP32 choice of the element, before its pair-precision r0
struct RotF {
  float e0, r1, r2, r3;
};

__device__ __forceinline__ Rot exact_rotation(const RotF &f) {
  const f2 r0 = two_sum(1.0f, f.e0);  // 1 + e0 exactly
  const f2 n2 = pair_add(pair_add(pair_mul(r0, r0), two_prod(f.r1, f.r1)),
                         pair_add(two_prod(f.r2, f.r2), two_prod(f.r3, f.r3)));
  const f2 inv = pair_rsqrt(n2);
  Rot r;
  r.e0 = pair_add(pair_mul(r0, inv), f2{-1.0f, 0.0f});
  r.r1 = pair_mul(f2{f.r1, 0.0f}, inv);
  r.r2 = pair_mul(f2{f.r2, 0.0f}, inv);
  r.r3 = pair_mul(f2{f.r3, 0.0f}, inv);
  return r;
}

// Sec. 3 closed-form SU(2) maximum of the projection (q0, q) (any positive
// scale), then Sec. 3.1 first-order overrelaxation or Sec. 3.2 squaring, all
// in the near-identity form r = (1 + e0, r_vec).
template <int ALGO>
__device__ __forceinline__ RotF subgroup_rotation(float q0, float q1, float q2, float q3, float omega, bool square) {
  const float v2 = q1 * q1 + q2 * q2 + q3 * q3;
  const float n2 = q0 * q0 + v2;
  RotF r = {0.0f, 0.0f, 0.0f, 0.0f};
  if (n2 > 0.0f) {
    const float inv = rsqrtf(n2);
    const float n = n2 * inv;
    r.r1 = -q1 * inv;
    r.r2 = -q2 * inv;
    r.r3 = -q3 * inv;
    // r0 - 1 = (q0 - |q|)/|q| = -|q_vec|^2 / (|q| (q0 + |q|)) without cancellation
    r.e0 = q0 > 0.0f ? -v2 * inv / (q0 + n) : q0 * inv - 1.0f;
  }
  if (ALGO == ALGO_OR) {
    // (1 - omega) 1 + omega r = (1 + omega e0, omega r_vec), rescaled to |.| = 1
    const float a0 = omega * r.e0;
    const float s1 = omega * r.r1, s2 = omega * r.r2, s3 = omega * r.r3;
    const float t = a0 * (2.0f + a0) + (s1 * s1 + s2 * s2 + s3 * s3);  // |s|^2 - 1
    const float sq = sqrtf(1.0f + t);
    const float inv = 1.0f / sq;
    r.e0 = a0 * inv - t * inv / (1.0f + sq);  // (1 + a0)/|s| - 1
    r.r1 = s1 * inv;
    r.r2 = s2 * inv;
    r.r3 = s3 * inv;
  } else if (square) {  // r^2 = (r0^2 - |r|^2, 2 r0 r_vec)
    const float vv = r.r1 * r.r1 + r.r2 * r.r2 + r.r3 * r.r3;
    const float f2x = 2.0f * (1.0f + r.e0);
    r.e0 = r.e0 * (2.0f + r.e0) - vv;
    r.r1 *= f2x;
    r.r2 *= f2x;
    r.r3 *= f2x;
  }
  return r;
}

// rows (i, j) of m <- R rows, R = [[r0 + i r3, r2 + i r1], [-r2 + i r1, r0 - i r3]],
// written as m + rho m with rho = R - 1 and the increment in pair arithmetic
template <int I, int J>
__device__ __forceinline__ void rotate_rows(f2 m[18], const Rot &r) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const f2 xi = m[LGT_RE(I, c)], yi = m[LGT_IM(I, c)];
    const f2 xj = m[LGT_RE(J, c)], yj = m[LGT_IM(J, c)];
    const f2 e = r.e0, r1 = r.r1, r2 = r.r2, r3 = r.r3, n1 = pair_neg(r.r1), n2 = pair_neg(r.r2), n3 = pair_neg(r.r3);
    // (e0 + i r3) (xi + i yi) + (r2 + i r1) (xj + i yj)
    m[LGT_RE(I, c)] = pair_add(xi, pair_dot4(e, xi, n3, yi, r2, xj, n1, yj));
    m[LGT_IM(I, c)] = pair_add(yi, pair_dot4(e, yi, r3, xi, r2, yj, r1, xj));
    // (-r2 + i r1) (xi + i yi) + (e0 - i r3) (xj + i yj)
    m[LGT_RE(J, c)] = pair_add(xj, pair_dot4(n2, xi, n1, yi, e, xj, r3, yj));
    m[LGT_IM(J, c)] = pair_add(yj, pair_dot4(n2, yi, r1, xi, e, yj, n3, xj));
  }
}

// W <- W + rho W on rows (i, j) with the increment in FP32 (it only steers the
// next subgroup's choice; the applied rotations are exact regardless)
template <int I, int J>
__device__ __forceinline__ void steer_rows(f2 W[18], const RotF &r) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const float xi = W[LGT_RE(I, c)].hi, yi = W[LGT_IM(I, c)].hi;
    const float xj = W[LGT_RE(J, c)].hi, yj = W[LGT_IM(J, c)].hi;
    W[LGT_RE(I, c)] = pair_add(W[LGT_RE(I, c)], f2{r.e0 * xi - r.r3 * yi + r.r2 * xj - r.r1 * yj, 0.0f});
    W[LGT_IM(I, c)] = pair_add(W[LGT_IM(I, c)], f2{r.e0 * yi + r.r3 * xi + r.r2 * yj + r.r1 * xj, 0.0f});
    W[LGT_RE(J, c)] = pair_add(W[LGT_RE(J, c)], f2{-r.r2 * xi - r.r1 * yi + r.e0 * xj + r.r3 * yj, 0.0f});
    W[LGT_IM(J, c)] = pair_add(W[LGT_IM(J, c)], f2{-r.r2 * yi + r.r1 * xi + r.e0 * yj - r.r3 * xj, 0.0f});
  }
}

// Sec. 3 local update at pair precision: the three subgroup elements for
// W = K (the block projections taken from the pair values without
// cancellation loss).
template <int ALGO>
__device__ __forceinline__ void pair_local_update(f2 W[18], Rot rot[3], float omega, uint64_t sr_thr, uint4 draws) {
#pragma unroll
  for (int s = 0; s < 3; s++) {
    const int i = (s == 2) ? 1 : 0;
    const int j = (s == 0) ? 1 : 2;
    const float q0 = pair_to_float(pair_add(W[LGT_RE(i, i)], W[LGT_RE(j, j)]));
    const float q1 = pair_to_float(pair_add(W[LGT_IM(i, j)], W[LGT_IM(j, i)]));
    const float q2 = pair_to_float(pair_add(W[LGT_RE(i, j)], pair_neg(W[LGT_RE(j, i)])));
    const float q3 = pair_to_float(pair_add(W[LGT_IM(i, i)], pair_neg(W[LGT_IM(j, j)])));
    const uint32_t d = s == 0 ? draws.x : (s == 1 ? draws.y : draws.z);
    const RotF rf = subgroup_rotation<ALGO>(q0, q1, q2, q3, omega, (uint64_t)d < sr_thr);
    rot[s] = exact_rotation(rf);
    if (s == 0) steer_rows<0, 1>(W, rf);
    if (s == 1) steer_rows<0, 2>(W, rf);
  }
}

// complex pair numbers
struct c2 {
  f2 re, im;
};

__device__ __forceinline__ c2 cmul2(c2 a, c2 b) {
  return {pair_add(pair_mul(a.re, b.re), pair_neg(pair_mul(a.im, b.im))),
          pair_add(pair_mul(a.re, b.im), pair_mul(a.im, b.re))};
}

__device__ __forceinline__ c2 cadd2(c2 a, c2 b) { return {pair_add(a.re, b.re), pair_add(a.im, b.im)}; }

// The deviation from the identity of a subgroup element r, as its 2x2 block
// [[a, B], [C, d]] with a = A - 1 = e0 + i r3, B = r2 + i r1, C = -r2 + i r1,
// d = D - 1 = e0 - i r3 (all small near convergence).
__device__ __forceinline__ void rot_small(const Rot &r, c2 &a, c2 &B, c2 &C, c2 &d) {
  a = {r.e0, r.r3};
  B = {r.r2, r.r1};
  C = {pair_neg(r.r2), r.r1};
  d = {r.e0, pair_neg(r.r3)};
}

// delta = g - 1 for g = R2 R1 R0 (subgroups (0,1), (0,2), (1,2)), in pair
// precision, written with the small quantities only so that its error is
// relative to |delta| (no 1 is added and taken away):
//   with A = 1 + a, D = 1 + d for each element,
//   R1 R0 = [[A1 A0, A1 B0, B1], [C0, D0, 0], [C1 A0, C1 B0, D1]],
//   g row 0 = R1R0 row 0, row 1 = A2 (R1R0 row 1) + B2 (row 2),
//   row 2 = C2 (row 1) + D2 (row 2).
__device__ __forceinline__ void pair_delta(const Rot rot[3], f2 d[18]) {
  c2 a0, B0, C0, d0, a1, B1, C1, d1, a2, B2, C2, d2;
  rot_small(rot[0], a0, B0, C0, d0);
  rot_small(rot[1], a1, B1, C1, d1);
  rot_small(rot[2], a2, B2, C2, d2);
  const c2 C1A0 = cadd2(C1, cmul2(C1, a0));  // C1 A0
  const c2 C1B0 = cmul2(C1, B0);
  c2 g[3][3];
  g[0][0] = cadd2(cadd2(a1, a0), cmul2(a1, a0));                      // A1 A0 - 1
  g[0][1] = cadd2(B0, cmul2(a1, B0));                                  // A1 B0
  g[0][2] = B1;
  g[1][0] = cadd2(cadd2(C0, cmul2(a2, C0)), cmul2(B2, C1A0));          // A2 C0 + B2 C1 A0
  g[1][1] = cadd2(cadd2(cadd2(a2, d0), cmul2(a2, d0)), cmul2(B2, C1B0));  // A2 D0 + B2 C1 B0 - 1
  g[1][2] = cadd2(B2, cmul2(B2, d1));                                  // B2 D1
  g[2][0] = cadd2(cadd2(cmul2(C2, C0), C1A0), cmul2(d2, C1A0));        // C2 C0 + D2 C1 A0
  g[2][1] = cadd2(cadd2(C2, cmul2(C2, d0)), cadd2(C1B0, cmul2(d2, C1B0)));  // C2 D0 + D2 C1 B0
  g[2][2] = cadd2(cadd2(d2, d1), cmul2(d2, d1));                      // D2 D1 - 1
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      d[LGT_RE(i, j)] = g[i][j].re;
      d[LGT_IM(i, j)] = g[i][j].im;
    }
}

// U <- g U = U + delta U  (pair arithmetic)
__device__ __forceinline__ void pair_apply_left(f2 u[18], const f2 d[18]) {
  f2 r[18];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      f2 c[6], x[6];
#pragma unroll
      for (int k = 0; k < 3; k++) {  // re: d_re u_re - d_im u_im
        c[2 * k] = d[LGT_RE(i, k)];
        x[2 * k] = u[LGT_RE(k, j)];
        c[2 * k + 1] = pair_neg(d[LGT_IM(i, k)]);
        x[2 * k + 1] = u[LGT_IM(k, j)];
      }
      r[LGT_RE(i, j)] = pair_axpy6(u[LGT_RE(i, j)], c, x);
#pragma unroll
      for (int k = 0; k < 3; k++) {  // im: d_re u_im + d_im u_re
        c[2 * k] = d[LGT_RE(i, k)];
        x[2 * k] = u[LGT_IM(k, j)];
        c[2 * k + 1] = d[LGT_IM(i, k)];
        x[2 * k + 1] = u[LGT_RE(k, j)];
      }
      r[LGT_IM(i, j)] = pair_axpy6(u[LGT_IM(i, j)], c, x);
    }
#pragma unroll
  for (int e = 0; e < 18; e++) u[e] = r[e];
}

// U <- U g^dagger = U + U delta^dagger  (pair arithmetic)
__device__ __forceinline__ void pair_apply_right_dag(f2 u[18], const f2 d[18]) {
  f2 r[18];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      f2 c[6], x[6];
#pragma unroll
      for (int k = 0; k < 3; k++) {  // re: u_re d_re + u_im d_im  (d_jk conjugated)
        c[2 * k] = d[LGT_RE(j, k)];
        x[2 * k] = u[LGT_RE(i, k)];
        c[2 * k + 1] = d[LGT_IM(j, k)];
        x[2 * k + 1] = u[LGT_IM(i, k)];
      }
      r[LGT_RE(i, j)] = pair_axpy6(u[LGT_RE(i, j)], c, x);
#pragma unroll
      for (int k = 0; k < 3; k++) {  // im: u_im d_re - u_re d_im
        c[2 * k] = d[LGT_RE(j, k)];
        x[2 * k] = u[LGT_IM(i, k)];
        c[2 * k + 1] = pair_neg(d[LGT_IM(j, k)]);
        x[2 * k + 1] = u[LGT_RE(i, k)];
      }
      r[LGT_IM(i, j)] = pair_axpy6(u[LGT_IM(i, j)], c, x);
    }
#pragma unroll
  for (int e = 0; e < 18; e++) u[e] = r[e];
}

// Fused estimate from the pair K: Re tr K and tr[Delta Delta^dagger],
// Delta = traceless part of (K - K^dagger)/(2i) (differences taken in pairs).
__device__ __forceinline__ void pair_violation(const f2 K[18], float &retr, float &delta2) {
  retr = pair_to_float(pair_add(pair_add(K[LGT_RE(0, 0)], K[LGT_RE(1, 1)]), K[LGT_RE(2, 2)]));
  const float d0 = pair_to_float(K[LGT_IM(0, 0)]), d1 = pair_to_float(K[LGT_IM(1, 1)]);
  const float d2 = pair_to_float(K[LGT_IM(2, 2)]);
  const float tr3 = pair_to_float(pair_add(pair_add(K[LGT_IM(0, 0)], K[LGT_IM(1, 1)]), K[LGT_IM(2, 2)])) *
                    (1.0f / 3.0f);
  float s = (d0 - tr3) * (d0 - tr3) + (d1 - tr3) * (d1 - tr3) + (d2 - tr3) * (d2 - tr3);
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = a + 1; b < 3; b++) {
      const float zre = pair_to_float(pair_add(K[LGT_RE(a, b)], pair_neg(K[LGT_RE(b, a)])));
      const float zim = pair_to_float(pair_add(K[LGT_IM(a, b)], K[LGT_IM(b, a)]));
      s += 0.5f * (zre * zre + zim * zim);
    }
  delta2 = s;
}

}  // namespace lgt
