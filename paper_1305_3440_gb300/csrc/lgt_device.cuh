// lgt_device.cuh -- device building blocks of the relaxation sweep on sm_103a.
//
// Matrices live in registers as R m[18]: element (a,b) of a 3x3 complex matrix
// is (m[2*(3a+b)], m[2*(3a+b)+1]) = (re, im).  All indices are compile-time
// constants after unrolling, so the arrays stay in registers.
//
// Link storage on the device is structure-of-arrays split by parity: every
// (parity, direction, 16-byte chunk) is a contiguous stream over the V/2 sites
// of that parity, so thread i of a warp loads chunk k of site i with one
// coalesced 128-bit access.  Formats:
//   FMT_F64   : 9 chunks of double2 (element c in chunk c)            1152 B / 8 links
//   FMT_F32_18: 4 chunks of float4 (elements 2k, 2k+1) + 1 float2 (element 8)
//   FMT_F32_12: 3 chunks of float4 = rows 0 and 1; row 2 = conj(row0 x row1)
// Within one parity a site's index is its lexicographic index / 2 (N1 even).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lgt {

enum { FMT_F64 = 0, FMT_F32_18 = 1, FMT_F32_12 = 2 };
// FP32-pair storage (each real an unevaluated sum hi + lo of two floats,
// ~48-bit significand): 9 float4 chunks per link, (hi_re, lo_re, hi_im, lo_im)
// of element c in chunk c -- the same 16 B per element as FMT_F64, so a field
// converts in place.
enum { FMT_PAIR = 3 };
// Anchored polish (lgt_anchor.cuh): not a link format but the sweep over a
// fixed anchor field (FP32-12 copy + K0 pairs) with D = G - 1 as pairs.
enum { FMT_ANCHOR = 4 };
enum { GAUGE_LANDAU = 0, GAUGE_COULOMB = 1, GAUGE_MAG = 2 };  // MAG: maximally Abelian gauge
enum { ALGO_OR = 0, ALGO_SR = 1, ALGO_SA = 2 };  // SA: simulated-annealing heat bath

#define LGT_RE(a, b) (2 * (3 * (a) + (b)))
#define LGT_IM(a, b) (2 * (3 * (a) + (b)) + 1)

// ------------------------------------------------------------------ geometry
struct Geom {
  int n1, n2, n3, nt;  // extents along x1, x2, x3, t
  int half1;           // n1 / 2
  int vs_half;         // sites of one parity in one timeslice
  int vh;              // sites of one parity
};

struct Coords {
  int x1, x2, x3, t;
};

// site j (0 <= j < vs_half) of parity p in timeslice t
__host__ __device__ __forceinline__ Coords coords_in_slice(const Geom &g, int p, int t, int j) {
  Coords c;
  const int row = j / g.half1;
  c.x2 = row % g.n2;
  c.x3 = row / g.n2;
  c.t = t;
  c.x1 = 2 * (j - row * g.half1) + ((p + t + c.x2 + c.x3) & 1);
  return c;
}

// within-parity index of a site
__host__ __device__ __forceinline__ int cb_index(const Geom &g, int x1, int x2, int x3, int t) {
  return ((t * g.n3 + x3) * g.n2 + x2) * g.half1 + (x1 >> 1);
}

// within-parity index of x + dir * mu-hat (dir = +-1)
__host__ __device__ __forceinline__ int cb_shift(const Geom &g, const Coords &c, int mu, int dir) {
  int x1 = c.x1, x2 = c.x2, x3 = c.x3, t = c.t;
  if (mu == 0) {
    t += dir;
    t = t < 0 ? t + g.nt : (t >= g.nt ? t - g.nt : t);
  } else if (mu == 1) {
    x1 += dir;
    x1 = x1 < 0 ? x1 + g.n1 : (x1 >= g.n1 ? x1 - g.n1 : x1);
  } else if (mu == 2) {
    x2 += dir;
    x2 = x2 < 0 ? x2 + g.n2 : (x2 >= g.n2 ? x2 - g.n2 : x2);
  } else {
    x3 += dir;
    x3 = x3 < 0 ? x3 + g.n3 : (x3 >= g.n3 ? x3 - g.n3 : x3);
  }
  return cb_index(g, x1, x2, x3, t);
}

// ------------------------------------------------------------- link formats
__host__ __device__ __forceinline__ size_t link_bytes_per_half_site(int fmt) {
  // bytes of 4 links of one site (one parity's share of one site)
  return (fmt == FMT_F64 || fmt == FMT_PAIR) ? 4 * 144 : (fmt == FMT_F32_18 ? 4 * 72 : 4 * 48);
}

template <int FMT>
struct LinkIO;

template <>
struct LinkIO<FMT_F64> {
  typedef double real;
  static constexpr bool kCompressed = false;
  static __device__ __forceinline__ void load(const void *base, int vh, int p, int mu, int i, double m[18]) {
    const double2 *b = reinterpret_cast<const double2 *>(base) + (size_t)((p * 4 + mu) * 9) * vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      double2 v = __ldg(b + (size_t)c * vh);
      m[2 * c] = v.x;
      m[2 * c + 1] = v.y;
    }
  }
  static __device__ __forceinline__ void load_raw(const void *base, int vh, int p, int mu, int i, double m[18]) {
    load(base, vh, p, mu, i, m);
  }
  static __device__ __forceinline__ void store(void *base, int vh, int p, int mu, int i, const double m[18]) {
    double2 *b = reinterpret_cast<double2 *>(base) + (size_t)((p * 4 + mu) * 9) * vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) b[(size_t)c * vh] = make_double2(m[2 * c], m[2 * c + 1]);
  }
};

template <>
struct LinkIO<FMT_F32_18> {
  typedef float real;
  static constexpr bool kCompressed = false;
  static __device__ __forceinline__ void load(const void *base, int vh, int p, int mu, int i, float m[18]) {
    const float4 *b4 = reinterpret_cast<const float4 *>(base) + (size_t)((p * 4 + mu) * 4) * vh + i;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      float4 v = __ldg(b4 + (size_t)k * vh);
      m[4 * k] = v.x;
      m[4 * k + 1] = v.y;
      m[4 * k + 2] = v.z;
      m[4 * k + 3] = v.w;
    }
    const float2 *b2 = reinterpret_cast<const float2 *>(reinterpret_cast<const float4 *>(base) + (size_t)32 * vh) +
                       (size_t)(p * 4 + mu) * vh + i;
    float2 w = __ldg(b2);
    m[16] = w.x;
    m[17] = w.y;
  }
  static __device__ __forceinline__ void load_raw(const void *base, int vh, int p, int mu, int i, float m[18]) {
    load(base, vh, p, mu, i, m);
  }
  static __device__ __forceinline__ void store(void *base, int vh, int p, int mu, int i, const float m[18]) {
    float4 *b4 = reinterpret_cast<float4 *>(base) + (size_t)((p * 4 + mu) * 4) * vh + i;
#pragma unroll
    for (int k = 0; k < 4; k++) b4[(size_t)k * vh] = make_float4(m[4 * k], m[4 * k + 1], m[4 * k + 2], m[4 * k + 3]);
    float2 *b2 = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(base) + (size_t)32 * vh) +
                 (size_t)(p * 4 + mu) * vh + i;
    *b2 = make_float2(m[16], m[17]);
  }
};

// row 2 of an SU(3) matrix from rows 0 and 1: row2 = conj(row0 x row1)
template <typename R>
__device__ __forceinline__ void rebuild_row2(R m[18]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    // (r0[a] r1[b] - r0[b] r1[a])^*
    const R re = m[LGT_RE(0, a)] * m[LGT_RE(1, b)] - m[LGT_IM(0, a)] * m[LGT_IM(1, b)] -
                 (m[LGT_RE(0, b)] * m[LGT_RE(1, a)] - m[LGT_IM(0, b)] * m[LGT_IM(1, a)]);
    const R im = m[LGT_RE(0, a)] * m[LGT_IM(1, b)] + m[LGT_IM(0, a)] * m[LGT_RE(1, b)] -
                 (m[LGT_RE(0, b)] * m[LGT_IM(1, a)] + m[LGT_IM(0, b)] * m[LGT_RE(1, a)]);
    m[LGT_RE(2, c)] = re;
    m[LGT_IM(2, c)] = -im;
  }
}

template <>
struct LinkIO<FMT_F32_12> {
  typedef float real;
  static constexpr bool kCompressed = true;
  // rows 0 and 1 only (row 2 left zero; rebuild_row2 restores it)
  static __device__ __forceinline__ void load_raw(const void *base, int vh, int p, int mu, int i, float m[18]) {
    const float4 *b4 = reinterpret_cast<const float4 *>(base) + (size_t)((p * 4 + mu) * 3) * vh + i;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float4 v = __ldg(b4 + (size_t)k * vh);
      m[4 * k] = v.x;
      m[4 * k + 1] = v.y;
      m[4 * k + 2] = v.z;
      m[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int k = 12; k < 18; k++) m[k] = 0.0f;
  }
  static __device__ __forceinline__ void load(const void *base, int vh, int p, int mu, int i, float m[18]) {
    load_raw(base, vh, p, mu, i, m);
    rebuild_row2(m);
  }
  // rows 0 and 1 only; row 2 is never stored
  static __device__ __forceinline__ void store(void *base, int vh, int p, int mu, int i, const float m[18]) {
    float4 *b4 = reinterpret_cast<float4 *>(base) + (size_t)((p * 4 + mu) * 3) * vh + i;
#pragma unroll
    for (int k = 0; k < 3; k++) b4[(size_t)k * vh] = make_float4(m[4 * k], m[4 * k + 1], m[4 * k + 2], m[4 * k + 3]);
  }
};

// The accumulated gauge transformation G(x) of the FP32 phase: one SU(3) per
// site in FP32, stored as rows 0 and 1 (3 float4 chunks per parity stream);
// row 2 = conj(row0 x row1) is rebuilt on load.
struct GIO {
  static __device__ __forceinline__ void load(const void *base, int vh, int p, int i, float m[18]) {
    const float4 *b4 = reinterpret_cast<const float4 *>(base) + (size_t)(p * 3) * vh + i;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float4 v = __ldg(b4 + (size_t)k * vh);
      m[4 * k] = v.x;
      m[4 * k + 1] = v.y;
      m[4 * k + 2] = v.z;
      m[4 * k + 3] = v.w;
    }
    rebuild_row2(m);
  }
  static __device__ __forceinline__ void store(void *base, int vh, int p, int i, const float m[18]) {
    float4 *b4 = reinterpret_cast<float4 *>(base) + (size_t)(p * 3) * vh + i;
#pragma unroll
    for (int k = 0; k < 3; k++) b4[(size_t)k * vh] = make_float4(m[4 * k], m[4 * k + 1], m[4 * k + 2], m[4 * k + 3]);
  }
};

__host__ __device__ __forceinline__ size_t g_bytes(int vh) { return (size_t)vh * 2 * 3 * 16; }

__host__ __device__ __forceinline__ size_t field_bytes(int fmt, int vh) {
  return (size_t)vh * 2 * link_bytes_per_half_site(fmt);
}

// ------------------------------------------------------------ 3x3 algebra
template <typename R>
__device__ __forceinline__ void mat_zero(R m[18]) {
#pragma unroll
  for (int k = 0; k < 18; k++) m[k] = R(0);
}

// c = a * b
template <typename R>
__device__ __forceinline__ void mat_mul(const R a[18], const R b[18], R c[18]) {
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int s = 0; s < 3; s++) {
      R re = R(0), im = R(0);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        re = fma(a[LGT_RE(r, k)], b[LGT_RE(k, s)], re);
        re = fma(-a[LGT_IM(r, k)], b[LGT_IM(k, s)], re);
        im = fma(a[LGT_RE(r, k)], b[LGT_IM(k, s)], im);
        im = fma(a[LGT_IM(r, k)], b[LGT_RE(k, s)], im);
      }
      c[LGT_RE(r, s)] = re;
      c[LGT_IM(r, s)] = im;
    }
}

// c = a * b^dagger
template <typename R>
__device__ __forceinline__ void mat_mul_dag(const R a[18], const R b[18], R c[18]) {
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int s = 0; s < 3; s++) {
      R re = R(0), im = R(0);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        // a[r][k] * conj(b[s][k])
        re = fma(a[LGT_RE(r, k)], b[LGT_RE(s, k)], re);
        re = fma(a[LGT_IM(r, k)], b[LGT_IM(s, k)], re);
        im = fma(a[LGT_IM(r, k)], b[LGT_RE(s, k)], im);
        im = fma(-a[LGT_RE(r, k)], b[LGT_IM(s, k)], im);
      }
      c[LGT_RE(r, s)] = re;
      c[LGT_IM(r, s)] = im;
    }
}

// K += U
template <typename R>
__device__ __forceinline__ void acc_add(R k[18], const R u[18]) {
#pragma unroll
  for (int e = 0; e < 18; e++) k[e] += u[e];
}

// K += U^dagger
template <typename R>
__device__ __forceinline__ void acc_add_dag(R k[18], const R u[18]) {
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      k[LGT_RE(a, b)] += u[LGT_RE(b, a)];
      k[LGT_IM(a, b)] -= u[LGT_IM(b, a)];
    }
}

template <typename R>
__device__ __forceinline__ R rsqrt_t(R x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// Reunitarise: Gram-Schmidt on rows 0 and 1, then row 2 = conj(row0 x row1).
template <typename R>
__device__ __forceinline__ void reunitarise(R m[18]) {
  R n0 = R(0);
#pragma unroll
  for (int c = 0; c < 3; c++) n0 += m[LGT_RE(0, c)] * m[LGT_RE(0, c)] + m[LGT_IM(0, c)] * m[LGT_IM(0, c)];
  n0 = rsqrt_t(n0);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    m[LGT_RE(0, c)] *= n0;
    m[LGT_IM(0, c)] *= n0;
  }
  R pre = R(0), pim = R(0);  // <row0, row1> = sum conj(r0) r1
#pragma unroll
  for (int c = 0; c < 3; c++) {
    pre += m[LGT_RE(0, c)] * m[LGT_RE(1, c)] + m[LGT_IM(0, c)] * m[LGT_IM(1, c)];
    pim += m[LGT_RE(0, c)] * m[LGT_IM(1, c)] - m[LGT_IM(0, c)] * m[LGT_RE(1, c)];
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    m[LGT_RE(1, c)] -= pre * m[LGT_RE(0, c)] - pim * m[LGT_IM(0, c)];
    m[LGT_IM(1, c)] -= pre * m[LGT_IM(0, c)] + pim * m[LGT_RE(0, c)];
  }
  R n1 = R(0);
#pragma unroll
  for (int c = 0; c < 3; c++) n1 += m[LGT_RE(1, c)] * m[LGT_RE(1, c)] + m[LGT_IM(1, c)] * m[LGT_IM(1, c)];
  n1 = rsqrt_t(n1);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    m[LGT_RE(1, c)] *= n1;
    m[LGT_IM(1, c)] *= n1;
  }
  rebuild_row2(m);
}

// ------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds of two
// 32x32->64-bit multiplies with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
  for (int round = 0; round < 10; round++) {
    const uint32_t lo_a = 0xD2511F53u * ctr.x, hi_a = __umulhi(0xD2511F53u, ctr.x);
    const uint32_t lo_b = 0xCD9E8D57u * ctr.z, hi_b = __umulhi(0xCD9E8D57u, ctr.z);
    ctr = make_uint4(hi_b ^ ctr.y ^ key.x, lo_b, hi_a ^ ctr.w ^ key.y, lo_a);
    key.x += 0x9E3779B9u;
    key.y += 0xBB67AE85u;
  }
  return ctr;
}

#define LGT_SR_TAG 0x53524C58u  // stream tag of the stochastic-relaxation draws

// ------------------------------------------- simulated annealing (heat bath)
// Simulated annealing (named by the paper as a preconditioner, Sec. 1) is
// read as sweeps whose subgroup elements r are drawn from exp(beta Re tr[r M])
// times Haar measure, beta rising over the sweeps.  With p the maximum
// (closed form above) and q the block projection, Re tr[r M] = 2 |q| (r . p),
// so r = a p (matrix product), a0 = x drawn from sqrt(1 - x^2) exp(alpha x)
// on [-1, 1] with alpha = 2 beta |q| (Kennedy and Pendleton 1985: at most
// LGT_SA_ATTEMPTS tries, else the subgroup is left unchanged), the vector
// part of a uniform on the sphere of radius sqrt(1 - x^2).  Draws: Philox,
// key = seed, counter = (site, subgroup << 24 | attempt, sweep, tag).
#define LGT_SA_TAG 0x53414842u  // stream tag of the heat-bath draws
#define LGT_SA_ATTEMPTS 64u
#define LGT_SA_DIRECTION 0xFFFFFFu

struct SaDraw {
  double beta;
  uint2 key;
  uint32_t site, sweep;
};

template <typename R>
__device__ __forceinline__ R unit_open(uint32_t w) {
  return (R(w) + R(0.5)) * R(1.0 / 4294967296.0);
}
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }
__device__ __forceinline__ float cos_t(float x) { return cosf(x); }
__device__ __forceinline__ double cos_t(double x) { return cos(x); }
__device__ __forceinline__ float sin_t(float x) { return sinf(x); }
__device__ __forceinline__ double sin_t(double x) { return sin(x); }

// Heat-bath element for a block projection given at twice the unit scale
// (qq = 2 q, as local_update forms it): alpha = 2 beta |q| = beta |qq|.
// r stays the identity on a degenerate block or when every attempt fails.
template <typename R>
__device__ __forceinline__ void su2_heatbath(R qq0, R qq1, R qq2, R qq3, const SaDraw &sd, int s, R &r0, R &r1,
                                             R &r2, R &r3) {
  r0 = R(1), r1 = R(0), r2 = R(0), r3 = R(0);
  const R n2 = qq0 * qq0 + qq1 * qq1 + qq2 * qq2 + qq3 * qq3;
  if (!(n2 > R(0)) || !(sd.beta > 0.0)) return;
  const R norm = sqrt(n2);
  const R alpha = R(sd.beta) * norm;
  const R two_pi = R(6.283185307179586476925286766559);
  R x = R(1);
  bool ok = false;
  for (uint32_t k = 0; k < LGT_SA_ATTEMPTS && !ok; k++) {
    const uint4 w = philox4x32_10(make_uint4(sd.site, ((uint32_t)s << 24) | k, sd.sweep, LGT_SA_TAG), sd.key);
    const R c = cos_t(two_pi * unit_open<R>(w.y));
    const R delta = -(log_t(unit_open<R>(w.x)) + c * c * log_t(unit_open<R>(w.z))) / alpha;
    const R u3 = unit_open<R>(w.w);
    if (u3 * u3 <= R(1) - R(0.5) * delta) {
      x = R(1) - delta;
      ok = true;
    }
  }
  if (!ok) return;
  const R inv = R(1) / norm;
  const R p0 = qq0 * inv, p1 = -qq1 * inv, p2 = -qq2 * inv, p3 = -qq3 * inv;
  const uint4 w = philox4x32_10(make_uint4(sd.site, ((uint32_t)s << 24) | LGT_SA_DIRECTION, sd.sweep, LGT_SA_TAG), sd.key);
  const R cth = R(2) * unit_open<R>(w.x) - R(1);
  const R sth = sqrt(R(1) - cth * cth), phi = two_pi * unit_open<R>(w.y);
  const R rad = x * x < R(1) ? sqrt(R(1) - x * x) : R(0);
  const R a0 = x, a1 = rad * sth * cos_t(phi), a2 = rad * sth * sin_t(phi), a3 = rad * cth;
  // r = a p for the matrices [[r0 + i r3, r2 + i r1], [-r2 + i r1, r0 - i r3]]
  r0 = a0 * p0 - a1 * p1 - a2 * p2 - a3 * p3;
  r1 = a0 * p1 + a1 * p0 + a3 * p2 - a2 * p3;
  r2 = a0 * p2 + a2 * p0 + a1 * p3 - a3 * p1;
  r3 = a0 * p3 + a3 * p0 + a2 * p1 - a1 * p2;
}

// --------------------------------------------------- Sec. 3: local update
// Maximise Re tr[g K] over SU(3) by one pass over the SU(2) subgroups
// (0,1), (0,2), (1,2) (Cabibbo-Marinari).  W starts as K; for each subgroup
// the 2x2 block of W is projected on SU(2) (q0 + i q.sigma), the closed-form
// maximum r = (q0, -q)/|q| (g = K^dagger/sqrt(det K^dagger) of Sec. 3) is
// overrelaxed to first order (Sec. 3.1) or squared with probability p
// (Sec. 3.2), and W <- R W, g <- R g.  On return g holds the update.
template <typename R, int ALGO>
__device__ __forceinline__ void local_update(R W[18], R g[18], R omega, uint64_t sr_thr, uint4 draws,
                                             const SaDraw *sa = nullptr) {
#pragma unroll
  for (int s = 0; s < 3; s++) {
    const int i = (s == 2) ? 1 : 0;
    const int j = (s == 0) ? 1 : 2;
    // projection of the (i,j) block (scaled by 2; only its direction matters)
    const R q0 = W[LGT_RE(i, i)] + W[LGT_RE(j, j)];
    const R q1 = W[LGT_IM(i, j)] + W[LGT_IM(j, i)];
    const R q2 = W[LGT_RE(i, j)] - W[LGT_RE(j, i)];
    const R q3 = W[LGT_IM(i, i)] - W[LGT_IM(j, j)];
    const R n2 = q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3;
    R r0 = R(1), r1 = R(0), r2 = R(0), r3 = R(0);
    if (ALGO == ALGO_SA) {
      su2_heatbath<R>(q0, q1, q2, q3, *sa, s, r0, r1, r2, r3);
    } else if (n2 > R(0)) {
      const R inv = rsqrt_t(n2);
      r0 = q0 * inv;
      r1 = -q1 * inv;
      r2 = -q2 * inv;
      r3 = -q3 * inv;
    }
    if (ALGO == ALGO_SA) {
      // drawn above
    } else if (ALGO == ALGO_OR) {
      r0 = (R(1) - omega) + omega * r0;
      r1 *= omega;
      r2 *= omega;
      r3 *= omega;
      const R inv = rsqrt_t(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
      r0 *= inv;
      r1 *= inv;
      r2 *= inv;
      r3 *= inv;
    } else {
      const uint32_t d = s == 0 ? draws.x : (s == 1 ? draws.y : draws.z);
      if ((uint64_t)d < sr_thr) {
        const R a0 = r0 * r0 - (r1 * r1 + r2 * r2 + r3 * r3);
        const R two_r0 = R(2) * r0;
        r1 *= two_r0;
        r2 *= two_r0;
        r3 *= two_r0;
        r0 = a0;
      }
    }
    // R_s = [[r0 + i r3, r2 + i r1], [-r2 + i r1, r0 - i r3]] on rows (i, j)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const R wire = W[LGT_RE(i, c)], wiim = W[LGT_IM(i, c)];
      const R wjre = W[LGT_RE(j, c)], wjim = W[LGT_IM(j, c)];
      W[LGT_RE(i, c)] = r0 * wire - r3 * wiim + r2 * wjre - r1 * wjim;
      W[LGT_IM(i, c)] = r0 * wiim + r3 * wire + r2 * wjim + r1 * wjre;
      W[LGT_RE(j, c)] = -r2 * wire - r1 * wiim + r0 * wjre + r3 * wjim;
      W[LGT_IM(j, c)] = -r2 * wiim + r1 * wire + r0 * wjim - r3 * wjre;
    }
    if (s == 0) {
      mat_zero(g);
      g[LGT_RE(0, 0)] = r0;
      g[LGT_IM(0, 0)] = r3;
      g[LGT_RE(0, 1)] = r2;
      g[LGT_IM(0, 1)] = r1;
      g[LGT_RE(1, 0)] = -r2;
      g[LGT_IM(1, 0)] = r1;
      g[LGT_RE(1, 1)] = r0;
      g[LGT_IM(1, 1)] = -r3;
      g[LGT_RE(2, 2)] = R(1);
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const R gire = g[LGT_RE(i, c)], giim = g[LGT_IM(i, c)];
        const R gjre = g[LGT_RE(j, c)], gjim = g[LGT_IM(j, c)];
        g[LGT_RE(i, c)] = r0 * gire - r3 * giim + r2 * gjre - r1 * gjim;
        g[LGT_IM(i, c)] = r0 * giim + r3 * gire + r2 * gjim + r1 * gjre;
        g[LGT_RE(j, c)] = -r2 * gire - r1 * giim + r0 * gjre + r3 * gjim;
        g[LGT_IM(j, c)] = -r2 * giim + r1 * gire + r0 * gjim - r3 * gjre;
      }
    }
  }
}

// Re tr K and tr[Delta Delta^dagger] with Delta = traceless part of
// (K - K^dagger)/(2i): the violation at a site whose neighbours carry g = 1
// (sum_mu A_mu(x) - A_mu(x-mu) expands to exactly this), Sec. 2.
// Computed in the precision R of the sweep.
template <typename R>
__device__ __forceinline__ void violation_of_K(const R K[18], R &retr, R &delta2) {
  retr = K[LGT_RE(0, 0)] + K[LGT_RE(1, 1)] + K[LGT_RE(2, 2)];
  // D = (K - K^dagger)/(2i): D_aa = Im K_aa; D_ab = (z.im/2, -z.re/2), z = K_ab - conj(K_ba)
  const R d0 = K[LGT_IM(0, 0)], d1 = K[LGT_IM(1, 1)], d2 = K[LGT_IM(2, 2)];
  const R tr3 = (d0 + d1 + d2) * (R(1) / R(3));
  R s = (d0 - tr3) * (d0 - tr3) + (d1 - tr3) * (d1 - tr3) + (d2 - tr3) * (d2 - tr3);
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = a + 1; b < 3; b++) {
      const R zre = K[LGT_RE(a, b)] - K[LGT_RE(b, a)];
      const R zim = K[LGT_IM(a, b)] + K[LGT_IM(b, a)];
      s += R(0.5) * (zre * zre + zim * zim);  // 2 |z/2|^2
    }
  delta2 = s;
}

// --------------------------------------------------- deterministic reductions
// Sum NV doubles over the block in a fixed order (xor butterfly within each
// warp, then warps in index order); the block total lands in out[] of thread 0.
// T is the per-thread value type (the warp stage runs in T); warp partials
// and the block total are FP64.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T v[NV], double *out) {
  __shared__ double warp_part[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; k++) warp_part[k][warp] = (double)v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double s = 0.0;
      for (int w = 0; w < nw; w++) s += warp_part[k][w];
      out[k] = s;
    }
  }
  __syncthreads();
}

// --------------------------------------------- maximally Abelian gauge
// The abstract names the maximally Abelian gauge; the text gives neither its
// functional nor its update.  Reading: F_MAG = 1/(N_c N_d V) sum_{x,mu} sum_a
// |U_mu(x)_aa|^2, maximised.  Its gauge gradient at x is carried by
//   X(x) = sum_mu ( U_mu(x) D_mu(x)^dagger - D_mu(x-mu)^dagger U_mu(x-mu) )
// (D the diagonal part), theta_MAG = 1/(N_c V) sum_x tr[Delta Delta^dagger]
// with Delta the traceless part of (X - X^dagger)/(2i).  For an SU(2)
// subgroup element R on rows/columns (i, j), the site's functional is
// const + n.v/2 with n.sigma = R^dagger sigma_3 R and v summed over the 8
// links from s(a, b) = (2 Re(a* b), 2 Im(a* b), |a|^2 - |b|^2): forward links
// give s((gU)_ii, (gU)_ji) - s((gU)_ij, (gU)_jj), backward links
// s(conj (Ug+)_ii, conj (Ug+)_ij) - s(conj (Ug+)_ji, conj (Ug+)_jj).  The
// maximum is n = v/|v|; of its circle of elements (left factors
// exp(i phi sigma_3) keep every |diagonal entry|) the one nearest the identity
// is r = (|v| + v_3, -v_2, v_1, 0)/norm, or (0, 1, 0, 0) when v = -|v| e_3.

// v += sign * s(a, b), a = (are, aim), b = (bre, bim)
template <typename R>
__device__ __forceinline__ void mag_s(R are, R aim, R bre, R bim, R sign, R v[3]) {
  const R zre = are * bre + aim * bim, zim = are * bim - aim * bre;  // conj(a) b
  v[0] += sign * (R(2) * zre);
  v[1] += sign * (R(2) * zim);
  v[2] += sign * ((are * are + aim * aim) - (bre * bre + bim * bim));
}

template <typename R>
__device__ __forceinline__ void mag_maximum(const R v[3], R &r0, R &r1, R &r2, R &r3) {
  r0 = R(1), r1 = R(0), r2 = R(0), r3 = R(0);
  const R n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  if (!(n2 > R(0))) return;
  const R a = sqrt(n2) + v[2];
  const R m2 = a * a + v[0] * v[0] + v[1] * v[1];
  if (!(m2 > R(0))) {
    r0 = R(0), r1 = R(1);
    return;
  }
  const R inv = rsqrt_t(m2);
  r0 = a * inv;
  r1 = -v[1] * inv;
  r2 = v[0] * inv;
}

}  // namespace lgt
