/*
 * lgt_oracle.c -- plain FP64 CPU oracle for relaxation gauge fixing of SU(3)
 * lattice gauge fields (Schroeck & Vogt, "Gauge fixing in lattice QCD with
 * multi-GPUs", Excited QCD 2013).
 *
 * TEST INFRASTRUCTURE.  This file exists to check the CUDA library.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it; the library never calls it and shares no code with it (not even the
 * random-number generator: the stochastic-relaxation draws below come from an
 * own implementation of Philox4x32-10).
 *
 * What it computes, in the paper's notation (Sections 2 and 3):
 *   F^g[U]   = 1/(N_c N_d V) Re sum_{mu,x} tr U^g_mu(x)            (Sec. 2, functional)
 *   U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dagger                         (Sec. 2, transformation)
 *   Delta(x) = sum_mu (A_mu(x) - A_mu(x-mu))                         (Sec. 2, violation)
 *   theta    = 1/(N_c V) sum_x tr[Delta(x) Delta(x)^dagger]          (Sec. 2, precision)
 *   f^g(x)   = Re tr[g(x) K(x)]                                       (Sec. 3, local functional)
 *   K(x)     = sum_mu (U_mu(x) g(x+mu)^dagger + U_mu(x-mu)^dagger g(x-mu)^dagger)  (Sec. 3)
 *   SU(2) maximum g = K^dagger / sqrt(det K^dagger)                   (Sec. 3)
 *   SU(3): iterate over the three SU(2) subgroups (Cabibbo-Marinari)  (Sec. 3)
 *   overrelaxation g -> g^omega to first order, omega in [1,2)        (Sec. 3.1)
 *   stochastic relaxation g -> g^2 with probability p                 (Sec. 3.2)
 *   the two parity subsets are updated one after the other           (Sec. 3, Sec. 4)
 *
 * Readings where the paper is silent (each stated again where it is used):
 *   - A_mu(x) is the traceless part of (U_mu(x) - U_mu(x)^dagger)/(2i).
 *   - Links are transformed in place after every local update, so K(x) is
 *     evaluated with g(x +- mu) = 1 on the current links.
 *   - For an SU(3) 2x2 block that is not itself proportional to SU(2), the
 *     closed form is applied to its projection q0 + i q.sigma onto the span
 *     of SU(2): Re tr(r M) depends on M only through that projection.
 *   - Subgroups in the order (0,1), (0,2), (1,2), one pass per site update.
 *   - First-order overrelaxation acts on each subgroup element r:
 *     r -> normalise((1-omega) 1 + omega r).
 *   - Stochastic relaxation: one Philox4x32-10 block per (seed, sweep, site),
 *     word s decides subgroup s; take r^2 iff word < floor(p * 2^32).
 *   - Even parity (x1+x2+x3+t even) first in every sweep.
 *   - Coulomb gauge: per timeslice, spatial directions only (N_d = 3,
 *     V -> V_s); parity is the 4-D parity, and by default g(x) also acts on
 *     the temporal links U_0(x) and U_0(x-0) so the result stays a gauge
 *     transform of the input.
 *   - Maximally Abelian gauge (named in the abstract beside Landau and
 *     Coulomb gauge; the text gives neither its functional nor its update):
 *     see the section "maximally Abelian gauge" below.
 *
 * Precision: FP64 throughout, no fused multiply-add contraction
 * (-ffp-contract=off), sums in fixed order.  OpenMP runs the sites of one
 * parity concurrently; they touch disjoint links, so results are
 * bit-identical for every thread count and every site order.
 *
 * Link layout (complex128 AoS): links[((site*4 + mu)*9 + 3*row + col)*2 + {re,im}],
 * site = x1 + N1*(x2 + N2*(x3 + N3*t)), dims = {N_t, N_3, N_2, N_1},
 * mu = 0 is t, mu = 1, 2, 3 are x1, x2, x3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define NC 3

enum { ORC_LANDAU = 0, ORC_COULOMB = 1, ORC_MAG = 2 };
enum { ORC_OR = 0, ORC_SR = 1, ORC_SA = 2 };

/* ------------------------------------------------------------------ complex */
typedef struct { double re, im; } cplx;

static cplx c_make(double re, double im) { cplx z = {re, im}; return z; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_sub(cplx a, cplx b) { return c_make(a.re - b.re, a.im - b.im); }
static cplx c_mul(cplx a, cplx b) { return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cplx c_conj(cplx a) { return c_make(a.re, -a.im); }

/* --------------------------------------------------------------- 3x3 matrix */
typedef struct { cplx e[NC][NC]; } su3;

static su3 m_identity(void) {
  su3 r;
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) r.e[a][b] = c_make(a == b ? 1.0 : 0.0, 0.0);
  return r;
}

static su3 m_mul(const su3 *x, const su3 *y) {
  su3 r;
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) {
      cplx s = c_make(0.0, 0.0);
      for (int c = 0; c < NC; c++) s = c_add(s, c_mul(x->e[a][c], y->e[c][b]));
      r.e[a][b] = s;
    }
  return r;
}

static su3 m_dagger(const su3 *x) {
  su3 r;
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) r.e[a][b] = c_conj(x->e[b][a]);
  return r;
}

static su3 m_add(const su3 *x, const su3 *y) {
  su3 r;
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) r.e[a][b] = c_add(x->e[a][b], y->e[a][b]);
  return r;
}

static su3 m_sub(const su3 *x, const su3 *y) {
  su3 r;
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) r.e[a][b] = c_sub(x->e[a][b], y->e[a][b]);
  return r;
}

static double m_retrace(const su3 *x) { return x->e[0][0].re + x->e[1][1].re + x->e[2][2].re; }

/* ----------------------------------------------------------------- geometry */
typedef struct {
  int64_t n[4]; /* extent per direction mu: n[0] = N_t, n[1] = N1, n[2] = N2, n[3] = N3 */
  int64_t vol;
  int64_t vol_s; /* one timeslice */
} lattice;

static lattice make_lattice(const int32_t dims[4]) {
  lattice l;
  l.n[0] = dims[0];
  l.n[1] = dims[3];
  l.n[2] = dims[2];
  l.n[3] = dims[1];
  l.vol_s = l.n[1] * l.n[2] * l.n[3];
  l.vol = l.vol_s * l.n[0];
  return l;
}

/* coordinates x[mu] of a lexicographic site index */
static void site_coords(const lattice *l, int64_t site, int64_t x[4]) {
  x[1] = site % l->n[1];
  site /= l->n[1];
  x[2] = site % l->n[2];
  site /= l->n[2];
  x[3] = site % l->n[3];
  x[0] = site / l->n[3];
}

static int64_t site_index(const lattice *l, const int64_t x[4]) {
  return x[1] + l->n[1] * (x[2] + l->n[2] * (x[3] + l->n[3] * x[0]));
}

/* x + dir * mu-hat, periodic */
static int64_t site_shift(const lattice *l, int64_t site, int mu, int dir) {
  int64_t x[4];
  site_coords(l, site, x);
  x[mu] = (x[mu] + dir + l->n[mu]) % l->n[mu];
  return site_index(l, x);
}

static int site_parity(const lattice *l, int64_t site) {
  int64_t x[4];
  site_coords(l, site, x);
  return (int)((x[0] + x[1] + x[2] + x[3]) & 1);
}

static int64_t site_time(const lattice *l, int64_t site) { return site / l->vol_s; }

/* ------------------------------------------------------------- link access */
static su3 load_link(const double *links, int64_t site, int mu) {
  const double *p = links + ((size_t)site * 4 + (size_t)mu) * 18;
  su3 u;
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) u.e[a][b] = c_make(p[2 * (3 * a + b)], p[2 * (3 * a + b) + 1]);
  return u;
}

static void store_link(double *links, int64_t site, int mu, const su3 *u) {
  double *p = links + ((size_t)site * 4 + (size_t)mu) * 18;
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) {
      p[2 * (3 * a + b)] = u->e[a][b].re;
      p[2 * (3 * a + b) + 1] = u->e[a][b].im;
    }
}

/* The directions that enter the functional: all four for Landau gauge, the
 * three spatial ones for Coulomb gauge (one timeslice at a time). */
static int first_mu(int gauge) { return gauge == ORC_COULOMB ? 1 : 0; }

/* ------------------------------------------------------ Philox4x32-10 (RNG) */
/* Own implementation of the counter-based generator of Salmon et al. (SC'11):
 * ten rounds of two 32x32->64 multiplies with the Weyl-sequence key schedule. */
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  int round;
  for (round = 0; round < 10; round++) {
    const uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
    const uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    const uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
    const uint32_t y1 = (uint32_t)prod_b;
    const uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
    const uint32_t y3 = (uint32_t)prod_a;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
    k0 += 0x9E3779B9u; /* golden ratio */
    k1 += 0xBB67AE85u; /* sqrt(3) - 1 */
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

#define SR_TAG 0x53524C58u /* "SRLX": stochastic-relaxation stream */

/* The three draws (one per SU(2) subgroup) for one site update. */
static void sr_draws(uint64_t seed, uint64_t sweep, int64_t site, uint32_t u[3]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {(uint32_t)site, (uint32_t)((uint64_t)site >> 32), (uint32_t)sweep, SR_TAG};
  uint32_t w[4];
  philox4x32_10(ctr, key, w);
  u[0] = w[0];
  u[1] = w[1];
  u[2] = w[2];
}

/* integer acceptance threshold for probability p: accept iff draw < floor(p 2^32) */
static uint64_t sr_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return (uint64_t)1 << 32;
  return (uint64_t)floor(p * 4294967296.0);
}

/* ----------------------------------------------------- Section 3: K(x) */
/* K(x) = sum_mu ( U_mu(x) g(x+mu)^dagger + U_mu(x-mu)^dagger g(x-mu)^dagger ).
 * The links are transformed in place after each local update, so on the
 * current links the neighbours' g are the identity and
 *   K(x) = sum_mu ( U_mu(x) + U_mu(x-mu)^dagger ). */
static su3 gather_K(const lattice *l, const double *links, int64_t site, int gauge) {
  su3 k;
  memset(&k, 0, sizeof k);
  for (int mu = first_mu(gauge); mu < 4; mu++) {
    su3 fwd = load_link(links, site, mu);
    su3 bwd = load_link(links, site_shift(l, site, mu, -1), mu);
    su3 bwd_dag = m_dagger(&bwd);
    k = m_add(&k, &fwd);
    k = m_add(&k, &bwd_dag);
  }
  return k;
}

/* ------------------------------------- Section 3: SU(2) closed-form maximum */
/* An SU(2) element as a unit quaternion r = r0 1 + i (r1 s1 + r2 s2 + r3 s3)
 * (s_k the Pauli matrices):
 *      [  r0 + i r3    r2 + i r1 ]
 *      [ -r2 + i r1    r0 - i r3 ]
 * The 2x2 block M of W restricted to rows/cols (i,j) is projected onto
 * span{1, i s_k} (real inner product Re tr A^dagger B, basis norm^2 = 2):
 *   q0 = Re(M00 + M11)/2, q1 = Im(M01 + M10)/2, q2 = Re(M01 - M10)/2, q3 = Im(M00 - M11)/2.
 * Then Re tr(r M) = 2 (r0 q0 - r.q), maximal over unit r at r = (q0, -q)/|q|,
 * which is g = K^dagger / sqrt(det K^dagger) applied to the projection. */
static void su2_project(cplx m00, cplx m01, cplx m10, cplx m11, double q[4]) {
  q[0] = 0.5 * (m00.re + m11.re);
  q[1] = 0.5 * (m01.im + m10.im);
  q[2] = 0.5 * (m01.re - m10.re);
  q[3] = 0.5 * (m00.im - m11.im);
}

static void su2_maximum(const double q[4], double r[4]) {
  const double norm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (norm == 0.0) { /* degenerate block: every r is a maximum; keep identity */
    r[0] = 1.0;
    r[1] = r[2] = r[3] = 0.0;
    return;
  }
  r[0] = q[0] / norm;
  r[1] = -q[1] / norm;
  r[2] = -q[2] / norm;
  r[3] = -q[3] / norm;
}

/* Section 3.1: g^omega to first order, (1 - omega) 1 + omega g, back on SU(2). */
static void su2_overrelax(double r[4], double omega) {
  double s[4];
  s[0] = (1.0 - omega) + omega * r[0];
  s[1] = omega * r[1];
  s[2] = omega * r[2];
  s[3] = omega * r[3];
  const double norm = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
  for (int k = 0; k < 4; k++) r[k] = s[k] / norm;
}

/* Section 3.2: g -> g^2 (quaternion square). */
static void su2_square(double r[4]) {
  const double r0 = r[0];
  r[0] = r0 * r0 - (r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
  r[1] = 2.0 * r0 * r[1];
  r[2] = 2.0 * r0 * r[2];
  r[3] = 2.0 * r0 * r[3];
}

/* Embedding of the SU(2) element r into SU(3) acting on rows/cols (i, j). */
static su3 su2_embed(const double r[4], int i, int j) {
  su3 m = m_identity();
  m.e[i][i] = c_make(r[0], r[3]);
  m.e[i][j] = c_make(r[2], r[1]);
  m.e[j][i] = c_make(-r[2], r[1]);
  m.e[j][j] = c_make(r[0], -r[3]);
  return m;
}

static const int SUBGROUP[3][2] = {{0, 1}, {0, 2}, {1, 2}};

/* ------------------------------------------- maximally Abelian gauge */
/* Reading (the standard functional, which the text does not write down):
 *   F_MAG[U] = 1/(N_c N_d V) sum_{x,mu} sum_a |U_mu(x)_aa|^2,  maximised (N_d = 4).
 * Under g(x) = 1 + i eps T at one site the links U_mu(x) -> g U_mu(x) and
 * U_mu(x-mu) -> U_mu(x-mu) g^dagger change F_MAG by 2 eps Re tr[i T X(x)]
 * (times the normalisation), with
 *   X(x) = sum_mu ( U_mu(x) D_mu(x)^dagger - D_mu(x-mu)^dagger U_mu(x-mu) ),
 * D = the diagonal part of U.  So the gauge is reached where the traceless
 * part Delta_MAG(x) of (X - X^dagger)/(2i) vanishes, and the precision is
 *   theta_MAG = 1/(N_c V) sum_x tr[Delta_MAG(x) Delta_MAG(x)^dagger],
 * the same construction as the Landau-gauge theta with K(x) replaced by X(x).
 *
 * Local update, per SU(2) subgroup (i, j) as in Sec. 3: with R the subgroup
 * element, only the diagonal entries i, j of the site's 8 links change:
 * (R U)_ii, (R U)_jj for the forward links, (U R^dagger)_ii, (U R^dagger)_jj for
 * the backward ones.  Writing n.sigma = R^dagger sigma_3 R (on the block),
 *   |(R U)_ii|^2 + |(R U)_jj|^2 = const + n.(s(U_ii, U_ji) - s(U_ij, U_jj)) / 2,
 *   |(W R^dagger)_ii|^2 + |(W R^dagger)_jj|^2
 *                        = const + n.(s(W_ii*, W_ij*) - s(W_ji*, W_jj*)) / 2,
 * s(a, b) = (2 Re(a* b), 2 Im(a* b), |a|^2 - |b|^2): the site functional is
 * linear in the unit vector n, maximal at n = v/|v| with v the sum of those
 * vectors over the 8 links.  Left factors exp(i phi sigma_3) leave every
 * |diagonal entry| unchanged, so the maximisers form a circle; take the one
 * nearest the identity, the rotation of n onto e_3 about n x e_3:
 *   r = (|v| + v_3, -v_2, v_1, 0) / norm     (r = (0, 1, 0, 0) if v = -|v| e_3).
 * The subgroup steps run in the order (0,1), (0,2), (1,2) on the links as
 * updated by the steps before; overrelaxation and stochastic relaxation act
 * on r exactly as for Landau gauge (Sec. 3.1, 3.2). */
static void mag_s(cplx a, cplx b, double sign, double v[3]) {
  const cplx z = c_mul(c_conj(a), b);
  v[0] += sign * 2.0 * z.re;
  v[1] += sign * 2.0 * z.im;
  v[2] += sign * (a.re * a.re + a.im * a.im - b.re * b.re - b.im * b.im);
}

/* the vector v of subgroup (i, j) for the site's current links */
static void mag_vector(const su3 fwd[4], const su3 bwd[4], int i, int j, double v[3]) {
  v[0] = v[1] = v[2] = 0.0;
  for (int mu = 0; mu < 4; mu++) {
    mag_s(fwd[mu].e[i][i], fwd[mu].e[j][i], 1.0, v);
    mag_s(fwd[mu].e[i][j], fwd[mu].e[j][j], -1.0, v);
    mag_s(c_conj(bwd[mu].e[i][i]), c_conj(bwd[mu].e[i][j]), 1.0, v);
    mag_s(c_conj(bwd[mu].e[j][i]), c_conj(bwd[mu].e[j][j]), -1.0, v);
  }
}

/* the subgroup element nearest the identity that maximises n.v */
static void mag_maximum(const double v[3], double r[4]) {
  const double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  r[0] = 1.0; r[1] = r[2] = r[3] = 0.0;
  if (!(nv > 0.0)) return;
  const double a = nv + v[2];
  const double norm = sqrt(a * a + v[0] * v[0] + v[1] * v[1]);
  if (!(norm > 0.0)) {
    r[0] = 0.0; r[1] = 1.0;
    return;
  }
  r[0] = a / norm;
  r[1] = -v[1] / norm;
  r[2] = v[0] / norm;
  r[3] = 0.0;
}

/* sum over the four directions of sum_a |U_mu(x)_aa|^2 */
static double site_mag_functional(const double *links, int64_t site) {
  double s = 0.0;
  for (int mu = 0; mu < 4; mu++) {
    su3 u = load_link(links, site, mu);
    for (int a = 0; a < NC; a++) s += u.e[a][a].re * u.e[a][a].re + u.e[a][a].im * u.e[a][a].im;
  }
  return s;
}

static su3 m_diag(const su3 *u) {
  su3 d;
  memset(&d, 0, sizeof d);
  for (int a = 0; a < NC; a++) d.e[a][a] = u->e[a][a];
  return d;
}

/* X(x) of the current links */
static su3 mag_X(const lattice *l, const double *links, int64_t site) {
  su3 X;
  memset(&X, 0, sizeof X);
  for (int mu = 0; mu < 4; mu++) {
    su3 fwd = load_link(links, site, mu);
    su3 bwd = load_link(links, site_shift(l, site, mu, -1), mu);
    su3 df = m_diag(&fwd), db = m_diag(&bwd);
    su3 dfd = m_dagger(&df), dbd = m_dagger(&db);
    su3 t1 = m_mul(&fwd, &dfd);
    su3 t2 = m_mul(&dbd, &bwd);
    X = m_add(&X, &t1);
    X = m_sub(&X, &t2);
  }
  return X;
}

/* ------------------------------------ simulated annealing: SU(2) heat bath */
/* Simulated annealing (named by the paper as a preconditioner, Sec. 1; its
 * details are in a reference this text lacks) is read as sweeps whose SU(2)
 * subgroup elements are drawn from exp(beta Re tr[r M]) with respect to Haar
 * measure, beta rising over the sweeps.  With the block projection q,
 * Re tr[r M] = 2 |q| (r . p) for the maximum p = (q0, -q)/|q| (4-vector dot
 * product), so r = a p (matrix product) with a0 = x drawn from the density
 * proportional to sqrt(1 - x^2) exp(alpha x), alpha = 2 beta |q|, and the
 * vector part of a uniform on the sphere of radius sqrt(1 - x^2).  x is drawn
 * by the method of Kennedy and Pendleton (1985), at most SA_MAX_ATTEMPTS
 * tries; if all are rejected the subgroup is left unchanged. */
#define SA_TAG 0x53414842u /* "SAHB": heat-bath stream */
#define SA_MAX_ATTEMPTS 64u
#define SA_DIRECTION 0xFFFFFFu

/* uniform in (0, 1) from a 32-bit word */
static double unit_open(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* the four uniforms of (site, subgroup, attempt) in one sweep */
static void sa_uniforms(uint64_t seed, uint64_t sweep, int64_t site, int s, uint32_t attempt, double u[4]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {(uint32_t)site, ((uint32_t)s << 24) | attempt, (uint32_t)sweep, SA_TAG};
  uint32_t w[4];
  philox4x32_10(ctr, key, w);
  for (int k = 0; k < 4; k++) u[k] = unit_open(w[k]);
}

/* Kennedy-Pendleton draw of x in [-1, 1], density ~ sqrt(1 - x^2) exp(alpha x):
 * delta = -(ln u0 + cos^2(2 pi u1) ln u2) / alpha has density ~ sqrt(delta)
 * exp(-alpha delta); accepting with probability sqrt(1 - delta / 2) supplies
 * the rest of sqrt(1 - x^2) = sqrt(2 delta) sqrt(1 - delta / 2), x = 1 - delta.
 * Returns 0 on success, 1 when every attempt was rejected. */
static int kp_draw(double alpha, uint64_t seed, uint64_t sweep, int64_t site, int s, double *x, double *margin) {
  const double two_pi = 6.283185307179586476925286766559;
  for (uint32_t k = 0; k < SA_MAX_ATTEMPTS; k++) {
    double u[4];
    sa_uniforms(seed, sweep, site, s, k, u);
    const double c = cos(two_pi * u[1]);
    const double delta = -(log(u[0]) + c * c * log(u[2])) / alpha;
    if (margin) {  /* how close this comparison came to its threshold, relative to delta */
      const double m = fabs(u[3] * u[3] - (1.0 - 0.5 * delta)) / (fabs(delta) > 1.0 ? fabs(delta) : 1.0);
      if (m < *margin) *margin = m;
    }
    if (u[3] * u[3] <= 1.0 - 0.5 * delta) {
      *x = 1.0 - delta;
      return 0;
    }
  }
  return 1;
}

/* quaternion of the matrix product A B (matrices in the su2_embed convention) */
static void su2_mul(const double a[4], const double b[4], double r[4]) {
  const cplx a00 = c_make(a[0], a[3]), a01 = c_make(a[2], a[1]), a10 = c_make(-a[2], a[1]), a11 = c_make(a[0], -a[3]);
  const cplx b00 = c_make(b[0], b[3]), b01 = c_make(b[2], b[1]), b10 = c_make(-b[2], b[1]);
  const cplx c00 = c_add(c_mul(a00, b00), c_mul(a01, b10));
  const cplx c01 = c_add(c_mul(a00, b01), c_mul(a01, c_make(b[0], -b[3])));
  (void)a10;
  (void)a11;
  r[0] = c00.re;
  r[3] = c00.im;
  r[2] = c01.re;
  r[1] = c01.im;
}

/* heat-bath element for the block projection q at inverse temperature beta */
static void su2_heatbath(const double q[4], double beta, uint64_t seed, uint64_t sweep, int64_t site, int s,
                         double r[4], double *margin) {
  const double norm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double x;
  if (!(norm > 0.0) || !(beta > 0.0) || kp_draw(2.0 * beta * norm, seed, sweep, site, s, &x, margin)) {
    r[0] = 1.0; /* no update of this subgroup */
    r[1] = r[2] = r[3] = 0.0;
    return;
  }
  double p[4], u[4];
  su2_maximum(q, p);
  sa_uniforms(seed, sweep, site, s, SA_DIRECTION, u);
  const double two_pi = 6.283185307179586476925286766559;
  const double cth = 2.0 * u[0] - 1.0, sth = sqrt(1.0 - cth * cth), phi = two_pi * u[1];
  const double rad = sqrt(x * x < 1.0 ? 1.0 - x * x : 0.0);
  const double a[4] = {x, rad * sth * cos(phi), rad * sth * sin(phi), rad * cth};
  su2_mul(a, p, r);
}

/* the simulated-annealing schedule: beta rises geometrically from beta0 (sweep
 * 0) to beta1 (sweep n - 1) */
static double sa_beta(double beta0, double beta1, int n, int i) {
  if (n <= 1) return beta1;
  return beta0 * pow(beta1 / beta0, (double)i / (double)(n - 1));
}

typedef struct {
  int algo;          /* ORC_OR, ORC_SR or ORC_SA */
  double omega;      /* overrelaxation parameter */
  uint64_t sr_thr;   /* stochastic relaxation: accept iff draw < sr_thr */
  double beta;       /* simulated annealing: inverse temperature */
  uint64_t seed;     /* simulated annealing: stream of the site, sweep below */
  uint64_t sweep;
  int64_t site;
  double *margin;    /* simulated annealing, test support (nullable): the smallest relative margin of
                        the heat bath's accept/reject comparisons */
} update_rule;

/* Section 3: maximise f = Re tr[g K] by iterating over the three SU(2)
 * subgroups (Cabibbo-Marinari).  W = g K is the running matrix; each subgroup
 * element R maximises Re tr[R W] over its subgroup, then W <- R W, g <- R g.
 * trace_W / trace_R (nullable) receive W before each step and the R used. */
static su3 local_gauge_update(const su3 *K, const update_rule *rule, const uint32_t draws[3],
                              su3 *trace_W, su3 *trace_R) {
  su3 W = *K;
  su3 g = m_identity();
  for (int s = 0; s < 3; s++) {
    const int i = SUBGROUP[s][0], j = SUBGROUP[s][1];
    double q[4], r[4];
    su2_project(W.e[i][i], W.e[i][j], W.e[j][i], W.e[j][j], q);
    if (rule->algo == ORC_SA) {
      su2_heatbath(q, rule->beta, rule->seed, rule->sweep, rule->site, s, r, rule->margin);
    } else {
      su2_maximum(q, r);
      if (rule->algo == ORC_OR) {
        su2_overrelax(r, rule->omega);
      } else if ((uint64_t)draws[s] < rule->sr_thr) {
        su2_square(r);
      }
    }
    su3 R = su2_embed(r, i, j);
    if (trace_W) trace_W[s] = W;
    if (trace_R) trace_R[s] = R;
    W = m_mul(&R, &W);
    g = m_mul(&R, &g);
  }
  return g;
}

/* Maximally Abelian gauge: the subgroup steps on the site's own links (the
 * site functional is quadratic in g, so K(x) does not suffice).  fwd/bwd are
 * the 4 forward and 4 backward links; they are updated in place; returns g.
 * trace_v (nullable) receives the vector v of each step (3 x 3 doubles). */
static su3 mag_local_update(su3 fwd[4], su3 bwd[4], const update_rule *rule, const uint32_t draws[3],
                            double trace_v[3][3]) {
  su3 g = m_identity();
  for (int s = 0; s < 3; s++) {
    const int i = SUBGROUP[s][0], j = SUBGROUP[s][1];
    double v[3], r[4];
    mag_vector(fwd, bwd, i, j, v);
    if (trace_v) memcpy(trace_v[s], v, sizeof v);
    mag_maximum(v, r);
    if (rule->algo == ORC_OR) {
      su2_overrelax(r, rule->omega);
    } else if ((uint64_t)draws[s] < rule->sr_thr) {
      su2_square(r);
    }
    su3 R = su2_embed(r, i, j);
    su3 Rd = m_dagger(&R);
    for (int mu = 0; mu < 4; mu++) {
      fwd[mu] = m_mul(&R, &fwd[mu]);
      bwd[mu] = m_mul(&bwd[mu], &Rd);
    }
    g = m_mul(&R, &g);
  }
  return g;
}

/* Section 2 transformation, in place at one site:
 *   U_mu(x) <- g U_mu(x),  U_mu(x-mu) <- U_mu(x-mu) g^dagger
 * for every direction in the functional; Coulomb gauge optionally also the
 * temporal links (so the output stays a gauge transform of the input). */
static void apply_gauge_update(const lattice *l, double *links, int64_t site, const su3 *g, int gauge,
                               int transform_temporal) {
  su3 gd = m_dagger(g);
  const int mu0 = (gauge == ORC_COULOMB && !transform_temporal) ? 1 : 0;
  for (int mu = mu0; mu < 4; mu++) {
    su3 fwd = load_link(links, site, mu);
    fwd = m_mul(g, &fwd);
    store_link(links, site, mu, &fwd);
    const int64_t back = site_shift(l, site, mu, -1);
    su3 bwd = load_link(links, back, mu);
    bwd = m_mul(&bwd, &gd);
    store_link(links, back, mu, &bwd);
  }
}

typedef struct {
  int gauge;
  update_rule rule;
  uint64_t seed;
  int transform_temporal;
  int64_t site_offset; /* added to a site's index where it keys random streams (a slab of a larger lattice) */
} sweep_cfg;

/* g of one site update on the current links (which it does not touch) */
static su3 site_g(const lattice *l, const double *links, int64_t site, const sweep_cfg *cfg, uint64_t sweep) {
  uint32_t u[3] = {0, 0, 0};
  if (cfg->rule.algo == ORC_SR) sr_draws(cfg->seed, sweep, site + cfg->site_offset, u);
  update_rule rule = cfg->rule;
  rule.seed = cfg->seed;
  rule.sweep = sweep;
  rule.site = site + cfg->site_offset;
  if (cfg->gauge == ORC_MAG) {
    su3 fwd[4], bwd[4];
    for (int mu = 0; mu < 4; mu++) {
      fwd[mu] = load_link(links, site, mu);
      bwd[mu] = load_link(links, site_shift(l, site, mu, -1), mu);
    }
    return mag_local_update(fwd, bwd, &rule, u, NULL);
  }
  su3 K = gather_K(l, links, site, cfg->gauge);
  return local_gauge_update(&K, &rule, u, NULL, NULL);
}

static void update_site(const lattice *l, double *links, int64_t site, const sweep_cfg *cfg, uint64_t sweep) {
  su3 g = site_g(l, links, site, cfg, sweep);
  apply_gauge_update(l, links, site, &g, cfg->gauge, cfg->transform_temporal);
}

/* lexicographic site of the idx-th site of a parity (sites of one parity are
 * every other site along x1, N1 even) */
static int64_t parity_site(const lattice *l, int parity, int64_t idx) {
  const int64_t half1 = l->n[1] / 2;
  const int64_t row = idx / half1; /* (x2, x3, t) row */
  const int64_t j = idx % half1;
  int64_t x[4];
  x[2] = row % l->n[2];
  x[3] = (row / l->n[2]) % l->n[3];
  x[0] = row / (l->n[2] * l->n[3]);
  x[1] = 2 * j + ((parity + x[0] + x[2] + x[3]) & 1);
  return site_index(l, x);
}

/* One half-sweep: every site of `parity` (and, for Coulomb, of an active
 * timeslice) gets its local update.  `order` (nullable) fixes a site order
 * and runs single-threaded; the result does not depend on it. */
static void half_sweep(const lattice *l, double *links, int parity, const sweep_cfg *cfg, uint64_t sweep,
                       const uint8_t *active, const int64_t *order) {
  const int64_t nh = l->vol / 2;
  if (order) {
    for (int64_t k = 0; k < nh; k++) {
      const int64_t site = parity_site(l, parity, order[k]);
      if (active && !active[site_time(l, site)]) continue;
      update_site(l, links, site, cfg, sweep);
    }
    return;
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nh; k++) {
    const int64_t site = parity_site(l, parity, k);
    if (active && !active[site_time(l, site)]) continue;
    update_site(l, links, site, cfg, sweep);
  }
}

/* ------------------------------------------------ Section 2: F and theta */
/* A_mu(x) = traceless part of (U_mu(x) - U_mu(x)^dagger) / (2i) */
static su3 gauge_field_A(const su3 *u) {
  su3 ud = m_dagger(u);
  su3 d = m_sub(u, &ud);
  su3 a;
  for (int r = 0; r < NC; r++)
    for (int c = 0; c < NC; c++) a.e[r][c] = c_make(0.5 * d.e[r][c].im, -0.5 * d.e[r][c].re); /* d / (2i) */
  const double tr3 = (a.e[0][0].re + a.e[1][1].re + a.e[2][2].re) / 3.0;
  for (int r = 0; r < NC; r++) a.e[r][r].re -= tr3;
  return a;
}

/* tr[Delta(x) Delta(x)^dagger] with Delta(x) = sum_mu (A_mu(x) - A_mu(x-mu)) */
static double violation_norm(const lattice *l, const double *links, int64_t site, int gauge) {
  su3 delta;
  memset(&delta, 0, sizeof delta);
  for (int mu = first_mu(gauge); mu < 4; mu++) {
    su3 fwd = load_link(links, site, mu);
    su3 bwd = load_link(links, site_shift(l, site, mu, -1), mu);
    su3 af = gauge_field_A(&fwd);
    su3 ab = gauge_field_A(&bwd);
    delta = m_add(&delta, &af);
    delta = m_sub(&delta, &ab);
  }
  double s = 0.0;
  for (int r = 0; r < NC; r++)
    for (int c = 0; c < NC; c++) s += delta.e[r][c].re * delta.e[r][c].re + delta.e[r][c].im * delta.e[r][c].im;
  return s;
}

/* sum over the functional's directions of Re tr U_mu(x) */
static double site_retrace(const double *links, int64_t site, int gauge) {
  double s = 0.0;
  for (int mu = first_mu(gauge); mu < 4; mu++) {
    su3 u = load_link(links, site, mu);
    s += m_retrace(&u);
  }
  return s;
}

/* sum over the six planes of Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger */
static double site_plaquettes(const lattice *l, const double *links, int64_t site) {
  double s = 0.0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++) {
      su3 a = load_link(links, site, mu);
      su3 b = load_link(links, site_shift(l, site, mu, +1), nu);
      su3 c = load_link(links, site_shift(l, site, nu, +1), mu);
      su3 d = load_link(links, site, nu);
      su3 cd = m_dagger(&c), dd = m_dagger(&d);
      su3 p = m_mul(&a, &b);
      p = m_mul(&p, &cd);
      p = m_mul(&p, &dd);
      s += m_retrace(&p);
    }
  return s;
}

/* --------------------------------------------------------- public entries */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static int check_dims(const int32_t dims[4]) {
  for (int d = 0; d < 4; d++)
    if (dims[d] < 2 || (dims[d] & 1)) return -1;
  return 0;
}

/* Exact measurement, fixed summation order.
 * Landau: F (Section 2 functional), theta (Section 2 precision), plaquette.
 * Maximally Abelian gauge: F_MAG and theta_MAG (see its section), plaquette.
 * Coulomb: F_t and theta_t per timeslice (spatial directions, N_d = 3,
 * V -> V_s); F = mean_t F_t, theta = max_t theta_t.  F_t / theta_t may be NULL. */
int orc_measure(const int32_t dims[4], const double *links, int gauge, double *F, double *theta, double *plaq,
                double *F_t, double *theta_t) {
  if (check_dims(dims)) return -1;
  const lattice l = make_lattice(dims);
  double *sf = (double *)malloc(sizeof(double) * (size_t)l.vol);
  double *st = (double *)malloc(sizeof(double) * (size_t)l.vol);
  double *sp = (double *)malloc(sizeof(double) * (size_t)l.vol);
  if (!sf || !st || !sp) {
    free(sf); free(st); free(sp);
    return -2;
  }
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < l.vol; x++) {
    if (gauge == ORC_MAG) {
      sf[x] = site_mag_functional(links, x);
      su3 X = mag_X(&l, links, x);
      su3 d = gauge_field_A(&X); /* traceless part of (X - X^dagger)/(2i) */
      double v = 0.0;
      for (int r = 0; r < NC; r++)
        for (int c = 0; c < NC; c++) v += d.e[r][c].re * d.e[r][c].re + d.e[r][c].im * d.e[r][c].im;
      st[x] = v;
    } else {
      sf[x] = site_retrace(links, x, gauge);
      st[x] = violation_norm(&l, links, x, gauge);
    }
    sp[x] = site_plaquettes(&l, links, x);
  }
  const int nd = gauge == ORC_COULOMB ? 3 : 4;
  double tot_f = 0.0, tot_t = 0.0, tot_p = 0.0, max_t = 0.0;
  for (int64_t t = 0; t < l.n[0]; t++) {
    double slf = 0.0, slt = 0.0, slp = 0.0;
    for (int64_t k = 0; k < l.vol_s; k++) {
      slf += sf[t * l.vol_s + k];
      slt += st[t * l.vol_s + k];
      slp += sp[t * l.vol_s + k];
    }
    tot_f += slf;
    tot_t += slt;
    tot_p += slp;
    const double ft = slf / ((double)NC * nd * (double)l.vol_s);
    const double tt = slt / ((double)NC * (double)l.vol_s);
    if (F_t) F_t[t] = ft;
    if (theta_t) theta_t[t] = tt;
    if (tt > max_t) max_t = tt;
  }
  if (gauge == ORC_COULOMB) {
    *F = tot_f / ((double)NC * nd * (double)l.vol);
    *theta = max_t;
  } else {
    *F = tot_f / ((double)NC * nd * (double)l.vol);
    *theta = tot_t / ((double)NC * (double)l.vol);
  }
  if (plaq) *plaq = tot_p / ((double)NC * 6.0 * (double)l.vol);
  free(sf);
  free(st);
  free(sp);
  return 0;
}

static sweep_cfg make_cfg(int gauge, int algo, double omega, double p, uint64_t seed, int transform_temporal) {
  sweep_cfg c;
  c.gauge = gauge;
  c.rule.algo = algo;
  c.rule.omega = omega;
  c.rule.sr_thr = sr_threshold(p);
  c.rule.beta = 0.0;
  c.rule.seed = seed;
  c.rule.sweep = 0;
  c.rule.site = 0;
  c.rule.margin = NULL;
  c.seed = seed;
  c.transform_temporal = transform_temporal;
  c.site_offset = 0;
  return c;
}

/* One half-sweep over `parity`.  active (nullable): per-timeslice mask.
 * order (nullable): the V/2 within-parity indices in the order to visit. */
int orc_half_sweep(const int32_t dims[4], double *links, int gauge, int parity, int algo, double omega, double p,
                   uint64_t seed, uint64_t sweep, int transform_temporal, const uint8_t *active,
                   const int64_t *order) {
  if (check_dims(dims)) return -1;
  const lattice l = make_lattice(dims);
  const sweep_cfg cfg = make_cfg(gauge, algo, omega, p, seed, transform_temporal);
  half_sweep(&l, links, parity & 1, &cfg, sweep, active, order);
  return 0;
}

/* As orc_half_sweep on a slab of a larger lattice held with its own geometry:
 * the random streams are keyed by site + site_offset, the site's index in the
 * whole lattice (the slab's first slice at global slice t0: site_offset =
 * t0 * V_s minus the slices held before it).  Which sites are updated is the
 * caller's `active` mask. */
int orc_half_sweep_offset(const int32_t dims[4], double *links, int gauge, int parity, int algo, double omega,
                          double p, uint64_t seed, uint64_t sweep, int transform_temporal, const uint8_t *active,
                          int64_t site_offset) {
  if (check_dims(dims)) return -1;
  const lattice l = make_lattice(dims);
  sweep_cfg cfg = make_cfg(gauge, algo, omega, p, seed, transform_temporal);
  cfg.site_offset = site_offset;
  half_sweep(&l, links, parity & 1, &cfg, sweep, active, NULL);
  return 0;
}

/* n full sweeps (even then odd), numbered sweep0, sweep0+1, ... */
int orc_sweeps(const int32_t dims[4], double *links, int gauge, int algo, double omega, double p, uint64_t seed,
               uint64_t sweep0, int n, int transform_temporal, const uint8_t *active) {
  if (check_dims(dims)) return -1;
  const lattice l = make_lattice(dims);
  const sweep_cfg cfg = make_cfg(gauge, algo, omega, p, seed, transform_temporal);
  for (int s = 0; s < n; s++) {
    half_sweep(&l, links, 0, &cfg, sweep0 + (uint64_t)s, active, NULL);
    half_sweep(&l, links, 1, &cfg, sweep0 + (uint64_t)s, active, NULL);
  }
  return 0;
}

/* The links one site update would write, without touching the field:
 * out[0..3] = new U_mu(x), out[4..7] = new U_mu(x-mu), 18 doubles each
 * (directions the update does not touch are copied unchanged). */
int orc_site_new_links(const int32_t dims[4], const double *links, int64_t site, int gauge, int algo, double omega,
                       double p, uint64_t seed, uint64_t sweep, int transform_temporal, double *out) {
  if (check_dims(dims)) return -1;
  const lattice l = make_lattice(dims);
  if (site < 0 || site >= l.vol) return -1;
  const sweep_cfg cfg = make_cfg(gauge, algo, omega, p, seed, transform_temporal);
  su3 g = site_g(&l, links, site, &cfg, sweep);
  su3 gd = m_dagger(&g);
  const int mu0 = (gauge == ORC_COULOMB && !transform_temporal) ? 1 : 0;
  for (int mu = 0; mu < 4; mu++) {
    su3 fwd = load_link(links, site, mu);
    su3 bwd = load_link(links, site_shift(&l, site, mu, -1), mu);
    if (mu >= mu0) {
      fwd = m_mul(&g, &fwd);
      bwd = m_mul(&bwd, &gd);
    }
    for (int a = 0; a < NC; a++)
      for (int b = 0; b < NC; b++) {
        out[mu * 18 + 2 * (3 * a + b)] = fwd.e[a][b].re;
        out[mu * 18 + 2 * (3 * a + b) + 1] = fwd.e[a][b].im;
        out[(4 + mu) * 18 + 2 * (3 * a + b)] = bwd.e[a][b].re;
        out[(4 + mu) * 18 + 2 * (3 * a + b) + 1] = bwd.e[a][b].im;
      }
  }
  return 0;
}

static void to_su3(const double *p, su3 *m) {
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) m->e[a][b] = c_make(p[2 * (3 * a + b)], p[2 * (3 * a + b) + 1]);
}

static void from_su3(const su3 *m, double *p) {
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) {
      p[2 * (3 * a + b)] = m->e[a][b].re;
      p[2 * (3 * a + b) + 1] = m->e[a][b].im;
    }
}

/* The local update of a given K (18 doubles), with its intermediate steps:
 * g_out = g, W_out[s] = W before subgroup step s, R_out[s] = embedded R_s
 * (3 x 18 doubles each, nullable). draws: three uint32 (ignored for OR). */
void orc_local_update(const double *K, int algo, double omega, double p, const uint32_t *draws, double *g_out,
                      double *W_out, double *R_out) {
  su3 k, W[3], R[3];
  to_su3(K, &k);
  update_rule rule;
  rule.algo = algo;
  rule.omega = omega;
  rule.sr_thr = sr_threshold(p);
  rule.beta = 0.0;
  rule.seed = 0;
  rule.sweep = 0;
  rule.site = 0;
  rule.margin = NULL;
  uint32_t u[3] = {0, 0, 0};
  if (draws) { u[0] = draws[0]; u[1] = draws[1]; u[2] = draws[2]; }
  su3 g = local_gauge_update(&k, &rule, u, W, R);
  from_su3(&g, g_out);
  for (int s = 0; s < 3; s++) {
    if (W_out) from_su3(&W[s], W_out + 18 * s);
    if (R_out) from_su3(&R[s], R_out + 18 * s);
  }
}

/* Conditioning of the site updates of one parity on the current links.
 * TEST INFRASTRUCTURE for the FP32 parity bounds: a site update computed in
 * FP32 is off from the FP64 one by about (rounding of its input) x (this
 * number), to first order.  The steps follow the update rule (overrelaxation
 * or stochastic relaxation), so each subgroup sees what the steps before it
 * left.
 *   Landau, Coulomb: kappa = 1 / min_s |q_s|, q_s the quaternion projection of
 *     the running W's (i, j) block before step s (Sec. 3 closed form: the
 *     subgroup element is (q0, -q)/|q|, whose first-order change is at most
 *     |dq| / |q|).
 *   Maximally Abelian gauge: kappa = sum_s sqrt(2 / (|v_s| (|v_s| + v_s3))):
 *     the element r = (|v| + v_3, -v_2, v_1, 0) / sqrt(2 |v| (|v| + v_3))
 *     depends on v through n = v/|v| (|dn| <= |dv| / |v|) and, near
 *     n = -e_3, through the rotation axis n x e_3 (|dr| grows as
 *     1 / sqrt(1 + n_3)); the three steps compound, so their terms add.
 * out[site] (V doubles) for the sites of `parity` (Coulomb: of every slice),
 * left untouched elsewhere; +infinity where a step is degenerate. */
int orc_site_conditioning(const int32_t dims[4], const double *links, int gauge, int parity, int algo, double omega,
                          double p, uint64_t seed, uint64_t sweep, double *out) {
  if (check_dims(dims)) return -1;
  if (algo != ORC_OR && algo != ORC_SR) return -1;
  const lattice l = make_lattice(dims);
  sweep_cfg cfg = make_cfg(gauge, algo, omega, p, seed, 1);
  const int64_t nh = l.vol / 2;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nh; k++) {
    const int64_t site = parity_site(&l, parity, k);
    uint32_t u[3] = {0, 0, 0};
    if (algo == ORC_SR) sr_draws(seed, sweep, site, u);
    update_rule rule = cfg.rule;
    rule.seed = seed;
    rule.sweep = sweep;
    rule.site = site;
    double kappa = 0.0;
    if (gauge == ORC_MAG) {
      su3 fwd[4], bwd[4];
      for (int mu = 0; mu < 4; mu++) {
        fwd[mu] = load_link(links, site, mu);
        bwd[mu] = load_link(links, site_shift(&l, site, mu, -1), mu);
      }
      double v[3][3];
      mag_local_update(fwd, bwd, &rule, u, v);
      for (int s = 0; s < 3; s++) {
        const double nv = sqrt(v[s][0] * v[s][0] + v[s][1] * v[s][1] + v[s][2] * v[s][2]);
        const double d = nv * (nv + v[s][2]);
        kappa += d > 0.0 ? sqrt(2.0 / d) : INFINITY;
      }
    } else {
      su3 K = gather_K(&l, links, site, gauge), W[3];
      local_gauge_update(&K, &rule, u, W, NULL);
      double qmin = INFINITY;
      for (int s = 0; s < 3; s++) {
        const int i = SUBGROUP[s][0], j = SUBGROUP[s][1];
        double q[4];
        su2_project(W[s].e[i][i], W[s].e[i][j], W[s].e[j][i], W[s].e[j][j], q);
        const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (nq < qmin) qmin = nq;
      }
      kappa = qmin > 0.0 ? 1.0 / qmin : INFINITY;
    }
    out[site] = kappa;
  }
  return 0;
}

/* Per timeslice, the sum over the sites of one parity of the site violation
 * tr[Delta(x) Delta(x)^dagger] of Sec. 2 (Delta from the A_mu of the links;
 * maximally Abelian gauge: from X(x)) on the current links.  TEST
 * INFRASTRUCTURE: the sweeps' fused estimate of theta adds exactly these over
 * its two half-sweeps, each on the field that half-sweep started from.
 * out_t: N_t doubles. */
int orc_parity_violation(const int32_t dims[4], const double *links, int gauge, int parity, double *out_t) {
  if (check_dims(dims)) return -1;
  const lattice l = make_lattice(dims);
  double *sv = (double *)malloc(sizeof(double) * (size_t)l.vol);
  if (!sv) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < l.vol; x++) {
    if (site_parity(&l, x) != (parity & 1)) {
      sv[x] = 0.0;
    } else if (gauge == ORC_MAG) {
      su3 X = mag_X(&l, links, x);
      su3 d = gauge_field_A(&X);
      double v = 0.0;
      for (int r = 0; r < NC; r++)
        for (int c = 0; c < NC; c++) v += d.e[r][c].re * d.e[r][c].re + d.e[r][c].im * d.e[r][c].im;
      sv[x] = v;
    } else {
      sv[x] = violation_norm(&l, links, x, gauge);
    }
  }
  for (int64_t t = 0; t < l.n[0]; t++) {
    double s = 0.0;
    for (int64_t k = 0; k < l.vol_s; k++) s += sv[t * l.vol_s + k];
    out_t[t] = s;
  }
  free(sv);
  return 0;
}

/* One simulated-annealing half-sweep over `parity` at inverse temperature
 * beta (the heat-bath steps of orc_sa_sweeps; see su2_heatbath). */
int orc_sa_half_sweep(const int32_t dims[4], double *links, int gauge, int parity, double beta, uint64_t seed,
                      uint64_t sweep, int transform_temporal) {
  if (check_dims(dims) || !(beta > 0.0) || gauge == ORC_MAG) return -1;
  const lattice l = make_lattice(dims);
  sweep_cfg cfg = make_cfg(gauge, ORC_SA, 1.0, 0.0, seed, transform_temporal);
  cfg.rule.beta = beta;
  half_sweep(&l, links, parity & 1, &cfg, sweep, NULL, NULL);
  return 0;
}

/* Per site of one parity, for the annealing update at inverse temperature beta
 * on the current links (TEST INFRASTRUCTURE for the FP32 annealing parity):
 * kappa_out[site] = 1 / min_s |q_s| as orc_site_conditioning, and
 * margin_out[site] = the smallest relative margin |u_3^2 - (1 - delta/2)| /
 * max(1, |delta|) of the Kennedy-Pendleton comparisons the update evaluates:
 * where it is within FP32 rounding, an FP32 update may take the other branch
 * and draw a different element.  Sites of the other parity are left untouched. */
int orc_sa_site_stats(const int32_t dims[4], const double *links, int gauge, int parity, double beta, uint64_t seed,
                      uint64_t sweep, double *kappa_out, double *margin_out) {
  if (check_dims(dims) || !(beta > 0.0) || gauge == ORC_MAG) return -1;
  const lattice l = make_lattice(dims);
  const sweep_cfg cfg = make_cfg(gauge, ORC_SA, 1.0, 0.0, seed, 1);
  const int64_t nh = l.vol / 2;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nh; k++) {
    const int64_t site = parity_site(&l, parity, k);
    update_rule rule = cfg.rule;
    double margin = INFINITY;
    rule.beta = beta;
    rule.seed = seed;
    rule.sweep = sweep;
    rule.site = site;
    rule.margin = &margin;
    const uint32_t u[3] = {0, 0, 0};
    su3 K = gather_K(&l, links, site, gauge), W[3];
    local_gauge_update(&K, &rule, u, W, NULL);
    double qmin = INFINITY;
    for (int s = 0; s < 3; s++) {
      const int i = SUBGROUP[s][0], j = SUBGROUP[s][1];
      double q[4];
      su2_project(W[s].e[i][i], W[s].e[i][j], W[s].e[j][i], W[s].e[j][j], q);
      const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      if (nq < qmin) qmin = nq;
    }
    kappa_out[site] = qmin > 0.0 ? 1.0 / qmin : INFINITY;
    margin_out[site] = margin;
  }
  return 0;
}

/* K(x) of the current links (18 doubles) */
int orc_gather_K(const int32_t dims[4], const double *links, int64_t site, int gauge, double *K_out) {
  if (check_dims(dims)) return -1;
  const lattice l = make_lattice(dims);
  su3 k = gather_K(&l, links, site, gauge);
  from_su3(&k, K_out);
  return 0;
}

/* closed-form SU(2) maximum of a 2x2 complex block (8 doubles, row-major) */
void orc_su2_maximum(const double *M, double *r_out) {
  double q[4];
  su2_project(c_make(M[0], M[1]), c_make(M[2], M[3]), c_make(M[4], M[5]), c_make(M[6], M[7]), q);
  su2_maximum(q, r_out);
}

void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) { philox4x32_10(ctr, key, out); }

void orc_sr_draws(uint64_t seed, uint64_t sweep, int64_t site, uint32_t *out) { sr_draws(seed, sweep, site, out); }

/* Driver loop of Section 4: sweep (even, odd) until the precision theta
 * reaches tol, measuring exactly every check_every sweeps (and before the
 * first).  Coulomb: per-timeslice convergence, converged slices are no longer
 * updated; converged when every theta_t < tol.
 * Returns 0 converged, 1 not converged within max_sweeps, <0 on error. */
/* Simulated annealing: n heat-bath sweeps (even then odd), sweep numbers
 * sweep0 .. sweep0+n-1, beta from the geometric schedule sa_beta. */
int orc_sa_sweeps(const int32_t dims[4], double *links, int gauge, double beta0, double beta1, int n, uint64_t seed,
                  uint64_t sweep0, int transform_temporal) {
  if (check_dims(dims) || n < 0 || !(beta0 > 0.0) || !(beta1 > 0.0) || gauge == ORC_MAG) return -1;
  const lattice l = make_lattice(dims);
  for (int i = 0; i < n; i++) {
    sweep_cfg cfg = make_cfg(gauge, ORC_SA, 1.0, 0.0, seed, transform_temporal);
    cfg.rule.beta = sa_beta(beta0, beta1, n, i);
    half_sweep(&l, links, 0, &cfg, sweep0 + (uint64_t)i, NULL, NULL);
    half_sweep(&l, links, 1, &cfg, sweep0 + (uint64_t)i, NULL, NULL);
  }
  return 0;
}

/* n Kennedy-Pendleton draws at alpha (stream: site = draw index, subgroup 0,
 * sweep 0); returns how many failed (all attempts rejected; out = NaN). */
int orc_kp_draws(double alpha, int64_t n, uint64_t seed, double *out) {
  int fails = 0;
  for (int64_t k = 0; k < n; k++) {
    double x;
    if (kp_draw(alpha, seed, 0, k, 0, &x, NULL)) {
      out[k] = NAN;
      fails++;
    } else {
      out[k] = x;
    }
  }
  return fails;
}

/* The heat-bath SU(2) element for one block projection q (as the sweep
 * would draw it for site, subgroup s, sweep). */
void orc_su2_heatbath(const double *q, double beta, uint64_t seed, uint64_t sweep, int64_t site, int s,
                      double *r_out) {
  su2_heatbath(q, beta, seed, sweep, site, s, r_out, NULL);
}

double orc_sa_beta(double beta0, double beta1, int n, int i) { return sa_beta(beta0, beta1, n, i); }

int orc_fix(const int32_t dims[4], double *links, int gauge, int algo, double omega, double p, uint64_t seed,
            double tol, int max_sweeps, int check_every, int transform_temporal, int *sweeps_out, double *F_out,
            double *theta_out) {
  if (check_dims(dims) || check_every < 1) return -1;
  const lattice l = make_lattice(dims);
  const sweep_cfg cfg = make_cfg(gauge, algo, omega, p, seed, transform_temporal);
  uint8_t *active = NULL;
  double *ft = NULL, *tt = NULL;
  if (gauge == ORC_COULOMB) {
    active = (uint8_t *)malloc((size_t)l.n[0]);
    ft = (double *)malloc(sizeof(double) * (size_t)l.n[0]);
    tt = (double *)malloc(sizeof(double) * (size_t)l.n[0]);
    if (!active || !ft || !tt) {
      free(active); free(ft); free(tt);
      return -2;
    }
    memset(active, 1, (size_t)l.n[0]);
  }
  int sweeps = 0, rc = 1;
  double F = 0.0, theta = 0.0;
  for (;;) {
    if (orc_measure(dims, links, gauge, &F, &theta, NULL, ft, tt)) { rc = -2; break; }
    if (gauge == ORC_COULOMB)
      for (int64_t t = 0; t < l.n[0]; t++)
        if (tt[t] < tol) active[t] = 0;
    if (theta < tol) { rc = 0; break; }
    if (sweeps >= max_sweeps) { rc = 1; break; }
    const int n = (max_sweeps - sweeps) < check_every ? (max_sweeps - sweeps) : check_every;
    for (int s = 0; s < n; s++) {
      half_sweep(&l, links, 0, &cfg, (uint64_t)sweeps, active, NULL);
      half_sweep(&l, links, 1, &cfg, (uint64_t)sweeps, active, NULL);
      sweeps++;
    }
  }
  *sweeps_out = sweeps;
  *F_out = F;
  *theta_out = theta;
  free(active);
  free(ft);
  free(tt);
  return rc;
}

/* Maximally Abelian gauge, one subgroup step on a site's links given
 * directly: links8 = 4 forward then 4 backward links (18 doubles each);
 * returns the vector v and the maximising element r (before overrelaxation). */
void orc_mag_subgroup(const double *links8, int s, double *v_out, double *r_out) {
  su3 fwd[4], bwd[4];
  for (int mu = 0; mu < 4; mu++) {
    to_su3(links8 + 18 * mu, &fwd[mu]);
    to_su3(links8 + 18 * (4 + mu), &bwd[mu]);
  }
  mag_vector(fwd, bwd, SUBGROUP[s][0], SUBGROUP[s][1], v_out);
  mag_maximum(v_out, r_out);
}
