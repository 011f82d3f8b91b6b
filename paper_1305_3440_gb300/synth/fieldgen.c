/*
 * Seeded synthetic SU(3) gauge fields: the input generator shared by the
 * FP64 CPU oracle's tests and the CUDA path's tests and benchmark.
 *
 * This module only MAKES inputs.  It contains none of the gauge-fixing
 * arithmetic (no K(x), no SU(2) maximisation, no F or theta); the oracle and
 * the CUDA library each have their own.  The recipe:
 *
 *   U_mu(x) = exp(i eps sum_{a=1..8} r_a lambda_a / 2),  r_a ~ N(0,1)
 *   U_mu(x) <- h(x) U_mu(x) h(x+mu)^dagger,               h(x) Haar on SU(3)
 *
 * so eps = 0 gives a pure-gauge field h(x) h(x+mu)^dagger, whose Landau
 * gauge-fixed form is the unit field (F = 1, theta = 0), and eps > 0 gives a
 * rough field hidden behind a random gauge, the kind of input the relaxation
 * of Section 3 is meant for.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
 * here from that paper's definition, keyed by the 64-bit seed and counted by
 * (site, kind, block, tag), so every site is generated independently and the
 * output does not depend on the thread count.  Normals by Box-Muller.
 *
 * Layout of the output (also the public link layout of the library):
 *   links[((site*4 + mu)*9 + 3*row + col)*2 + {0: re, 1: im}]   (complex128)
 *   site = x1 + N1*(x2 + N2*(x3 + N3*t)),   dims = {N_t, N_3, N_2, N_1}
 *   mu = 0 is t, mu = 1, 2, 3 are x1, x2, x3.
 *
 * Built with -ffp-contract=off so x86-64 and aarch64 hosts agree to rounding.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } zc;

static zc zmul(zc a, zc b) { zc r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static zc zadd(zc a, zc b) { zc r = {a.re + b.re, a.im + b.im}; return r; }
static zc zconj(zc a) { zc r = {a.re, -a.im}; return r; }
static zc zscale(zc a, double s) { zc r = {a.re * s, a.im * s}; return r; }

typedef struct { zc m[3][3]; } mat3;

static mat3 mat_mul(const mat3 *a, const mat3 *b) {
  mat3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      zc s = {0.0, 0.0};
      for (int k = 0; k < 3; k++) s = zadd(s, zmul(a->m[i][k], b->m[k][j]));
      r.m[i][j] = s;
    }
  return r;
}

static mat3 mat_dagger(const mat3 *a) {
  mat3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r.m[i][j] = zconj(a->m[j][i]);
  return r;
}

/* ---- Philox4x32-10 (own implementation of the published definition) ---- */
static void gen_philox(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

#define GEN_TAG 0x47454E31u /* "GEN1": keeps these streams apart from other users of the seed */

/* n standard normals for (site, kind); n <= 20. */
static void gen_normals(uint64_t seed, uint64_t site, uint32_t kind, int n, double *z) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
  int got = 0;
  for (uint32_t block = 0; got < n; block++) {
    const uint32_t ctr[4] = {(uint32_t)site, (uint32_t)(site >> 32) ^ (kind << 24), block, GEN_TAG};
    uint32_t r[4];
    gen_philox(ctr, key, r);
    for (int pair = 0; pair < 2 && got < n; pair++) {
      double u1 = ((double)r[2 * pair] + 0.5) * (1.0 / 4294967296.0);
      double u2 = ((double)r[2 * pair + 1] + 0.5) * (1.0 / 4294967296.0);
      double rad = sqrt(-2.0 * log(u1));
      z[got++] = rad * cos(two_pi * u2);
      if (got < n) z[got++] = rad * sin(two_pi * u2);
    }
  }
}

/* Make a near-unitary 3x3 exactly special unitary: Gram-Schmidt on rows 0 and 1,
 * then row 2 = conj(row0 x row1), which makes det = 1. */
static void gen_reunitarise(mat3 *u) {
  double n0 = 0.0;
  for (int j = 0; j < 3; j++) n0 += u->m[0][j].re * u->m[0][j].re + u->m[0][j].im * u->m[0][j].im;
  n0 = 1.0 / sqrt(n0);
  for (int j = 0; j < 3; j++) u->m[0][j] = zscale(u->m[0][j], n0);
  zc ip = {0.0, 0.0}; /* <row0, row1> = sum conj(r0) r1 */
  for (int j = 0; j < 3; j++) ip = zadd(ip, zmul(zconj(u->m[0][j]), u->m[1][j]));
  for (int j = 0; j < 3; j++) {
    zc t = zmul(ip, u->m[0][j]);
    u->m[1][j].re -= t.re;
    u->m[1][j].im -= t.im;
  }
  double n1 = 0.0;
  for (int j = 0; j < 3; j++) n1 += u->m[1][j].re * u->m[1][j].re + u->m[1][j].im * u->m[1][j].im;
  n1 = 1.0 / sqrt(n1);
  for (int j = 0; j < 3; j++) u->m[1][j] = zscale(u->m[1][j], n1);
  for (int j = 0; j < 3; j++) {
    int a = (j + 1) % 3, b = (j + 2) % 3;
    zc c = zadd(zmul(u->m[0][a], u->m[1][b]), zscale(zmul(u->m[0][b], u->m[1][a]), -1.0));
    u->m[2][j] = zconj(c);
  }
}

/* exp(X) by scaling and squaring of a truncated Taylor series. */
static mat3 gen_expm(const mat3 *x) {
  double nrm = 0.0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) nrm += x->m[i][j].re * x->m[i][j].re + x->m[i][j].im * x->m[i][j].im;
  nrm = sqrt(nrm);
  int s = 0;
  while (nrm > 0.25) { nrm *= 0.5; s++; }
  double scale = ldexp(1.0, -s);
  mat3 y, term, sum;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      y.m[i][j] = zscale(x->m[i][j], scale);
      zc one = {i == j ? 1.0 : 0.0, 0.0};
      term.m[i][j] = one;
      sum.m[i][j] = one;
    }
  for (int k = 1; k <= 18; k++) {
    term = mat_mul(&term, &y);
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        term.m[i][j] = zscale(term.m[i][j], 1.0 / k);
        sum.m[i][j] = zadd(sum.m[i][j], term.m[i][j]);
      }
  }
  for (int k = 0; k < s; k++) sum = mat_mul(&sum, &sum);
  return sum;
}

/* exp(i eps sum_a r_a lambda_a / 2) with the Gell-Mann matrices lambda_1..8. */
static mat3 gen_link(uint64_t seed, uint64_t site, int mu, double eps) {
  double r[8];
  gen_normals(seed, site, (uint32_t)mu, 8, r);
  const double inv_sqrt3 = 0.57735026918962576450914878050196;
  /* H = sum_a r_a lambda_a / 2, Hermitian and traceless */
  mat3 h;
  memset(&h, 0, sizeof h);
  h.m[0][1].re += r[0]; h.m[1][0].re += r[0];             /* lambda_1 */
  h.m[0][1].im += -r[1]; h.m[1][0].im += r[1];            /* lambda_2 */
  h.m[0][0].re += r[2]; h.m[1][1].re += -r[2];            /* lambda_3 */
  h.m[0][2].re += r[3]; h.m[2][0].re += r[3];             /* lambda_4 */
  h.m[0][2].im += -r[4]; h.m[2][0].im += r[4];            /* lambda_5 */
  h.m[1][2].re += r[5]; h.m[2][1].re += r[5];             /* lambda_6 */
  h.m[1][2].im += -r[6]; h.m[2][1].im += r[6];            /* lambda_7 */
  h.m[0][0].re += r[7] * inv_sqrt3;                       /* lambda_8 */
  h.m[1][1].re += r[7] * inv_sqrt3;
  h.m[2][2].re += -2.0 * r[7] * inv_sqrt3;
  /* X = i eps H / 2 */
  mat3 x;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      x.m[i][j].re = -0.5 * eps * h.m[i][j].im;
      x.m[i][j].im = 0.5 * eps * h.m[i][j].re;
    }
  mat3 u = gen_expm(&x);
  gen_reunitarise(&u);
  return u;
}

/* Haar-random SU(3): Gram-Schmidt (QR with positive R diagonal) of a complex
 * Gaussian matrix gives Haar U(3) (Mezzadri 2007); dividing by the principal
 * cube root of the determinant is equivariant under left SU(3) multiplication,
 * so the result is Haar on SU(3). */
static mat3 gen_haar(uint64_t seed, uint64_t site) {
  double z[18];
  gen_normals(seed, site, 4u, 18, z);
  mat3 a;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      a.m[i][j].re = z[2 * (3 * i + j)] * 0.70710678118654752440;
      a.m[i][j].im = z[2 * (3 * i + j) + 1] * 0.70710678118654752440;
    }
  /* Gram-Schmidt on the columns */
  mat3 q;
  for (int c = 0; c < 3; c++) {
    zc v[3] = {a.m[0][c], a.m[1][c], a.m[2][c]};
    for (int pass = 0; pass < 2; pass++) /* second pass restores orthogonality lost to rounding */
      for (int p = 0; p < c; p++) {
        zc ip = {0.0, 0.0};
        for (int i = 0; i < 3; i++) ip = zadd(ip, zmul(zconj(q.m[i][p]), v[i]));
        for (int i = 0; i < 3; i++) {
          zc t = zmul(ip, q.m[i][p]);
          v[i].re -= t.re;
          v[i].im -= t.im;
        }
      }
    double n = 0.0;
    for (int i = 0; i < 3; i++) n += v[i].re * v[i].re + v[i].im * v[i].im;
    n = 1.0 / sqrt(n);
    for (int i = 0; i < 3; i++) q.m[i][c] = zscale(v[i], n);
  }
  /* det(q) = e^{i phi}; multiply by e^{-i phi/3} */
  zc d = {0.0, 0.0};
  for (int j = 0; j < 3; j++) {
    int a1 = (j + 1) % 3, b1 = (j + 2) % 3;
    zc minor = zadd(zmul(q.m[1][a1], q.m[2][b1]), zscale(zmul(q.m[1][b1], q.m[2][a1]), -1.0));
    d = zadd(d, zmul(q.m[0][j], minor));
  }
  double phi = atan2(d.im, d.re) / 3.0;
  zc ph = {cos(phi), -sin(phi)};
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) q.m[i][j] = zmul(q.m[i][j], ph);
  return q;
}

static int64_t gen_shift(const int32_t dims[4], int64_t site, int mu) {
  /* forward neighbour site + mu-hat with periodic wrap */
  const int64_t n1 = dims[3], n2 = dims[2], n3 = dims[1], nt = dims[0];
  int64_t x1 = site % n1, r = site / n1;
  int64_t x2 = r % n2; r /= n2;
  int64_t x3 = r % n3;
  int64_t t = r / n3;
  if (mu == 0) t = (t + 1) % nt;
  else if (mu == 1) x1 = (x1 + 1) % n1;
  else if (mu == 2) x2 = (x2 + 1) % n2;
  else x3 = (x3 + 1) % n3;
  return x1 + n1 * (x2 + n2 * (x3 + n3 * t));
}

/* Public entry: fill out[V*4*9*2] (AoS complex128) with the synthetic field,
 * on nthreads OpenMP threads (0: the default team).  Every element comes from
 * its own counter, so the result does not depend on the thread count.
 * Returns 0 on success, -1 on bad dims, -2 if scratch could not be allocated. */
int lgtgen_field_threads(const int32_t dims[4], double eps, uint64_t seed, double *out, int nthreads) {
  for (int d = 0; d < 4; d++)
    if (dims[d] < 1) return -1;
  const int64_t vol = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  mat3 *h = (mat3 *)malloc(sizeof(mat3) * (size_t)vol);
  if (!h) return -2;
  const int team = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(team)
  for (int64_t s = 0; s < vol; s++) h[s] = gen_haar(seed, (uint64_t)s);
#pragma omp parallel for schedule(static) num_threads(team)
  for (int64_t s = 0; s < vol; s++) {
    for (int mu = 0; mu < 4; mu++) {
      mat3 u = gen_link(seed, (uint64_t)s, mu, eps);
      mat3 hd = mat_dagger(&h[gen_shift(dims, s, mu)]);
      mat3 t = mat_mul(&h[s], &u);
      t = mat_mul(&t, &hd);
      double *o = out + ((size_t)s * 4 + (size_t)mu) * 18;
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
          o[2 * (3 * i + j)] = t.m[i][j].re;
          o[2 * (3 * i + j) + 1] = t.m[i][j].im;
        }
    }
  }
  free(h);
  return 0;
}

int lgtgen_field(const int32_t dims[4], double eps, uint64_t seed, double *out) {
  return lgtgen_field_threads(dims, eps, seed, out, 0);
}

/* Haar samples alone (for the generator's own distribution tests). */
int lgtgen_haar(uint64_t seed, int64_t count, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < count; s++) {
    mat3 q = gen_haar(seed, (uint64_t)s);
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        out[(size_t)s * 18 + 2 * (3 * i + j)] = q.m[i][j].re;
        out[(size_t)s * 18 + 2 * (3 * i + j) + 1] = q.m[i][j].im;
      }
  }
  return 0;
}

/* Philox4x32-10 block for the generator's known-answer test. */
void lgtgen_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { gen_philox(ctr, key, out); }
