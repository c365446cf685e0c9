/*
 * Seeded synthetic inputs for the Wilson-Dirac operator: SU(3) gauge links,
 * Gaussian and uniform colour-spinor fields.
 *
 * This module holds no arithmetic of the method (no Dirac operator, no
 * projector, no solver, no storage codec).  It only draws random numbers and
 * turns them into link matrices and source vectors, which both the CPU oracle
 * and the CUDA path then consume as plain FP64 host arrays.
 *
 * Random numbers: Philox4x32-10, the counter-based generator of Salmon,
 * Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC'11), written here from its published definition: a 4x32-bit counter and
 * a 2x32-bit key, ten rounds of two 32x32->64-bit multiplications with the
 * round constants 0xD2511F53 / 0xCD9E8D57, and the key bumped by the Weyl
 * constants 0x9E3779B9 / 0xBB67AE85 between rounds.  Every output element is
 * keyed by (seed, element index, draw, stream tag), so any region of any
 * lattice is reproducible independently of thread count.
 *
 * Layouts (all FP64, complex numbers as [re, im]):
 *   link field  : [n][3][3][2]            row-major 3x3 complex matrix
 *   gauge field : [site][mu][3][3][2]     site lexicographic x+X(y+Y(z+Zt)),
 *                                         U_mu(x) the link from x to x+mu
 *   spinor field: [site][spin 4][colour 3][2]
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define LI_PHILOX_M0 0xD2511F53u
#define LI_PHILOX_M1 0xCD9E8D57u
#define LI_PHILOX_W0 0x9E3779B9u
#define LI_PHILOX_W1 0xBB67AE85u

static inline uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t *hi) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  return (uint32_t)p;
}

/* One Philox4x32-10 block: out = philox(ctr, key). */
void li_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += LI_PHILOX_W0;
      k1 += LI_PHILOX_W1;
    }
    uint32_t hi0, hi1;
    uint32_t lo0 = mulhilo32(LI_PHILOX_M0, c0, &hi0);
    uint32_t lo1 = mulhilo32(LI_PHILOX_M1, c2, &hi1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Two uniforms in (0, 1) with 53 random bits each, from one Philox block. */
static void uniform_pair(uint64_t seed, uint64_t index, uint32_t draw, uint32_t tag, double u[2]) {
  uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), draw, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  li_philox4x32_10(ctr, key, r);
  for (int k = 0; k < 2; ++k) {
    uint64_t bits = ((uint64_t)r[2 * k] << 32) | (uint64_t)r[2 * k + 1];
    u[k] = ((double)(bits >> 11) + 0.5) * (1.0 / 9007199254740992.0); /* 2^-53 */
  }
}

/* Two independent N(0,1) deviates (Box-Muller). */
static void gaussian_pair(uint64_t seed, uint64_t index, uint32_t draw, uint32_t tag, double g[2]) {
  double u[2];
  uniform_pair(seed, index, draw, tag, u);
  double rad = sqrt(-2.0 * log(u[0]));
  double ang = 6.283185307179586476925286766559 * u[1];
  g[0] = rad * cos(ang);
  g[1] = rad * sin(ang);
}

/* ---- small complex 3x3 helpers (input generation only) ---- */
typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx cconj(cplx a) { cplx r = {a.re, -a.im}; return r; }

static void mat_mul(const cplx a[9], const cplx b[9], cplx out[9]) {
  cplx t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx s = {0.0, 0.0};
      for (int k = 0; k < 3; ++k) s = cadd(s, cmul(a[3 * i + k], b[3 * k + j]));
      t[3 * i + j] = s;
    }
  memcpy(out, t, sizeof(t));
}

/* exp(A) for a small complex 3x3 A: scaling and squaring around a Taylor sum. */
static void mat_exp(const cplx a_in[9], cplx out[9]) {
  double fro = 0.0;
  for (int i = 0; i < 9; ++i) fro += a_in[i].re * a_in[i].re + a_in[i].im * a_in[i].im;
  fro = sqrt(fro);
  int s = 0;
  while (fro > 0.25) { fro *= 0.5; ++s; }
  double scale = ldexp(1.0, -s);
  cplx a[9], term[9], sum[9];
  for (int i = 0; i < 9; ++i) { a[i].re = a_in[i].re * scale; a[i].im = a_in[i].im * scale; }
  for (int i = 0; i < 9; ++i) { sum[i].re = (i % 4 == 0) ? 1.0 : 0.0; sum[i].im = 0.0; term[i] = sum[i]; }
  for (int k = 1; k <= 18; ++k) {
    mat_mul(term, a, term);
    for (int i = 0; i < 9; ++i) { term[i].re /= k; term[i].im /= k; sum[i] = cadd(sum[i], term[i]); }
  }
  for (int q = 0; q < s; ++q) mat_mul(sum, sum, sum);
  memcpy(out, sum, sizeof(sum));
}

/* Make rows a, b orthonormal (Gram-Schmidt) and set c = (a x b)^*, so that the
 * matrix is exactly special unitary up to FP64 rounding. */
static void reunitarise(cplx m[9]) {
  cplx *a = m, *b = m + 3, *c = m + 6;
  double na = 0.0;
  for (int i = 0; i < 3; ++i) na += a[i].re * a[i].re + a[i].im * a[i].im;
  na = 1.0 / sqrt(na);
  for (int i = 0; i < 3; ++i) { a[i].re *= na; a[i].im *= na; }
  cplx ab = {0.0, 0.0};
  for (int i = 0; i < 3; ++i) ab = cadd(ab, cmul(cconj(a[i]), b[i]));
  for (int i = 0; i < 3; ++i) { cplx p = cmul(ab, a[i]); b[i].re -= p.re; b[i].im -= p.im; }
  double nb = 0.0;
  for (int i = 0; i < 3; ++i) nb += b[i].re * b[i].re + b[i].im * b[i].im;
  nb = 1.0 / sqrt(nb);
  for (int i = 0; i < 3; ++i) { b[i].re *= nb; b[i].im *= nb; }
  for (int i = 0; i < 3; ++i) {
    int j = (i + 1) % 3, k = (i + 2) % 3;
    cplx x = cmul(a[j], b[k]);
    cplx y = cmul(a[k], b[j]);
    cplx d = {x.re - y.re, x.im - y.im};
    c[i] = cconj(d);
  }
}

/* One SU(3) matrix U = exp(i eps H), H = sum_a w_a lambda_a / 2 with
 * w_a ~ N(0,1) and lambda_a the Gell-Mann matrices, then re-unitarised. */
static void su3_element(uint64_t seed, uint64_t index, uint32_t tag, double eps, double *out) {
  double w[8];
  for (int d = 0; d < 4; ++d) gaussian_pair(seed, index, (uint32_t)d, tag, w + 2 * d);
  const double inv_sqrt3 = 0.57735026918962576451;
  /* H (Hermitian, traceless) written entry by entry from the Gell-Mann basis */
  cplx h[9];
  h[0].re = 0.5 * (w[2] + w[7] * inv_sqrt3); h[0].im = 0.0;
  h[4].re = 0.5 * (-w[2] + w[7] * inv_sqrt3); h[4].im = 0.0;
  h[8].re = -w[7] * inv_sqrt3; h[8].im = 0.0;
  h[1].re = 0.5 * w[0]; h[1].im = -0.5 * w[1];
  h[2].re = 0.5 * w[3]; h[2].im = -0.5 * w[4];
  h[5].re = 0.5 * w[5]; h[5].im = -0.5 * w[6];
  h[3] = cconj(h[1]);
  h[6] = cconj(h[2]);
  h[7] = cconj(h[5]);
  cplx a[9];
  for (int i = 0; i < 9; ++i) { a[i].re = -eps * h[i].im; a[i].im = eps * h[i].re; } /* i*eps*H */
  cplx u[9];
  mat_exp(a, u);
  reunitarise(u);
  for (int i = 0; i < 9; ++i) { out[2 * i] = u[i].re; out[2 * i + 1] = u[i].im; }
}

/* n SU(3) matrices, element i keyed by (seed, i, tag). */
void li_su3_field(double *out, int64_t n, double eps, uint64_t seed, uint32_t tag) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) su3_element(seed, (uint64_t)i, tag, eps, out + 18 * i);
}

/* n N(0,1) reals (n even), pair i keyed by (seed, i, tag). */
void li_gaussian(double *out, int64_t n, uint64_t seed, uint32_t tag) {
  int64_t npair = n / 2;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < npair; ++i) gaussian_pair(seed, (uint64_t)i, 0u, tag, out + 2 * i);
}

/* n uniforms in (0, 1) (n even), pair i keyed by (seed, i, tag). */
void li_uniform(double *out, int64_t n, uint64_t seed, uint32_t tag) {
  int64_t npair = n / 2;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < npair; ++i) uniform_pair(seed, (uint64_t)i, 0u, tag, out + 2 * i);
}
