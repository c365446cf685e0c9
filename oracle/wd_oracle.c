/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, FP64 CPU implementation of what the Wilson-Dirac hot path
 * of Clark, Babich, Barros, Brower and Rebbi, "Solving lattice QCD systems of
 * equations using mixed precision solvers on GPUs" (arXiv:0911.3191)
 * computes.  Only the test-suite, the package's smoke check and the CPU
 * baseline of the benchmark call it; the CUDA library never does, and the two
 * share no code.
 *
 * Deliberately no shortcuts of the GPU method: the spin projectors are applied
 * as full 4x4 complex matrices, the links as full 3x3 complex matrices (all 18
 * reals as given), no half spinors, no link reconstruction, no even-odd
 * storage.  Fields are full-lattice, lexicographic, DeGrand-Rossi basis:
 *   spinor [site][spin 4][colour 3] complex, gauge [site][mu 4][3][3] complex,
 *   site = x + X (y + Y (z + Z t)), parity(site) = (x+y+z+t) mod 2,
 *   U_mu(x) is the link from x to x + mu (mu = 0,1,2,3 <-> x,y,z,t).
 *
 * Sections of the paper followed:
 *   Sec. 3 eq. for M          : D and M (wo_dslash*, wo_apply_M)
 *   Sec. 3 Schur complement   : M_hat = 1 - kappa^2 D_eo D_oe (wo_apply_Mhat)
 *   App. B DeGrand-Rossi set  : the projectors P^{+mu} (wo_projector)
 *   Sec. 5.1                  : CG on the normal equations, BiCGstab
 *   Sec. 4.6 (half precision) : per-site-normalised 16-bit storage codecs
 *   App. A.2                  : the 8-number SU(3) parametrisation (wo_su3_to8/from8)
 *
 * Boundary conditions (paper silent): periodic in all directions; optionally
 * antiperiodic in t, i.e. a factor -1 on every hop that crosses t = T-1 <-> 0.
 *
 * Normalisation: M_kappa = 1 - kappa D, which is 2 kappa times the paper's
 * M = -D/2 + (4+m) with kappa = 1/(2(4+m)).
 *
 * Parity pins: every function here is pinned in tests/test_oracle_pins.py
 * against closed forms, identities or brute force; see the header of each.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cd;

typedef struct {
  int dims[4];
  int tbc_anti; /* 1: antiperiodic in t */
  const cd *U;  /* [V][4][3][3] */
} wo_lattice;

static int64_t lat_volume(const int d[4]) { return (int64_t)d[0] * d[1] * d[2] * d[3]; }

static void site_coords(const int d[4], int64_t s, int c[4]) {
  c[0] = (int)(s % d[0]); s /= d[0];
  c[1] = (int)(s % d[1]); s /= d[1];
  c[2] = (int)(s % d[2]); s /= d[2];
  c[3] = (int)s;
}

static int64_t site_index(const int d[4], const int c[4]) {
  return c[0] + (int64_t)d[0] * (c[1] + (int64_t)d[1] * (c[2] + (int64_t)d[2] * c[3]));
}

int wo_parity(const int d[4], int64_t s) {
  int c[4];
  site_coords(d, s, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* The DeGrand-Rossi projectors P^{+mu} = 1 + gamma_mu exactly as printed in
 * App. B (upper signs); P^{-mu} = 2 - P^{+mu}. */
void wo_projector(int mu, int sign, cd P[4][4]) {
  const cd J = I; /* imaginary unit */
  cd Pp[4][4][4] = {
      {{1, 0, 0, J}, {0, 1, J, 0}, {0, -J, 1, 0}, {-J, 0, 0, 1}},
      {{1, 0, 0, -1}, {0, 1, 1, 0}, {0, 1, 1, 0}, {-1, 0, 0, 1}},
      {{1, 0, J, 0}, {0, 1, 0, -J}, {-J, 0, 1, 0}, {0, J, 0, 1}},
      {{1, 0, 1, 0}, {0, 1, 0, 1}, {1, 0, 1, 0}, {0, 1, 0, 1}},
  };
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      cd delta = (a == b) ? 2.0 : 0.0;
      P[a][b] = (sign > 0) ? Pp[mu][a][b] : delta - Pp[mu][a][b];
    }
}

/* gamma_mu = P^{+mu} - 1 (App. B) */
void wo_gamma(int mu, double *out /* [4][4][2] */) {
  cd P[4][4];
  wo_projector(mu, +1, P);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      cd g = P[a][b] - ((a == b) ? 1.0 : 0.0);
      out[2 * (4 * a + b)] = creal(g);
      out[2 * (4 * a + b) + 1] = cimag(g);
    }
}

/* (D psi)(x) at one site, Sec. 3:
 *   sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
 * and, for dagger != 0, its adjoint D^dag, which has the two projectors
 * exchanged. */
static void dslash_site(const wo_lattice *L, const cd *psi, int dagger, int64_t s, cd out[4][3]) {
  const int *d = L->dims;
  int c[4];
  site_coords(d, s, c);
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) out[a][k] = 0;
  for (int mu = 0; mu < 4; ++mu) {
    cd Pfwd[4][4], Pbwd[4][4];
    wo_projector(mu, dagger ? +1 : -1, Pfwd);
    wo_projector(mu, dagger ? -1 : +1, Pbwd);

    /* forward hop: x -> x + mu */
    int cf[4] = {c[0], c[1], c[2], c[3]};
    double sf = 1.0;
    cf[mu] += 1;
    if (cf[mu] == d[mu]) {
      cf[mu] = 0;
      if (mu == 3 && L->tbc_anti) sf = -1.0;
    }
    int64_t yf = site_index(d, cf);
    const cd *Uf = L->U + (s * 4 + mu) * 9;
    const cd *pf = psi + yf * 12;
    cd w[4][3];
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        cd acc = 0;
        for (int j = 0; j < 3; ++j) acc += Uf[3 * i + j] * pf[3 * a + j];
        w[a][i] = acc;
      }
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        cd acc = 0;
        for (int b = 0; b < 4; ++b) acc += Pfwd[a][b] * w[b][i];
        out[a][i] += sf * acc;
      }

    /* backward hop: x -> x - mu, link U_mu(x - mu)^dagger */
    int cb[4] = {c[0], c[1], c[2], c[3]};
    double sb = 1.0;
    cb[mu] -= 1;
    if (cb[mu] < 0) {
      cb[mu] = d[mu] - 1;
      if (mu == 3 && L->tbc_anti) sb = -1.0;
    }
    int64_t yb = site_index(d, cb);
    const cd *Ub = L->U + (yb * 4 + mu) * 9;
    const cd *pb = psi + yb * 12;
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        cd acc = 0;
        for (int j = 0; j < 3; ++j) acc += conj(Ub[3 * j + i]) * pb[3 * a + j];
        w[a][i] = acc;
      }
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        cd acc = 0;
        for (int b = 0; b < 4; ++b) acc += Pbwd[a][b] * w[b][i];
        out[a][i] += sb * acc;
      }
  }
}

static wo_lattice make_lattice(const double *U, const int dims[4], int tbc_anti) {
  wo_lattice L;
  memcpy(L.dims, dims, sizeof(L.dims));
  L.tbc_anti = tbc_anti;
  L.U = (const cd *)U;
  return L;
}

/* out = D in (dagger: D^dag in) on the full lattice.  out_parity = 0/1 keeps
 * only output sites of that parity (the others are set to zero), which is
 * D_eo / D_oe of Sec. 3 when the input lives on the other parity; -1 keeps all. */
void wo_dslash(double *out, const double *in, const double *U, const int dims[4], int tbc_anti, int dagger,
               int out_parity) {
  wo_lattice L = make_lattice(U, dims, tbc_anti);
  int64_t V = lat_volume(dims);
  cd *o = (cd *)out;
  const cd *p = (const cd *)in;
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < V; ++s) {
    cd r[4][3];
    if (out_parity >= 0 && wo_parity(dims, s) != out_parity) {
      memset(r, 0, sizeof(r));
    } else {
      dslash_site(&L, p, dagger, s, r);
    }
    memcpy(o + 12 * s, r, sizeof(r));
  }
}

/* D in at a list of n sites only: out is [n][4][3] complex.  Used to check
 * sampled outputs of lattices too large to process whole. */
void wo_dslash_sites(double *out, const double *in, const double *U, const int dims[4], int tbc_anti, int dagger,
                     const int64_t *sites, int64_t n) {
  wo_lattice L = make_lattice(U, dims, tbc_anti);
  cd *o = (cd *)out;
  const cd *p = (const cd *)in;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    cd r[4][3];
    dslash_site(&L, p, dagger, sites[k], r);
    memcpy(o + 12 * k, r, sizeof(r));
  }
}

static void zero_parity(cd *v, const int dims[4], int parity) {
  int64_t V = lat_volume(dims);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < V; ++s)
    if (wo_parity(dims, s) == parity) memset(v + 12 * s, 0, 12 * sizeof(cd));
}

/* out = M_kappa in = in - kappa D in (full lattice). */
void wo_apply_M(double *out, const double *in, const double *U, const int dims[4], int tbc_anti, double kappa,
                int dagger) {
  int64_t V = lat_volume(dims);
  wo_dslash(out, in, U, dims, tbc_anti, dagger, -1);
  cd *o = (cd *)out;
  const cd *p = (const cd *)in;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < 12 * V; ++i) o[i] = p[i] - kappa * o[i];
}

/* Even-site Schur complement, Sec. 3: out_e = (1 - kappa^2 D_eo D_oe) in_e.
 * Full-lattice arrays; the odd sites of `in` are ignored, those of `out` are
 * zero.  dagger: M_hat^dag = 1 - kappa^2 (D^dag)_eo (D^dag)_oe. */
void wo_apply_Mhat(double *out, const double *in, const double *U, const int dims[4], int tbc_anti, double kappa,
                   int dagger) {
  int64_t V = lat_volume(dims);
  cd *in_e = (cd *)malloc(12 * V * sizeof(cd));
  cd *tmp = (cd *)malloc(12 * V * sizeof(cd));
  memcpy(in_e, in, 12 * V * sizeof(cd));
  zero_parity(in_e, dims, 1);
  wo_dslash((double *)tmp, (const double *)in_e, U, dims, tbc_anti, dagger, 1); /* D_oe in_e */
  wo_dslash(out, (const double *)tmp, U, dims, tbc_anti, dagger, 0);            /* D_eo tmp  */
  cd *o = (cd *)out;
  double k2 = kappa * kappa;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < 12 * V; ++i) o[i] = in_e[i] - k2 * o[i];
  free(in_e);
  free(tmp);
}

/* ---------------------------------------------------------------- solvers */

/* Sec. 5.1: global sums in FP64.  The index range is cut into a fixed number
 * of chunks, each summed in index order, and the chunk sums are added in chunk
 * order: the result does not depend on the number of threads or on their
 * timing (an OpenMP reduction clause combines the threads' partial sums in an
 * unspecified order, so its last bits varied from run to run). */
enum { kDotChunks = 256 };
static cd dot(const cd *a, const cd *b, int64_t n) {
  double pre[kDotChunks], pim[kDotChunks];
#pragma omp parallel for schedule(static)
  for (int c = 0; c < kDotChunks; ++c) {
    const int64_t i0 = n * c / kDotChunks, i1 = n * (c + 1) / kDotChunks;
    double re = 0.0, im = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
      cd p = conj(a[i]) * b[i];
      re += creal(p);
      im += cimag(p);
    }
    pre[c] = re;
    pim[c] = im;
  }
  double re = 0.0, im = 0.0;
  for (int c = 0; c < kDotChunks; ++c) {
    re += pre[c];
    im += pim[c];
  }
  return re + I * im;
}

static double norm2(const cd *a, int64_t n) { return creal(dot(a, a, n)); }

typedef struct {
  const double *U;
  int dims[4];
  int tbc_anti;
  double kappa;
  int schur; /* 0: full M_kappa, 1: even-site M_hat */
} wo_op;

/* out = A in or A^dag in, A = M_kappa (full) or M_hat (Schur form). */
static void apply_op(const wo_op *op, cd *out, const cd *in, int dagger) {
  if (op->schur)
    wo_apply_Mhat((double *)out, (const double *)in, op->U, op->dims, op->tbc_anti, op->kappa, dagger);
  else
    wo_apply_M((double *)out, (const double *)in, op->U, op->dims, op->tbc_anti, op->kappa, dagger);
}

/* BiCGstab (van der Vorst, 1992) for A x = b from x = 0, applied to the
 * matrix directly as in Sec. 5.1.  Stops when the iterated residual is
 * <= stop and the recomputed residual b - A x confirms it.  Returns 0
 * converged, 1 not converged within maxiter, 2 breakdown. */
static int bicgstab(const wo_op *op, cd *x, const cd *b, int64_t n, double stop, int maxiter, int *iters) {
  cd *r = calloc(n, sizeof(cd)), *rt = calloc(n, sizeof(cd)), *p = calloc(n, sizeof(cd));
  cd *v = calloc(n, sizeof(cd)), *s = calloc(n, sizeof(cd)), *t = calloc(n, sizeof(cd));
  memset(x, 0, n * sizeof(cd));
  memcpy(r, b, n * sizeof(cd));
  memcpy(rt, b, n * sizeof(cd));
  cd rho_prev = 1, alpha = 1, omega = 1;
  int status = 1, k = 0, done = 0;
  if (sqrt(norm2(b, n)) <= stop) { status = 0; done = 1; }
  for (k = 1; !done && k <= maxiter; ++k) {
    cd rho = dot(rt, r, n);
    if (cabs(rho) == 0.0) { status = 2; break; }
    cd beta = (rho / rho_prev) * (alpha / omega);
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    apply_op(op, v, p, 0);
    cd rtv = dot(rt, v, n);
    if (cabs(rtv) == 0.0) { status = 2; break; }
    alpha = rho / rtv;
    for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    apply_op(op, t, s, 0);
    double tt = norm2(t, n);
    if (tt == 0.0) { status = 2; break; }
    omega = dot(t, s, n) / tt;
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i] + omega * s[i];
      r[i] = s[i] - omega * t[i];
    }
    rho_prev = rho;
    if (sqrt(norm2(r, n)) <= stop) {
      apply_op(op, t, x, 0);
      for (int64_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
      if (sqrt(norm2(t, n)) <= stop) { status = 0; done = 1; }
    }
  }
  *iters = done ? (k - 1) : (k > maxiter ? maxiter : k);
  free(r); free(rt); free(p); free(v); free(s); free(t);
  return status;
}

/* CG on the normal equations A^dag A x = A^dag b from x = 0 (Sec. 5.1: CG is
 * applied to the normal equations because M is not Hermitian positive
 * definite).  The quantity that must end below `stop` is |b - A x|, while CG
 * sees the normal residual; so the normal residual is driven below a target
 * that starts at stop |A^dag b| / |b| and, whenever |b - A x| is recomputed
 * and still above stop, is scaled by stop / |b - A x| (one CG, no restart).
 * Uses <p, A^dag A p> = |A p|^2. */
static int cgnr(const wo_op *op, cd *x, const cd *b, int64_t n, double stop, int maxiter, int *iters) {
  cd *r = calloc(n, sizeof(cd)), *p = calloc(n, sizeof(cd)), *w = calloc(n, sizeof(cd));
  cd *q = calloc(n, sizeof(cd));
  memset(x, 0, n * sizeof(cd));
  apply_op(op, r, b, 1);
  memcpy(p, r, n * sizeof(cd));
  double rr = norm2(r, n);
  double bn = sqrt(norm2(b, n));
  double target = (bn > 0.0) ? stop * sqrt(rr) / bn : 0.0;
  int status = 1, k = 0, done = 0;
  if (bn <= stop) { status = 0; done = 1; }
  for (k = 1; !done && k <= maxiter; ++k) {
    apply_op(op, w, p, 0);
    double pq = norm2(w, n);
    if (pq == 0.0) { status = 2; break; }
    apply_op(op, q, w, 1);
    double alpha = rr / pq;
    for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
    double rr_new = norm2(r, n);
    if (sqrt(rr_new) <= target) {
      apply_op(op, w, x, 0);
      for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
      double rn = sqrt(norm2(w, n));
      if (rn <= stop) { status = 0; done = 1; break; }
      target *= stop / rn;
    }
    double beta = rr_new / rr;
    rr = rr_new;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
  }
  *iters = done ? k : (k > maxiter ? maxiter : k);
  free(r); free(p); free(w); free(q);
  return status;
}

/* Solve M_kappa x = b (full lattice, FP64); solver 0 = BiCGstab, 1 = CG on
 * the normal equations.
 *   schur = 0 : on the full matrix.
 *   schur = 1 : the even-odd form of Sec. 3: b_hat = b_e + kappa D_eo b_o,
 *               solve M_hat x_e = b_hat, then x_o = b_o + kappa D_oe x_e.
 * Stop: |b - M x| <= tol |b|.  In the Schur form this is the same condition
 * on |b_hat - M_hat x_e|, since the odd rows of b - M x vanish identically
 * once x_o is reconstructed.
 * Returns the status; out_info = {iterations, true relative residual}. */
int wo_solve(double *x_out, const double *b_in, const double *U, const int dims[4], int tbc_anti, double kappa,
             double tol, int maxiter, int solver, int schur, double *out_info) {
  int64_t V = lat_volume(dims);
  int64_t n = 12 * V;
  const cd *b = (const cd *)b_in;
  cd *x = (cd *)x_out;
  double stop = tol * sqrt(norm2(b, n));
  wo_op op = {U, {dims[0], dims[1], dims[2], dims[3]}, tbc_anti, kappa, schur};
  cd *rhs = calloc(n, sizeof(cd)), *tmp = calloc(n, sizeof(cd)), *xs = calloc(n, sizeof(cd));
  int status, iters = 0;
  if (schur) {
    /* b_hat = b_e + kappa D_eo b_o */
    memcpy(tmp, b, n * sizeof(cd));
    zero_parity(tmp, dims, 0);
    wo_dslash((double *)rhs, (const double *)tmp, U, dims, tbc_anti, 0, 0);
    for (int64_t s = 0; s < V; ++s)
      for (int i = 0; i < 12; ++i)
        rhs[12 * s + i] = (wo_parity(dims, s) == 0) ? b[12 * s + i] + kappa * rhs[12 * s + i] : 0.0;
  } else {
    memcpy(rhs, b, n * sizeof(cd));
  }
  if (solver == 0)
    status = bicgstab(&op, xs, rhs, n, stop, maxiter, &iters);
  else
    status = cgnr(&op, xs, rhs, n, stop, maxiter, &iters);
  if (schur) {
    /* x_o = b_o + kappa D_oe x_e */
    wo_dslash((double *)tmp, (const double *)xs, U, dims, tbc_anti, 0, 1);
    for (int64_t s = 0; s < V; ++s)
      for (int i = 0; i < 12; ++i)
        x[12 * s + i] = (wo_parity(dims, s) == 0) ? xs[12 * s + i] : b[12 * s + i] + kappa * tmp[12 * s + i];
  } else {
    memcpy(x, xs, n * sizeof(cd));
  }
  /* true residual |b - M x| / |b| */
  wo_apply_M((double *)tmp, (const double *)x, U, dims, tbc_anti, kappa, 0);
  for (int64_t i = 0; i < n; ++i) tmp[i] = b[i] - tmp[i];
  double rel = sqrt(norm2(tmp, n)) / sqrt(norm2(b, n));
  if (status == 0 && rel > tol) status = 1;
  out_info[0] = (double)iters;
  out_info[1] = rel;
  free(rhs); free(tmp); free(xs);
  return status;
}

/* A fixed number of BiCGstab iterations on the Schur system (for timing a
 * bounded sample of a solve).  Returns the iterated residual norm. */
double wo_bicgstab_schur_iters(const double *b_in, const double *U, const int dims[4], int tbc_anti, double kappa,
                               int iterations) {
  int64_t V = lat_volume(dims);
  int64_t n = 12 * V;
  cd *rhs = calloc(n, sizeof(cd)), *x = calloc(n, sizeof(cd));
  memcpy(rhs, b_in, n * sizeof(cd));
  zero_parity(rhs, dims, 1);
  wo_op op = {U, {dims[0], dims[1], dims[2], dims[3]}, tbc_anti, kappa, 1};
  int it = 0;
  bicgstab(&op, x, rhs, n, 0.0, iterations, &it);
  /* the residual of the truncated run */
  cd *t = calloc(n, sizeof(cd));
  apply_op(&op, t, x, 0);
  for (int64_t i = 0; i < n; ++i) t[i] = rhs[i] - t[i];
  double res = sqrt(norm2(t, n));
  free(rhs); free(x); free(t);
  return res;
}

/* ------------------------------------------------------------------ codecs
 * Sec. 4.6: a colour-spinor is stored as 24 16-bit numbers plus one FP32
 * number standing for its largest element.  The encode is defined in FP32
 * arithmetic (the arithmetic of the kernels that produce these fields):
 *   f_k  = (float) v_k                       (round to nearest even)
 *   norm = max_k |f_k|
 *   Q16  : q_k = rint(f_k * (32767 / norm))  (float ops, round half even)
 *          decode  f_k = (float) q_k * (norm * (float)(1/32767))
 *   H16N : h_k = fp16(f_k * (1 / norm))      decode f_k = (float) h_k * norm
 *   B16N : h_k = bf16(f_k * (1 / norm))      decode f_k = (float) h_k * norm
 *   norm = 0 gives all-zero codes.
 * Links (|u| <= 1): Q16 q = rint((float)u * 32767), decode q * (float)(1/32767);
 * H16N / B16N: fp16 / bf16 of (float)u.
 * fp16 and bf16 rounding is written from the IEEE 754 binary16 and the
 * bfloat16 definitions (10 or 7 fraction bits, minimum normal exponent -14 or
 * -126, gradual underflow, round to nearest even) on the exact double value. */

static float round_to_format(float w, int frac_bits, int emin) {
  if (w == 0.0f || !isfinite(w)) return w;
  int e;
  frexp((double)w, &e);
  int lead = e - 1;
  if (lead < emin) lead = emin;
  double quantum = ldexp(1.0, lead - frac_bits);
  return (float)(rint((double)w / quantum) * quantum);
}

float wo_round_fp16(float w) { return round_to_format(w, 10, -14); }
float wo_round_bf16(float w) { return round_to_format(w, 7, -126); }

static float site_norm(const double *v, float *f) {
  float m = 0.0f;
  for (int k = 0; k < 24; ++k) {
    f[k] = (float)v[k];
    float a = fabsf(f[k]);
    if (a > m) m = a;
  }
  return m;
}

/* fmt: 0 = Q16 (codes as int16 in `codes`), 1 = H16N, 2 = B16N (rounded
 * values as float in `vals`).  v: [n][24] doubles. */
void wo_encode_spinor(const double *v, int64_t n, int fmt, int16_t *codes, float *vals, float *norms) {
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; ++s) {
    float f[24];
    float norm = site_norm(v + 24 * s, f);
    norms[s] = norm;
    if (fmt == 0) {
      float scale = (norm > 0.0f) ? 32767.0f / norm : 0.0f;
      for (int k = 0; k < 24; ++k) {
        float q = rintf(f[k] * scale);
        if (q > 32767.0f) q = 32767.0f;
        if (q < -32767.0f) q = -32767.0f;
        codes[24 * s + k] = (int16_t)q;
      }
    } else {
      float inv = (norm > 0.0f) ? 1.0f / norm : 0.0f;
      for (int k = 0; k < 24; ++k) {
        float w = f[k] * inv;
        vals[24 * s + k] = (fmt == 1) ? wo_round_fp16(w) : wo_round_bf16(w);
      }
    }
  }
}

/* Decode to the float values the kernels compute with (returned as doubles). */
void wo_decode_spinor(const int16_t *codes, const float *vals, const float *norms, int64_t n, int fmt, double *out) {
  const float c = (float)(1.0 / 32767.0);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; ++s) {
    float norm = norms[s];
    if (fmt == 0) {
      float d = norm * c;
      for (int k = 0; k < 24; ++k) out[24 * s + k] = (double)((float)codes[24 * s + k] * d);
    } else {
      for (int k = 0; k < 24; ++k) out[24 * s + k] = (double)(vals[24 * s + k] * norm);
    }
  }
}

/* Links: u [n] doubles (real and imaginary parts), fmt as above.  Returns the
 * decoded float value of each stored element. */
void wo_encode_link_values(const double *u, int64_t n, int fmt, int16_t *codes, double *decoded) {
  const float c = (float)(1.0 / 32767.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    float f = (float)u[i];
    if (fmt == 0) {
      float q = rintf(f * 32767.0f);
      codes[i] = (int16_t)q;
      decoded[i] = (double)((float)(int16_t)q * c);
    } else {
      float r = (fmt == 1) ? wo_round_fp16(f) : wo_round_bf16(f);
      codes[i] = 0;
      decoded[i] = (double)r;
    }
  }
}

/* ---- App. A.2: 8-number parametrisation of an SU(3) link -----------------
 * Rows a, b, c of U.  Stored: p = {arg a1, arg c1, Re a2, Im a2, Re a3,
 * Im a3, Re b1, Im b1}.  Reconstruction, in the appendix's order:
 *   1. |a1| from the unit norm of row a, a1 = |a1| e^{i arg a1};
 *   2. |c1| from the unit norm of column 1, c1 = |c1| e^{i arg c1};
 *   3. with N = sqrt(|a2|^2 + |a3|^2), the unit vectors b' = (0, -a3^*, a2^*)/N
 *      and c' = (a x b')^* = (N, -a1^* a2/N, -a1^* a3/N) span the plane
 *      orthogonal to a (the appendix's matrix prints b' with a different
 *      sign and conjugation on its last entry; this b' is the one orthogonal
 *      to a: a . conj(b') = (-a2 a3 + a3 a2)/N = 0);
 *   4. rows b and c are the SU(2) rotation of (b', c'): with p2 = b1/N and
 *      p1 = conj(c1)/N, b = p1 b' + p2 c', c = -p2^* b' + p1^* c'.
 * Singular at N = 0 (|a1| = 1): to8 returns 1 there. */
int wo_su3_to8(const double *u, double *p) {
  const cd *U = (const cd *)u;
  p[0] = carg(U[0]);
  p[1] = carg(U[6]);
  p[2] = creal(U[1]); p[3] = cimag(U[1]);
  p[4] = creal(U[2]); p[5] = cimag(U[2]);
  p[6] = creal(U[3]); p[7] = cimag(U[3]);
  const double n2 = creal(U[1] * conj(U[1])) + creal(U[2] * conj(U[2]));
  return n2 > 0.0 ? 0 : 1;
}

void wo_su3_from8(const double *p, double *u) {
  cd *U = (cd *)u;
  const cd a2 = p[2] + I * p[3], a3 = p[4] + I * p[5], b1 = p[6] + I * p[7];
  const double n2 = creal(a2 * conj(a2)) + creal(a3 * conj(a3));
  const cd a1 = sqrt(fmax(0.0, 1.0 - n2)) * cexp(I * p[0]);
  const double b12 = creal(b1 * conj(b1));
  const cd c1 = sqrt(fmax(0.0, 1.0 - creal(a1 * conj(a1)) - b12)) * cexp(I * p[1]);
  const double N = sqrt(n2);
  const cd bp[3] = {0.0, -conj(a3) / N, conj(a2) / N};
  const cd cp[3] = {N, -conj(a1) * a2 / N, -conj(a1) * a3 / N};
  const cd p2 = b1 / N, p1 = conj(c1) / N;
  U[0] = a1; U[1] = a2; U[2] = a3;
  for (int j = 0; j < 3; ++j) {
    U[3 + j] = p1 * bp[j] + p2 * cp[j];
    U[6 + j] = -conj(p2) * bp[j] + conj(p1) * cp[j];
  }
}
