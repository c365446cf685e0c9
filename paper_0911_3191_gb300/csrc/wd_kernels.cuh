// Kernel templates and per-precision launchers.
//
// Each storage precision P (FP64, FP32, Q16, H16N, B16N) instantiates this
// header once in its own translation unit (wd_prec_*.cu) and exports a
// PrecOps table.  Kernels:
//   dslash_kernel : one dslash (Sec. 3-4) with a fused epilogue (xpay, the
//                   solver vector updates) and fused FP64 reductions (Sec. 5.1)
//   site_kernel   : BLAS-1, conversions, reorders, with fused FP64 reductions
// The Krylov scalars stay on the device (SolverCtl), computed by the
// finalisers of the reductions, so a solver iteration is a fixed sequence of
// launches that a CUDA graph can replay without host round trips.
#pragma once

#include "wd_internal.h"
#include "wd_slab.cuh"
#include "wd_async.cuh"

namespace wd {

constexpr int kDslashBlock = 128;
constexpr int kBlasBlock = 256;

// scalar coefficient: a value, or read from device memory when p != nullptr
struct Coef {
  double c;
  const double* p;
  long rs = 0;  // doubles from one right-hand side's value to the next
  __device__ __forceinline__ double get() const { return p ? *p : c; }
  __device__ __forceinline__ Coef at(int r) const { return Coef{c, p ? p + (long)r * rs : nullptr, rs}; }
};

// ---------------------------------------------------------- finalisers
__device__ __forceinline__ void ctl_fail(SolverCtl* ctl, int status) {
  if (ctl->status == WD_OK) ctl->status = status;
  ctl->done = 1;
}
__device__ __forceinline__ void ctl_set_update(SolverCtl* ctl, int v) {
  ctl->do_update = v;
  if (ctl->in_graph) cudaGraphSetConditional((cudaGraphConditionalHandle)ctl->h_update, (unsigned)v);
}

struct FinStore {
  double* out;
  int n;
  __device__ __forceinline__ FinStore at(int r) const { return FinStore{out + (long)r * n, n}; }
  __device__ void operator()(const double* t) const {
    for (int k = 0; k < n; ++k) out[k] = t[k];
  }
};

// BiCGstab: alpha = rho / <r_tilde, v>
struct FinBicgAlpha {
  SolverCtl* ctl;
  __device__ __forceinline__ FinBicgAlpha at(int r) const { return FinBicgAlpha{ctl + r}; }
  __device__ void operator()(const double* t) const {
    double2 rtv = make_double2(t[0], t[1]);
    if (!cfinite(rtv)) { ctl_fail(ctl, WD_ERR_NUMERIC); return; }
    if (rtv.x == 0.0 && rtv.y == 0.0) { ctl_fail(ctl, WD_ERR_BREAKDOWN); return; }
    ctl->alpha = cdiv(ctl->rho, rtv);
  }
};

// BiCGstab: omega = <t, s> / <t, t>
struct FinBicgOmega {
  SolverCtl* ctl;
  __device__ __forceinline__ FinBicgOmega at(int r) const { return FinBicgOmega{ctl + r}; }
  __device__ void operator()(const double* t) const {
    double2 ts = make_double2(t[0], t[1]);
    double tt = t[2];
    if (!cfinite(ts) || !isfinite(tt)) { ctl_fail(ctl, WD_ERR_NUMERIC); return; }
    if (tt == 0.0 || (ts.x == 0.0 && ts.y == 0.0)) { ctl_fail(ctl, WD_ERR_BREAKDOWN); return; }
    ctl->omega = make_double2(ts.x / tt, ts.y / tt);
  }
};

// Reliable-update trigger of Alg. 2: |r_hat_{k+1}| < delta M(r_hat), plus a
// forced update on apparent convergence (the FP64 true residual then decides)
// and at max_iter (so x holds everything computed).
__device__ __forceinline__ void decide_update(SolverCtl* ctl, double rr, double conv2) {
  const double r = sqrt(rr);
  const bool conv = rr <= conv2;
  const bool maxed = ctl->iter >= ctl->max_iter;
  const bool rel = r < ctl->delta * ctl->maxr;
  const int upd = (conv || maxed || rel) ? 1 : 0;
  ctl->forced = (conv || maxed) ? 1 : 0;
  // Alg. 2 compares with the largest residual since the last update; defect
  // correction (Alg. 1) solves to eps_in relative to the restart residual
  if (!upd && !ctl->restart) ctl->maxr = fmax(ctl->maxr, r);
  ctl_set_update(ctl, upd);
}

// BiCGstab end of iteration: |r|^2 and rho_new = <r_tilde, r>
struct FinBicgIter {
  SolverCtl* ctl;
  __device__ __forceinline__ FinBicgIter at(int r) const { return FinBicgIter{ctl + r}; }
  __device__ void operator()(const double* t) const {
    if (ctl->done) { ctl_set_update(ctl, 0); return; }
    const double rr = t[0];
    const double2 rho_new = make_double2(t[1], t[2]);
    ctl->iter += 1;
    if (!isfinite(rr) || !cfinite(rho_new)) { ctl_fail(ctl, WD_ERR_NUMERIC); ctl_set_update(ctl, 0); return; }
    ctl->rr = rr;
    ctl->rho_prev = ctl->rho;
    ctl->rho = rho_new;
    ctl->beta = cmul(cdiv(rho_new, ctl->rho_prev), cdiv(ctl->alpha, ctl->omega));
    decide_update(ctl, (rho_new.x == 0.0 && rho_new.y == 0.0) ? 0.0 : rr, ctl->stop2);
  }
};

// BiCGstab reliable update (Alg. 2): t = {|r|^2 FP64, <r_tilde, r_hat>, |r_hat|^2}
struct FinRelupBicg {
  SolverCtl* ctl;
  __device__ __forceinline__ FinRelupBicg at(int r) const { return FinRelupBicg{ctl + r}; }
  __device__ void operator()(const double* t) const {
    ctl->updates += 1;
    const double r2 = t[0];
    const double2 rho = make_double2(t[1], t[2]);
    if (!isfinite(r2) || !cfinite(rho)) { ctl_fail(ctl, WD_ERR_NUMERIC); return; }
    ctl->r2_true = r2;
    ctl->rr = t[3];
    ctl->maxr = sqrt(t[3]);
    if (ctl->restart) {
      // Alg. 1: a new inner solve from the new residual (r_tilde = r_hat,
      // p = v = 0, set by OpRestart in the same update)
      ctl->rho = make_double2(t[3], 0.0);
      ctl->rho_prev = ctl->alpha = ctl->omega = make_double2(1.0, 0.0);
      ctl->beta = make_double2(0.0, 0.0);
    } else {
      ctl->rho = rho;
      ctl->beta = cmul(cdiv(rho, ctl->rho_prev), cdiv(ctl->alpha, ctl->omega));
    }
    if (r2 <= ctl->stop2) { ctl->status = WD_OK; ctl->done = 1; }
    else if (ctl->iter >= ctl->max_iter) ctl_fail(ctl, WD_ERR_NOT_CONVERGED);
    else if (rho.x == 0.0 && rho.y == 0.0) ctl_fail(ctl, WD_ERR_BREAKDOWN);
  }
};

// BiCGstab setup: r_hat = r_tilde = quantised b_hat; t = {<r_t, r_hat>, |r_hat|^2}
struct FinBicgSetup {
  SolverCtl* ctl;
  __device__ __forceinline__ FinBicgSetup at(int r) const { return FinBicgSetup{ctl + r}; }
  __device__ void operator()(const double* t) const {
    ctl->rho = make_double2(t[0], t[1]);
    ctl->rr = t[2];
    ctl->maxr = sqrt(t[2]);
  }
};

// CG: alpha = |r|^2 / <p, A p>, with <p, M^dag M p> = |M p|^2
struct FinCgAlpha {
  SolverCtl* ctl;
  __device__ __forceinline__ FinCgAlpha at(int r) const { return FinCgAlpha{ctl + r}; }
  __device__ void operator()(const double* t) const {
    const double pap = t[0];
    if (!isfinite(pap)) { ctl_fail(ctl, WD_ERR_NUMERIC); return; }
    if (pap <= 0.0) { ctl_fail(ctl, WD_ERR_BREAKDOWN); return; }
    ctl->cg_alpha = ctl->rr / pap;
  }
};

struct FinCgIter {
  SolverCtl* ctl;
  __device__ __forceinline__ FinCgIter at(int r) const { return FinCgIter{ctl + r}; }
  __device__ void operator()(const double* t) const {
    if (ctl->done) { ctl_set_update(ctl, 0); return; }
    const double rr = t[0];
    ctl->iter += 1;
    if (!isfinite(rr)) { ctl_fail(ctl, WD_ERR_NUMERIC); ctl_set_update(ctl, 0); return; }
    ctl->rr_prev = ctl->rr;
    ctl->rr = rr;
    ctl->beta = make_double2(rr / ctl->rr_prev, 0.0);
    decide_update(ctl, rr, ctl->target2);
  }
};

// CG reliable update, first half: the FP64 Schur residual r = b_hat - M_hat x
struct FinRelupCgR {
  SolverCtl* ctl;
  __device__ __forceinline__ FinRelupCgR at(int r) const { return FinRelupCgR{ctl + r}; }
  __device__ void operator()(const double* t) const {
    ctl->updates += 1;
    const double r2 = t[0];
    if (!isfinite(r2)) { ctl_fail(ctl, WD_ERR_NUMERIC); return; }
    ctl->r2_true = r2;
    if (r2 <= ctl->stop2) { ctl->status = WD_OK; ctl->done = 1; return; }
    if (ctl->iter >= ctl->max_iter) { ctl_fail(ctl, WD_ERR_NOT_CONVERGED); return; }
    // apparent convergence of the normal residual without the Schur residual
    // being small enough: tighten the target by the missing factor
    if (ctl->forced && ctl->rr <= ctl->target2) ctl->target2 *= ctl->stop2 / r2;
  }
};

// CG reliable update, second half: r_hat = M_hat^dag r; the next direction
// uses beta = |r_hat_true|^2 / |r_hat_old|^2 (true residual in the numerator)
struct FinRelupCgN {
  SolverCtl* ctl;
  __device__ __forceinline__ FinRelupCgN at(int r) const { return FinRelupCgN{ctl + r}; }
  __device__ void operator()(const double* t) const {
    const double rr = t[0];
    if (!isfinite(rr)) { ctl_fail(ctl, WD_ERR_NUMERIC); return; }
    ctl->rr = rr;
    ctl->maxr = sqrt(rr);
    // defect correction restarts CG from the new residual: p = r_hat
    ctl->beta = ctl->restart ? make_double2(0.0, 0.0) : make_double2(rr / ctl->rr_prev, 0.0);
  }
};

// CG setup: r_hat = M_hat^dag b_hat; t = {|r_hat|^2}
struct FinCgSetup {
  SolverCtl* ctl;
  const double* bhat2;
  __device__ __forceinline__ FinCgSetup at(int r) const { return FinCgSetup{ctl + r, bhat2 + r}; }
  __device__ void operator()(const double* t) const {
    ctl->rr = t[0];
    ctl->rr_prev = t[0];
    ctl->maxr = sqrt(t[0]);
    ctl->beta = make_double2(0.0, 0.0);
    // normal-residual target tol |b| |M^dag b_hat| / |b_hat|
    ctl->target2 = (*bhat2 > 0.0) ? ctl->stop2 * t[0] / *bhat2 : 0.0;
  }
};

// ------------------------------------------------------------ epilogues
// Called once per output site with acc = (D in)(h).

template <class Out>
struct EpiStore {
  static constexpr int NRED = 0;
  Out out;
  __device__ __forceinline__ EpiStore at(int r) const { return EpiStore{out.at(r)}; }
  template <typename R>
  __device__ __forceinline__ void operator()(int h, R (&a)[24], double*) const { out.store(h, a); }
};

// out = x + c acc
template <class Out, class X>
struct EpiXpay {
  static constexpr int NRED = 0;
  Out out;
  X x;
  Coef c;
  __device__ __forceinline__ EpiXpay at(int r) const { return EpiXpay{out.at(r), x.at(r), c.at(r)}; }
  template <typename R>
  __device__ __forceinline__ void operator()(int h, R (&a)[24], double*) const {
    R xv[24];
    x.load(h, xv);
    const R cc = (R)c.get();
#pragma unroll
    for (int k = 0; k < 24; ++k) a[k] = xv[k] + cc * a[k];
    out.store(h, a);
  }
};

// v = x + c acc; reduce <w, v> (v as stored)
template <class Out, class X, class W, class Fin>
struct EpiXpayDot {
  static constexpr int NRED = 2;
  Out out;
  X x;
  W w;
  Coef c;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ EpiXpayDot at(int r) const {
    return EpiXpayDot{out.at(r), x.at(r), w.at(r), c.at(r), rs, fin.at(r)};
  }
  template <typename R>
  __device__ __forceinline__ void operator()(int h, R (&a)[24], double* red) const {
    R xv[24], wv[24];
    x.load(h, xv);
    const R cc = (R)c.get();
#pragma unroll
    for (int k = 0; k < 24; ++k) a[k] = xv[k] + cc * a[k];
    out.store_get(h, a);
    w.load(h, wv);
    R re = 0, im = 0;  // this site's 12 terms in the kernel's precision
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re += wv[2 * k] * a[2 * k];
      re += wv[2 * k + 1] * a[2 * k + 1];
      im += wv[2 * k] * a[2 * k + 1];
      im -= wv[2 * k + 1] * a[2 * k];
    }
    red[0] += (double)re;  // global sum in FP64
    red[1] += (double)im;
  }
};

// t = s + c acc with s = x; reduce <t, s> and <t, t>
template <class Out, class X, class Fin>
struct EpiXpayTS {
  static constexpr int NRED = 3;
  Out out;
  X x;
  Coef c;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ EpiXpayTS at(int r) const { return EpiXpayTS{out.at(r), x.at(r), c.at(r), rs, fin.at(r)}; }
  template <typename R>
  __device__ __forceinline__ void operator()(int h, R (&a)[24], double* red) const {
    R sv[24];
    x.load(h, sv);
    const R cc = (R)c.get();
#pragma unroll
    for (int k = 0; k < 24; ++k) a[k] = sv[k] + cc * a[k];
    out.store_get(h, a);
    R re = 0, im = 0, tt = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R tr = a[2 * k], ti = a[2 * k + 1], sr = sv[2 * k], si = sv[2 * k + 1];
      re += tr * sr;
      re += ti * si;
      im += tr * si;
      im -= ti * sr;
      tt += tr * tr;
      tt += ti * ti;
    }
    red[0] += (double)re;
    red[1] += (double)im;
    red[2] += (double)tt;
  }
};

// v = x + c acc; reduce |v|^2 (v as stored)
template <class Out, class X, class Fin>
struct EpiXpayNorm {
  static constexpr int NRED = 1;
  Out out;
  X x;
  Coef c;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ EpiXpayNorm at(int r) const {
    return EpiXpayNorm{out.at(r), x.at(r), c.at(r), rs, fin.at(r)};
  }
  template <typename R>
  __device__ __forceinline__ void operator()(int h, R (&a)[24], double* red) const {
    R xv[24];
    x.load(h, xv);
    const R cc = (R)c.get();
#pragma unroll
    for (int k = 0; k < 24; ++k) a[k] = xv[k] + cc * a[k];
    out.store_get(h, a);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) n += a[k] * a[k];
    red[0] += (double)n;
  }
};

// CG: q = w + c acc (= M_hat^dag M_hat p); x_hat += alpha p; r_hat -= alpha q;
// reduce |r_hat|^2.  q is never stored.
template <class S, class Fin, class SX = S>
struct EpiCgUpdate {
  static constexpr int NRED = 1;
  S w, p;
  SX xh;
  S r;
  Coef c;
  const SolverCtl* ctl;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ EpiCgUpdate at(int q) const {
    return EpiCgUpdate{w.at(q), p.at(q), xh.at(q), r.at(q), c.at(q), ctl + q, rs, fin.at(q)};
  }
  template <typename R>
  __device__ __forceinline__ void operator()(int h, R (&a)[24], double* red) const {
    const R al = (R)ctl->cg_alpha;
    const R cc = (R)c.get();
    R wv[24], pv[24], xv[24], rv[24];
    w.load(h, wv);
    p.load(h, pv);
    xh.load(h, xv);
    r.load(h, rv);
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      const R q = wv[k] + cc * a[k];
      xv[k] += al * pv[k];
      rv[k] -= al * q;
    }
    xh.store(h, xv);
    r.store_get(h, rv);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) n += rv[k] * rv[k];
    red[0] += (double)n;
  }
};

// r = b - (x + c acc) in the dslash precision (FP64 for the reliable update);
// optionally stored; reduce |r|^2
template <class Out, class B, class X, class Fin>
struct EpiResid {
  static constexpr int NRED = 1;
  Out out;
  bool store;
  B b;
  X x;
  Coef c;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ EpiResid at(int r) const {
    return EpiResid{out.at(r), store, b.at(r), x.at(r), c.at(r), rs, fin.at(r)};
  }
  template <typename R>
  __device__ __forceinline__ void operator()(int h, R (&a)[24], double* red) const {
    R bv[24], xv[24];
    b.load(h, bv);
    x.load(h, xv);
    const R cc = (R)c.get();
    R n = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      a[k] = bv[k] - (xv[k] + cc * a[k]);
      n += a[k] * a[k];
    }
    if (store) out.store(h, a);
    red[0] += (double)n;
  }
};

// x_o = b + c acc (stored) and, from the same acc, the odd rows of the true
// residual of the stored x: r_o = b - (x_o - c acc), reduced as |r_o|^2 (the
// expressions of EpiXpay and EpiResid, in FP64; Sec. 3: x_o is rebuilt from
// x_e, and the residual of the returned x is computed from the same D_oe x_e)
template <class Fin>
struct EpiReconResid {
  static constexpr int NRED = 1;
  SpinorF64 out, b;
  Coef c;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ void operator()(int h, double (&a)[24], double* red) const {
    double bv[24];
    b.load(h, bv);
    const double cc = c.get(), ncc = -cc;
    double n = 0.0;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      const double y = bv[k] + cc * a[k];
      const double r = bv[k] - (y + ncc * a[k]);
      a[k] = y;
      n += r * r;
    }
    out.store(h, a);
    red[0] += n;
  }
};

// BiCGstab reliable update: r = b_hat - (x + c acc) in FP64, r_hat = quantised
// r; reduce |r|^2 (FP64), <r_tilde, r_hat>, |r_hat|^2
template <class RH, class RT, class Fin>
struct EpiRelupBicg {
  static constexpr int NRED = 4;
  SpinorF64 b, x;
  RH rh;
  RT rt;
  Coef c;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ EpiRelupBicg at(int r) const {
    return EpiRelupBicg{b.at(r), x.at(r), rh.at(r), rt.at(r), c.at(r), rs, fin.at(r)};
  }
  __device__ __forceinline__ void operator()(int h, double (&a)[24], double* red) const {
    double bv[24], xv[24];
    b.load(h, bv);
    x.load(h, xv);
    const double cc = c.get();
#pragma unroll
    for (int k = 0; k < 24; ++k) a[k] = bv[k] - (xv[k] + cc * a[k]);
    // |r|^2 (the true-residual test of Alg. 2, needed to a few digits),
    // <r_tilde, r_hat> and |r_hat|^2 (inner-solver scalars, r_hat = r as
    // stored): per-site partials in the inner precision's arithmetic (FP32 for
    // FP32 and 16-bit storage), one FP64 add per site each
    using RI = typename RH::real;
    RI q[24];
    RI n = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      q[k] = (RI)a[k];
      n += q[k] * q[k];
    }
    red[0] += (double)n;
    rh.store_get(h, q);
    RI wv[24];
    rt.load(h, wv);
    RI re = 0, im = 0, m = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re += wv[2 * k] * q[2 * k];
      re += wv[2 * k + 1] * q[2 * k + 1];
      im += wv[2 * k] * q[2 * k + 1];
      im -= wv[2 * k + 1] * q[2 * k];
      m += q[2 * k] * q[2 * k];
      m += q[2 * k + 1] * q[2 * k + 1];
    }
    red[1] += (double)re;
    red[2] += (double)im;
    red[3] += (double)m;
  }
};

// The FP64 part of the BiCGstab reliable update for an FP32 or 16-bit inner
// precision: r = b_hat - (x + c acc) in FP64, stored rounded to FP32 (the
// values EpiRelupBicg rounds before quantising); OpRelupQuant then finishes
// the update in a bandwidth-bound pass, so the FP64-pipe-bound dslash carries
// no FP32 epilogue work and no reductions.
struct EpiResidF32 {
  static constexpr int NRED = 0;
  SpinorF32 out;
  SpinorF64 b, x;
  Coef c;
  __device__ __forceinline__ void operator()(int h, double (&a)[24], double*) const {
    double bv[24], xv[24];
    b.load(h, bv);
    x.load(h, xv);
    const double cc = c.get();
    float q[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) q[k] = (float)(bv[k] - (xv[k] + cc * a[k]));
    out.store_f(h, q);
  }
};

// r_hat = quantised r; reduce |r|^2 (from the FP32 values, one FP64 add per
// site), <r_tilde, r_hat> and |r_hat|^2: the reductions of EpiRelupBicg
template <class RH, class RT, class Fin>
struct OpRelupQuant {
  static constexpr int NRED = 4;
  SpinorF32 r;
  RH rh;
  RT rt;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ void operator()(int h, double* red) const {
    float q[24];
    r.load(h, q);
    float n = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) n += q[k] * q[k];
    red[0] += (double)n;
    rh.store_get(h, q);
    float wv[24];
    rt.load(h, wv);
    float re = 0.f, im = 0.f, m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re += wv[2 * k] * q[2 * k];
      re += wv[2 * k + 1] * q[2 * k + 1];
      im += wv[2 * k] * q[2 * k + 1];
      im -= wv[2 * k + 1] * q[2 * k];
      m += q[2 * k] * q[2 * k];
      m += q[2 * k + 1] * q[2 * k + 1];
    }
    red[1] += (double)re;
    red[2] += (double)im;
    red[3] += (double)m;
  }
};

// --------------------------------------------------------------- kernels
// Programmatic dependent launch: the solver's kernels are launched with the
// programmatic-serialization attribute, so a kernel's blocks are scheduled
// while its predecessor drains; each waits here, before it touches memory,
// until the predecessor has completed and its writes are visible.  For a
// launch without the attribute the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Resident blocks per SM the register allocation is held to (chosen from
// ptxas register and spill counts): the FP32 and 16-bit kernels are
// memory-latency bound and want warps, the fused-reduction epilogues need a
// few more registers, and the FP64 kernel is bound by the FP64 pipe.
template <typename R, class In, int NRED, bool TFIX, bool R8>
struct DslashOccupancy {
  // (the 16-bit temporal-gauge kernels with spin-paired hops spill at 5
  // blocks; the fp16 one, with scalar hops, is 1-2 % faster at 5)
  static constexpr int kMinBlocks = (sizeof(R) == 8) ? 3
                                    : R8            ? (NRED == 0 ? 4 : 3)
                                    : In::kScaled   ? (TFIX ? ((NRED == 0 && !In::kPairedHops) ? 5 : 4)
                                                            : (NRED == 0 ? 6 : 5))
                                                    : (NRED == 0 ? 5 : 4);
};

// 16-bit spinors with 12-real links take the cp.async pipeline of
// wd_async.cuh (neighbour words staged through shared memory)
constexpr bool kAsync16 = true;
template <class In, bool R8>
struct UseAsync {
  static constexpr bool value = kAsync16 && In::kBytesPerSite == 52 && !R8;
};
static_assert(kDslashBlock == kAsyncBlock, "the async slots are sized for the dslash block");

// TFIX: links in the temporal gauge; R8: FP32 / 16-bit links as the 8
// numbers of App. A.2.  Both are compile-time variants selected at launch.
template <bool DAGGER, bool TFIX, bool R8, typename R, class In, class G, class Epi>
__global__ void __launch_bounds__(kDslashBlock, (DslashOccupancy<R, In, Epi::NRED, TFIX, R8>::kMinBlocks))
    dslash_kernel(Geom g, In in, G gauge, int parity, Epi epi) {
  pdl_wait();
  constexpr int NR = Epi::NRED > 0 ? Epi::NRED : 1;
  double red[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) red[k] = 0.0;
  for (int h = g.h_begin + blockIdx.x * blockDim.x + threadIdx.x; h < g.h_end; h += gridDim.x * blockDim.x) {
    R acc[24];
    if constexpr (UseAsync<In, R8>::value) dslash_site_async<DAGGER, TFIX>(g, in, gauge, h, parity, acc);
    else dslash_site<DAGGER, TFIX, R8, Epi::NRED == 0>(g, in, gauge, h, parity, acc);
    epi(h, acc, red);
  }
  if constexpr (Epi::NRED > 0) grid_reduce<Epi::NRED>(red, epi.rs, epi.fin);
}

template <class Op>
__global__ void __launch_bounds__(kBlasBlock) site_kernel(int n, Op op) {
  pdl_wait();
  constexpr int NR = Op::NRED > 0 ? Op::NRED : 1;
  double red[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) red[k] = 0.0;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) op(h, red);
  if constexpr (Op::NRED > 0) grid_reduce<Op::NRED>(red, op.rs, op.fin);
}

__global__ void loop_control_kernel(SolverCtl* ctl);

// ------------------------------------------------------------ BLAS ops
template <class S, typename R>
__device__ __forceinline__ void cmac(R (&y)[24], double2 a, const R (&x)[24]) {  // y += a x
  const R ar = (R)a.x, ai = (R)a.y;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const R xr = x[2 * k], xi = x[2 * k + 1];
    y[2 * k] += ar * xr;
    y[2 * k] -= ai * xi;
    y[2 * k + 1] += ar * xi;
    y[2 * k + 1] += ai * xr;
  }
}

// BiCGstab: p = r + beta (p - omega v)
template <class S>
struct OpBicgP {
  static constexpr int NRED = 0;
  S r, p, v;
  const SolverCtl* ctl;
  __device__ __forceinline__ OpBicgP at(int q) const { return OpBicgP{r.at(q), p.at(q), v.at(q), ctl + q}; }
  __device__ __forceinline__ void operator()(int h, double*) const {
    using R = typename S::real;
    const double2 be = ctl->beta, om = ctl->omega;
    const double2 bo = make_double2(-(be.x * om.x - be.y * om.y), -(be.x * om.y + be.y * om.x));  // -beta omega
    R rv[24], pv[24], vv[24], o[24];
    r.load(h, rv);
    p.load(h, pv);
    v.load(h, vv);
#pragma unroll
    for (int k = 0; k < 24; ++k) o[k] = rv[k];
    cmac<S>(o, be, pv);
    cmac<S>(o, bo, vv);
    p.store(h, o);
  }
};

// s = r - alpha v, in place in r
template <class S>
struct OpBicgS {
  static constexpr int NRED = 0;
  S r, v;
  const SolverCtl* ctl;
  __device__ __forceinline__ OpBicgS at(int q) const { return OpBicgS{r.at(q), v.at(q), ctl + q}; }
  __device__ __forceinline__ void operator()(int h, double*) const {
    using R = typename S::real;
    const double2 al = ctl->alpha;
    R rv[24], vv[24];
    r.load(h, rv);
    v.load(h, vv);
    cmac<S>(rv, make_double2(-al.x, -al.y), vv);
    r.store(h, rv);
  }
};

// x_hat += alpha p + omega s; r = s - omega t (s lives in r); reduce |r|^2, <r_tilde, r>
template <class S, class SX = S>
struct OpBicgFinal {
  static constexpr int NRED = 3;
  SX xh;
  S p, r, t, rt;
  const SolverCtl* ctl;
  RedScratch rs;
  FinBicgIter fin;
  __device__ __forceinline__ OpBicgFinal at(int q) const {
    return OpBicgFinal{xh.at(q), p.at(q), r.at(q), t.at(q), rt.at(q), ctl + q, rs, fin.at(q)};
  }
  __device__ __forceinline__ void operator()(int h, double* red) const {
    using R = typename S::real;
    const double2 al = ctl->alpha, om = ctl->omega;
    R xv[24], pv[24], sv[24], tv[24], wv[24];
    xh.load(h, xv);
    p.load(h, pv);
    r.load(h, sv);
    t.load(h, tv);
    cmac<S>(xv, al, pv);
    cmac<S>(xv, om, sv);
    xh.store(h, xv);
    cmac<S>(sv, make_double2(-om.x, -om.y), tv);
    r.store_get(h, sv);
    rt.load(h, wv);
    R n = 0, re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R a = sv[2 * k], b = sv[2 * k + 1], wr = wv[2 * k], wi = wv[2 * k + 1];
      n += a * a;
      n += b * b;
      re += wr * a;
      re += wi * b;
      im += wr * b;
      im -= wi * a;
    }
    red[0] += (double)n;
    red[1] += (double)re;
    red[2] += (double)im;
  }
};

// CG: p = r + beta p
template <class S>
struct OpCgP {
  static constexpr int NRED = 0;
  S r, p;
  const SolverCtl* ctl;
  __device__ __forceinline__ OpCgP at(int q) const { return OpCgP{r.at(q), p.at(q), ctl + q}; }
  __device__ __forceinline__ void operator()(int h, double*) const {
    using R = typename S::real;
    const R be = (R)ctl->beta.x;
    R rv[24], pv[24];
    r.load(h, rv);
    p.load(h, pv);
#pragma unroll
    for (int k = 0; k < 24; ++k) pv[k] = rv[k] + be * pv[k];
    p.store(h, pv);
  }
};

// Alg. 2: x = x + x_hat (FP64 accumulation), x_hat = 0
template <class S>
struct OpAccumulate {
  static constexpr int NRED = 0;
  SpinorF64 x;
  S xh;
  __device__ __forceinline__ OpAccumulate at(int r) const { return OpAccumulate{x.at(r), xh.at(r)}; }
  __device__ __forceinline__ void operator()(int h, double*) const {
    double xv[24], hv[24];
    x.load(h, xv);
    xh.load(h, hv);
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      xv[k] += hv[k];
      hv[k] = 0.0;
    }
    x.store(h, xv);
    xh.store(h, hv);
  }
};

// defect correction only (ctl->restart): r_tilde = r_hat, p = v = 0
template <class S>
struct OpRestart {
  static constexpr int NRED = 0;
  S rt, rh, p, v;
  const SolverCtl* ctl;
  __device__ __forceinline__ OpRestart at(int q) const {
    return OpRestart{rt.at(q), rh.at(q), p.at(q), v.at(q), ctl + q};
  }
  __device__ __forceinline__ void operator()(int h, double*) const {
    using R = typename S::real;
    if (!ctl->restart) return;
    R a[24];
    rh.load(h, a);
    rt.store(h, a);
#pragma unroll
    for (int k = 0; k < 24; ++k) a[k] = 0;
    p.store(h, a);
    v.store(h, a);
  }
};

// out = in with precision conversion
template <class Out, class In>
struct OpConvert {
  static constexpr int NRED = 0;
  Out out;
  In in;
  __device__ __forceinline__ OpConvert at(int r) const { return OpConvert{out.at(r), in.at(r)}; }
  __device__ __forceinline__ void operator()(int h, double*) const {
    using R = typename In::real;
    R v[24];
    in.load(h, v);
    out.store(h, v);
  }
};

// out1 = out2 = quantised in; reduce <out, out> (complex) and |out|^2
template <class Out, class In, class Fin>
struct OpQuantDup {
  static constexpr int NRED = 3;
  Out out1, out2;
  In in;
  RedScratch rs;
  Fin fin;
  __device__ __forceinline__ OpQuantDup at(int r) const {
    return OpQuantDup{out1.at(r), out2.at(r), in.at(r), rs, fin.at(r)};
  }
  __device__ __forceinline__ void operator()(int h, double* red) const {
    double v[24], v2[24];
    in.load(h, v);
#pragma unroll
    for (int k = 0; k < 24; ++k) v2[k] = v[k];
    out1.store_get(h, v);
    out2.store(h, v2);  // same source, same encoding: identical bits
    double n = 0.0;
#pragma unroll
    for (int k = 0; k < 24; ++k) n += v[k] * v[k];
    red[0] += n;
    red[2] += n;
  }
};

template <class S>
struct OpNorm2 {
  static constexpr int NRED = 1;
  S in;
  RedScratch rs;
  FinStore fin;
  __device__ __forceinline__ OpNorm2 at(int r) const { return OpNorm2{in.at(r), rs, fin.at(r)}; }
  __device__ __forceinline__ void operator()(int h, double* red) const {
    using R = typename S::real;
    R v[24];
    in.load(h, v);
    double n = 0.0;  // API norm: every square accumulated in FP64 (not on the solver path)
#pragma unroll
    for (int k = 0; k < 24; ++k) n += (double)v[k] * v[k];
    red[0] += n;
  }
};

template <class S>
struct OpZero {
  static constexpr int NRED = 0;
  S out;
  __device__ __forceinline__ OpZero at(int r) const { return OpZero{out.at(r)}; }
  __device__ __forceinline__ void operator()(int h, double*) const {
    float z[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) z[k] = 0.f;
    out.store(h, z);
  }
};

// App. B basis change, applied when a spinor crosses the host boundary:
// psi_int = S psi_DR with the real orthogonal
//   S = (1/sqrt 2) [[0,1,0,1], [-1,0,-1,0], [0,1,0,-1], [-1,0,1,0]],
// for which S gamma_mu S^T is the gamma_mu of the UKQCD set printed in App. B
// (gamma_4 diagonal).  Spinor index (spin * 3 + colour) * 2 + reim.
__device__ __forceinline__ void to_internal_basis(const double (&d)[24], double (&v)[24]) {
  constexpr double r = 0.70710678118654752440;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double p0 = d[k], p1 = d[6 + k], p2 = d[12 + k], p3 = d[18 + k];
    v[k] = r * (p1 + p3);
    v[6 + k] = -r * (p0 + p2);
    v[12 + k] = r * (p1 - p3);
    v[18 + k] = r * (p2 - p0);
  }
}
__device__ __forceinline__ void to_host_basis(const double (&v)[24], double (&d)[24]) {
  constexpr double r = 0.70710678118654752440;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double u0 = v[k], u1 = v[6 + k], u2 = v[12 + k], u3 = v[18 + k];
    d[k] = -r * (u1 + u3);
    d[6 + k] = r * (u0 + u2);
    d[12 + k] = r * (u3 - u1);
    d[18 + k] = r * (u0 - u2);
  }
}

// Temporal gauge (Sec. 4.3): colour rotation of every spin component of a
// site by G(x) (import) or G(x)^dag (export).  G: [parity][9][stride]
// double2, row-major 3x3.
__device__ __forceinline__ void gauge_rotate(double (&v)[24], const double2* G, const Geom& g, int parity, int h,
                                             bool dag) {
  double2 m[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = G[(size_t)(parity * 9 + k) * g.stride + h];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    double o[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double2 e = dag ? m[j * 3 + i] : m[i * 3 + j];
        const double vr = v[(sp * 3 + j) * 2], vi = v[(sp * 3 + j) * 2 + 1];
        if (dag) {  // conj(G_ji) v_j
          re += e.x * vr;
          re += e.y * vi;
          im += e.x * vi;
          im -= e.y * vr;
        } else {  // G_ij v_j
          re += e.x * vr;
          re -= e.y * vi;
          im += e.x * vi;
          im += e.y * vr;
        }
      }
      o[2 * i] = re;
      o[2 * i + 1] = im;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) v[sp * 6 + k] = o[k];
  }
}

// host layout (lexicographic FP64, [site][spin][colour][re,im]) <-> field
template <class S>
struct OpImport {
  static constexpr int NRED = 0;
  Geom g;
  S out;
  const double* lex;
  int parity;
  const double2* gfix;  // temporal-gauge transformation, or nullptr
  __device__ __forceinline__ void operator()(int h, double*) const {
    int x, y, z, t;
    site_coords(g, h, parity, x, y, z, t);
    const size_t s = (size_t)x + (size_t)g.X * (y + (size_t)g.Y * (z + (size_t)g.Z * t));
    double d[24], v[24];
    const double2* src = reinterpret_cast<const double2*>(lex + 24 * s);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 e = src[k];
      d[2 * k] = e.x;
      d[2 * k + 1] = e.y;
    }
    to_internal_basis(d, v);
    if (gfix) gauge_rotate(v, gfix, g, parity, h, false);
    out.store(h, v);
  }
};

template <class S>
struct OpExport {
  static constexpr int NRED = 0;
  Geom g;
  S in;
  double* lex;
  int parity;
  const double2* gfix;
  __device__ __forceinline__ void operator()(int h, double*) const {
    using R = typename S::real;
    int x, y, z, t;
    site_coords(g, h, parity, x, y, z, t);
    const size_t s = (size_t)x + (size_t)g.X * (y + (size_t)g.Y * (z + (size_t)g.Z * t));
    R v[24];
    in.load(h, v);
    double w[24], d[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) w[k] = (double)v[k];
    if (gfix) gauge_rotate(w, gfix, g, parity, h, true);
    to_host_basis(w, d);
    double2* dst = reinterpret_cast<double2*>(lex + 24 * s);
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = make_double2(d[2 * k], d[2 * k + 1]);
  }
};

// ---------------------------------------------------------------- views
template <int P>
struct Tr;

template <>
struct Tr<WD_F64> {
  using S = SpinorF64;
  using G = GaugeF64;
  using R = double;
  static size_t bytes(int stride) { return align256(192 * (size_t)stride); }
  static S view(const void* p, const Geom& g, size_t rs = 0) { return S{(double2*)p, g.stride, rs}; }
  static G gauge(const Ctx& c) { return G{(const double2*)c.gauge[WD_F64], c.g.stride, c.recon}; }
  // T-slab faces (wd_slab.cuh)
  using Fc = FaceF64;
  static size_t face_bytes(int fs) { return align256(96 * (size_t)fs); }
  static Fc face(const void* p, int fs) { return Fc{(const double2*)p, fs}; }
  static size_t link_face_bytes(const Ctx& c, int fs) { return align256((size_t)2 * (c.recon / 2) * 16 * fs); }
  static LinkFace<G> link_face(const Ctx& c, const void* p, int fs) { return {G{(const double2*)p, fs, c.recon}}; }
  static void pack_faces(const Ctx& c, void* lo, void* hi, const void* in, int fs, int dagger, int grid,
                         cudaStream_t s) {
    pack_faces_f64_kernel<<<grid, 256, 0, s>>>(c.g, (const double2*)in, c.g.stride, (double2*)lo, (double2*)hi, fs,
                                               dagger);
  }
  static void pack_link_face(const Ctx& c, void* out, int fs, int grid, cudaStream_t s) {
    pack_link_face_kernel<double2><<<grid, 256, 0, s>>>(c.g, (const double2*)c.gauge[WD_F64], c.recon / 2,
                                                        c.g.stride, (double2*)out, fs);
  }
};
template <>
struct Tr<WD_F32> {
  using S = SpinorF32;
  using G = GaugeF32;
  using R = float;
  static size_t bytes(int stride) { return align256(96 * (size_t)stride); }
  static S view(const void* p, const Geom& g, size_t rs = 0) { return S{(float4*)p, g.stride, rs}; }
  static G gauge(const Ctx& c) { return G{(const float4*)c.gauge[WD_F32], c.g.stride, c.low_recon}; }
  using Fc = FaceF32;
  static size_t face_bytes(int fs) { return align256(48 * (size_t)fs); }
  static Fc face(const void* p, int fs) { return Fc{(const float4*)p, fs}; }
  static size_t link_face_bytes(const Ctx&, int fs) { return align256((size_t)2 * 3 * 16 * fs); }
  static LinkFace<G> link_face(const Ctx&, const void* p, int fs) { return {G{(const float4*)p, fs, 12}}; }
  static void pack_faces(const Ctx& c, void* lo, void* hi, const void* in, int fs, int dagger, int grid,
                         cudaStream_t s) {
    pack_faces_f32_kernel<<<grid, 256, 0, s>>>(c.g, (const float4*)in, c.g.stride, (float4*)lo, (float4*)hi, fs,
                                               dagger);
  }
  static void pack_link_face(const Ctx& c, void* out, int fs, int grid, cudaStream_t s) {
    pack_link_face_kernel<float4><<<grid, 256, 0, s>>>(c.g, (const float4*)c.gauge[WD_F32], 3, c.g.stride,
                                                       (float4*)out, fs);
  }
};
template <Fmt16 F, int P>
struct Tr16 {
  using S = Spinor16<F>;
  using G = Gauge16<F>;
  using R = float;
  static size_t bytes(int stride) { return align256(48 * (size_t)stride) + align256(4 * (size_t)stride); }
  static S view(const void* p, const Geom& g, size_t rs = 0) {
    return S{(uint4*)p, (float*)((char*)p + align256(48 * (size_t)g.stride)), g.stride, rs};
  }
  static G gauge(const Ctx& c) {
    return G{(const uint4*)c.gauge[P], (const uint2*)c.gauge4[P], c.g.stride, c.low_recon};
  }
  using Fc = Face16<F>;
  static size_t face_bytes(int fs) {
    return align256(16 * (size_t)fs) + align256(8 * (size_t)fs) + align256(4 * (size_t)fs);
  }
  static Fc face(const void* p, int fs) {
    const char* b = (const char*)p;
    return Fc{(const uint4*)b, (const uint2*)(b + align256(16 * (size_t)fs)),
              (const float*)(b + align256(16 * (size_t)fs) + align256(8 * (size_t)fs)), fs};
  }
  static size_t link_face_bytes(const Ctx&, int fs) { return align256(32 * (size_t)fs) + align256(16 * (size_t)fs); }
  static LinkFace<G> link_face(const Ctx&, const void* p, int fs) {
    const char* b = (const char*)p;
    return {G{(const uint4*)b, (const uint2*)(b + align256(32 * (size_t)fs)), fs, 12}};
  }
  static void pack_faces(const Ctx& c, void* lo, void* hi, const void* in, int fs, int dagger, int grid,
                         cudaStream_t s) {
    const size_t ob = align256(16 * (size_t)fs), on = ob + align256(8 * (size_t)fs);
    char* l = (char*)lo;
    char* h = (char*)hi;
    pack_faces_16_kernel<<<grid, 256, 0, s>>>(c.g, (const uint4*)in,
                                              (const float*)((const char*)in + align256(48 * (size_t)c.g.stride)),
                                              c.g.stride, (uint4*)l, (uint2*)(l + ob), (float*)(l + on), (uint4*)h,
                                              (uint2*)(h + ob), (float*)(h + on), fs, dagger);
  }
  static void pack_link_face(const Ctx& c, void* out, int fs, int grid, cudaStream_t s) {
    char* o = (char*)out;
    pack_link_face_kernel<uint4><<<grid, 256, 0, s>>>(c.g, (const uint4*)c.gauge[P], 1, c.g.stride, (uint4*)o, fs);
    pack_link_face_kernel<uint2><<<grid, 256, 0, s>>>(c.g, (const uint2*)c.gauge4[P], 1, c.g.stride,
                                                      (uint2*)(o + align256(32 * (size_t)fs)), fs);
  }
};
template <>
struct Tr<WD_Q16> : Tr16<Fmt16::Q16, WD_Q16> {};
template <>
struct Tr<WD_H16N> : Tr16<Fmt16::H16, WD_H16N> {};
template <>
struct Tr<WD_B16N> : Tr16<Fmt16::B16, WD_B16N> {};

// ------------------------------------------------------------ launchers
// Resident blocks per SM of a kernel at a block size (asked once per kernel
// instantiation by its launcher).
template <class K>
inline int resident_blocks(K kernel, int block) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 2;
  }
  return occ;
}
// Launch with the programmatic-serialization attribute (see pdl_wait); on a
// stream being captured it becomes a programmatic edge of the graph.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Grid of the grid-stride kernels: one wave of resident blocks (every block
// resident for the whole launch, no partially filled last wave), or fewer
// blocks when the sites do not fill it.
inline int wave_grid(int units, int block, int num_sms, int per_sm) {
  const int b = (units + block - 1) / block;
  const int w = num_sms * per_sm;
  return b < w ? b : w;
}

template <typename R, class In, class G, class Epi>
void launch_dslash(const Ctx& c, const In& in, const G& gauge, int parity, int dagger, const Epi& epi,
                   cudaStream_t s, const Geom* sub = nullptr) {
  // sub: the context's geometry with a narrower output-site range
  const Geom& geo = sub ? *sub : c.g;
  // FP64 links never use the 8 numbers
  const bool r8 = (sizeof(R) == 4) && c.low_recon == 8;
  auto go = [&](auto dag, auto tfix, auto rec8) {
    constexpr bool kTfix = decltype(tfix)::value;
    auto* k = dslash_kernel<decltype(dag)::value, kTfix, decltype(rec8)::value, R, In, G, Epi>;
    // One wave of resident blocks, measured per kernel class against 16
    // blocks per SM (several waves, the last one partly filled) at 64^3x128:
    // FP32 15 % faster, 16-bit temporal-gauge and 8-number kernels 5-8 %,
    // H16N/B16N general links 2-3 %; at 24^3x64 the plain Q16 dslash is 2 %
    // slower on one wave but its reduction epilogues (fewer block partials)
    // gain more: the benchmark solve is 3.4 % faster than with 16 blocks per
    // SM for the small lattices.  The FP64 kernel (FP64-pipe bound; 6 %
    // slower at 24^3x64) and the general-link Q16 kernel (6 % slower at
    // 64^3x128) keep 16 blocks per SM.
    constexpr bool kWave = !(sizeof(R) == 8 || (In::kIntCodes && !kTfix));
    static const int per_sm = kWave ? resident_blocks(k, kDslashBlock) : 16;
    const int grid = wave_grid(geo.h_end - geo.h_begin, kDslashBlock, c.num_sms, per_sm);
    launch_pdl(k, dim3(grid), dim3(kDslashBlock), 0, s, geo, in, gauge, parity, epi);
  };
  using T_ = std::true_type;
  using F_ = std::false_type;
  if constexpr (sizeof(R) == 4) {
    if (r8) {
      if (c.g.tfix) dagger ? go(T_{}, T_{}, T_{}) : go(F_{}, T_{}, T_{});
      else dagger ? go(T_{}, F_{}, T_{}) : go(F_{}, F_{}, T_{});
      return;
    }
  }
  if (c.g.tfix) dagger ? go(T_{}, T_{}, F_{}) : go(F_{}, T_{}, F_{});
  else dagger ? go(T_{}, F_{}, F_{}) : go(F_{}, F_{}, F_{});
}

template <class Op>
void launch_sites(const Ctx& c, int n, const Op& op, cudaStream_t s) {
  static const int per_sm = resident_blocks(site_kernel<Op>, kBlasBlock);
  launch_pdl(site_kernel<Op>, dim3(wave_grid(n, kBlasBlock, c.num_sms, per_sm)), dim3(kBlasBlock), 0, s, n, op);
}

// Per-precision implementation.  Inner fields are of precision P; the
// reliable update runs the FP64 dslash with P-precision outputs.
template <int P>
struct Impl {
  using T = Tr<P>;
  using S = typename T::S;
  using R = typename T::R;
  using T64 = Tr<WD_F64>;

  static size_t field_bytes(int stride) { return T::bytes(stride); }

  static void dslash(const Ctx& c, void* out, const void* in, int parity, int dagger, cudaStream_t s) {
    EpiStore<S> e{T::view(out, c.g)};
    launch_dslash<R>(c, T::view(in, c.g), T::gauge(c), parity, dagger, e, s);
  }
  static void dslash_xpay(const Ctx& c, void* out, const void* in, const void* x, double a, const double* a_dev,
                          int parity, int dagger, cudaStream_t s) {
    EpiXpay<S, S> e{T::view(out, c.g), T::view(x, c.g), Coef{a, a_dev}};
    launch_dslash<R>(c, T::view(in, c.g), T::gauge(c), parity, dagger, e, s);
  }
  static void import_lex(const Ctx& c, void* field, const double* lex, int parity, cudaStream_t s) {
    launch_sites(c, c.g.Vh, OpImport<S>{c.g, T::view(field, c.g), lex, parity, c.gfix}, s);
  }
  static void export_lex(const Ctx& c, double* lex, const void* field, int parity, cudaStream_t s) {
    launch_sites(c, c.g.Vh, OpExport<S>{c.g, T::view(field, c.g), lex, parity, c.gfix}, s);
  }
  static void from_f64(const Ctx& c, void* out, const void* in, cudaStream_t s) {
    launch_sites(c, c.g.Vh, OpConvert<S, SpinorF64>{T::view(out, c.g), T64::view(in, c.g)}, s);
  }
  static void to_f64(const Ctx& c, void* out, const void* in, cudaStream_t s) {
    launch_sites(c, c.g.Vh, OpConvert<SpinorF64, S>{T64::view(out, c.g), T::view(in, c.g)}, s);
  }
  static void norm2(const Ctx& c, double* out, const void* field, cudaStream_t s) {
    launch_sites(c, c.g.Vh, OpNorm2<S>{T::view(field, c.g), c.red, FinStore{out, 1}}, s);
  }
  static void zero(const Ctx& c, void* field, cudaStream_t s) {
    launch_sites(c, c.g.Vh, OpZero<S>{T::view(field, c.g)}, s);
  }

  // ---- BiCGstab on M_hat (Sec. 5.1), inner precision P
  // x_hat in FP32 instead of the 16-bit inner precision (SolveBufs::xhat_f32)
  using TX = Tr<WD_F32>;
  static bool xf32(const SolveBufs& b) { return b.xhat_f32 && T::S::kBytesPerSite < 96; }
  static void zero_xhat(const Ctx& c, SolveBufs& b, cudaStream_t s) {
    if (xf32(b)) launch_sites(c, c.g.Vh, OpZero<SpinorF32>{TX::view(b.x_hat, c.g)}, s);
    else zero(c, b.x_hat, s);
  }
  static void accumulate(const Ctx& c, SolveBufs& b, cudaStream_t s) {
    if (xf32(b)) launch_sites(c, c.g.Vh, OpAccumulate<SpinorF32>{T64::view(b.x, c.g), TX::view(b.x_hat, c.g)}, s);
    else launch_sites(c, c.g.Vh, OpAccumulate<S>{T64::view(b.x, c.g), T::view(b.x_hat, c.g)}, s);
  }

  static void bicg_setup(const Ctx& c, SolveBufs& b, const void* src, cudaStream_t s) {
    using Q = OpQuantDup<S, SpinorF64, FinBicgSetup>;
    launch_sites(c, c.g.Vh, Q{T::view(b.r_hat, c.g), T::view(b.r_tilde, c.g), T64::view(src, c.g), c.red,
                               FinBicgSetup{b.ctl}}, s);
    zero(c, b.p, s);
    zero(c, b.v, s);
    zero_xhat(c, b, s);
  }
  static void bicg_iteration(const Ctx& c, SolveBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    const Coef nk2{0.0, &b.ctl->neg_kappa2};
    // p = r + beta (p - omega v)
    launch_sites(c, g.Vh, OpBicgP<S>{T::view(b.r_hat, g), T::view(b.p, g), T::view(b.v, g), b.ctl}, s);
    // v = M_hat p, alpha = rho / <r_tilde, v>
    dslash(c, b.tmp, b.p, 1, 0, s);
    {
      EpiXpayDot<S, S, S, FinBicgAlpha> e{T::view(b.v, g), T::view(b.p, g), T::view(b.r_tilde, g), nk2, c.red,
                                          FinBicgAlpha{b.ctl}};
      launch_dslash<R>(c, T::view(b.tmp, g), T::gauge(c), 0, 0, e, s);
    }
    // s = r - alpha v
    launch_sites(c, g.Vh, OpBicgS<S>{T::view(b.r_hat, g), T::view(b.v, g), b.ctl}, s);
    // t = M_hat s, omega = <t, s> / <t, t>
    dslash(c, b.tmp, b.r_hat, 1, 0, s);
    {
      EpiXpayTS<S, S, FinBicgOmega> e{T::view(b.t, g), T::view(b.r_hat, g), nk2, c.red, FinBicgOmega{b.ctl}};
      launch_dslash<R>(c, T::view(b.tmp, g), T::gauge(c), 0, 0, e, s);
    }
    // x_hat += alpha p + omega s, r = s - omega t, |r|^2, rho = <r_tilde, r>
    if (xf32(b))
      launch_sites(c, g.Vh,
                   OpBicgFinal<S, SpinorF32>{TX::view(b.x_hat, g), T::view(b.p, g), T::view(b.r_hat, g),
                                             T::view(b.t, g), T::view(b.r_tilde, g), b.ctl, c.red,
                                             FinBicgIter{b.ctl}},
                   s);
    else
      launch_sites(c, g.Vh,
                   OpBicgFinal<S>{T::view(b.x_hat, g), T::view(b.p, g), T::view(b.r_hat, g), T::view(b.t, g),
                                  T::view(b.r_tilde, g), b.ctl, c.red, FinBicgIter{b.ctl}},
                   s);
  }
  // Alg. 2 reliable update: x += x_hat, x_hat = 0, r = b_hat - M_hat x (FP64),
  // r_hat = r (quantised), rho = <r_tilde, r_hat>
  static void bicg_update(const Ctx& c, SolveBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    accumulate(c, b, s);
    EpiStore<SpinorF64> e0{T64::view(b.tmp64, g)};
    launch_dslash<double>(c, T64::view(b.x, g), T64::gauge(c), 1, 0, e0, s);
    if constexpr (P != WD_F64) {
      // r in FP32 in the FP64 residual buffer (unused by BiCGstab), then the
      // quantisation and reductions in a pass of their own
      EpiResidF32 e1{TX::view(b.r, g), T64::view(b.b_hat, g), T64::view(b.x, g), Coef{0.0, &b.ctl->neg_kappa2}};
      launch_dslash<double>(c, T64::view(b.tmp64, g), T64::gauge(c), 0, 0, e1, s);
      launch_sites(c, g.Vh,
                   OpRelupQuant<S, S, FinRelupBicg>{TX::view(b.r, g), T::view(b.r_hat, g), T::view(b.r_tilde, g),
                                                    c.red, FinRelupBicg{b.ctl}},
                   s);
    } else {
      EpiRelupBicg<S, S, FinRelupBicg> e1{T64::view(b.b_hat, g), T64::view(b.x, g), T::view(b.r_hat, g),
                                           T::view(b.r_tilde, g), Coef{0.0, &b.ctl->neg_kappa2}, c.red,
                                           FinRelupBicg{b.ctl}};
      launch_dslash<double>(c, T64::view(b.tmp64, g), T64::gauge(c), 0, 0, e1, s);
    }
    launch_sites(c, g.Vh, OpRestart<S>{T::view(b.r_tilde, g), T::view(b.r_hat, g), T::view(b.p, g), T::view(b.v, g),
                                       b.ctl},
                 s);
  }

  // ---- CG on M_hat^dag M_hat (Sec. 5.1), inner precision P
  static void cg_setup(const Ctx& c, SolveBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    // r_hat = M_hat^dag b_hat  (FP64 dslash, output quantised)
    EpiStore<SpinorF64> e0{T64::view(b.tmp64, g)};
    launch_dslash<double>(c, T64::view(b.b_hat, g), T64::gauge(c), 1, 1, e0, s);
    EpiXpayNorm<S, SpinorF64, FinCgSetup> e1{T::view(b.r_hat, g), T64::view(b.b_hat, g),
                                             Coef{0.0, &b.ctl->neg_kappa2}, c.red,
                                             FinCgSetup{b.ctl, c.scalars + 2}};
    launch_dslash<double>(c, T64::view(b.tmp64, g), T64::gauge(c), 0, 1, e1, s);
    zero(c, b.p, s);
    zero_xhat(c, b, s);
  }
  static void cg_iteration(const Ctx& c, SolveBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    const Coef nk2{0.0, &b.ctl->neg_kappa2};
    launch_sites(c, g.Vh, OpCgP<S>{T::view(b.r_hat, g), T::view(b.p, g), b.ctl}, s);
    // w = M_hat p, alpha = |r|^2 / |w|^2
    dslash(c, b.tmp, b.p, 1, 0, s);
    {
      EpiXpayNorm<S, S, FinCgAlpha> e{T::view(b.v, g), T::view(b.p, g), nk2, c.red, FinCgAlpha{b.ctl}};
      launch_dslash<R>(c, T::view(b.tmp, g), T::gauge(c), 0, 0, e, s);
    }
    // q = M_hat^dag w; x_hat += alpha p; r -= alpha q; |r|^2
    dslash(c, b.tmp, b.v, 1, 1, s);
    if (xf32(b)) {
      EpiCgUpdate<S, FinCgIter, SpinorF32> e{T::view(b.v, g), T::view(b.p, g), TX::view(b.x_hat, g),
                                             T::view(b.r_hat, g), nk2, b.ctl, c.red, FinCgIter{b.ctl}};
      launch_dslash<R>(c, T::view(b.tmp, g), T::gauge(c), 0, 1, e, s);
    } else {
      EpiCgUpdate<S, FinCgIter> e{T::view(b.v, g), T::view(b.p, g), T::view(b.x_hat, g), T::view(b.r_hat, g),
                                  nk2, b.ctl, c.red, FinCgIter{b.ctl}};
      launch_dslash<R>(c, T::view(b.tmp, g), T::gauge(c), 0, 1, e, s);
    }
  }
  static void cg_update(const Ctx& c, SolveBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    const Coef nk2{0.0, &b.ctl->neg_kappa2};
    accumulate(c, b, s);
    // r = b_hat - M_hat x  (FP64, stored)
    EpiStore<SpinorF64> e0{T64::view(b.tmp64, g)};
    launch_dslash<double>(c, T64::view(b.x, g), T64::gauge(c), 1, 0, e0, s);
    EpiResid<SpinorF64, SpinorF64, SpinorF64, FinRelupCgR> e1{
        T64::view(b.r, g), true, T64::view(b.b_hat, g), T64::view(b.x, g), nk2, c.red, FinRelupCgR{b.ctl}};
    launch_dslash<double>(c, T64::view(b.tmp64, g), T64::gauge(c), 0, 0, e1, s);
    // r_hat = M_hat^dag r (quantised)
    launch_dslash<double>(c, T64::view(b.r, g), T64::gauge(c), 1, 1, e0, s);
    EpiXpayNorm<S, SpinorF64, FinRelupCgN> e2{T::view(b.r_hat, g), T64::view(b.r, g), nk2, c.red,
                                              FinRelupCgN{b.ctl}};
    launch_dslash<double>(c, T64::view(b.tmp64, g), T64::gauge(c), 0, 1, e2, s);
  }

  // ---- T-slab decomposition (Sec. 6): faces and the split dslash
  static size_t slab_face_bytes(const Ctx& c) { return T::face_bytes(face_stride(c.g)); }
  static size_t slab_link_face_bytes(const Ctx& c) { return T::link_face_bytes(c, face_stride(c.g)); }
  static void slab_pack_faces(const Ctx& c, void* lo, void* hi, const void* in, int dagger, cudaStream_t s) {
    const int grid = wave_grid(2 * c.g.XhYZ, 256, c.num_sms, 8);
    T::pack_faces(c, lo, hi, in, face_stride(c.g), dagger, grid, s);
  }
  static void slab_pack_link_face(const Ctx& c, void* face, cudaStream_t s) {
    const int grid = wave_grid(2 * c.g.XhYZ * 9, 256, c.num_sms, 8);
    T::pack_link_face(c, face, face_stride(c.g), grid, s);
  }
  static void slab_dslash(const Ctx& c, void* out, const void* in, const void* halo_lo, const void* halo_hi,
                          const void* link_halo, int flip_lo, int flip_hi, int parity, int dagger, int region,
                          cudaStream_t s) {
    // the interior slices need no halo: the whole-lattice kernel (cp.async
    // pipeline, spin-paired hops) over their site range; region 2 is the
    // interior launch followed by the boundary one, so that it writes what
    // regions 0 and 1 write
    if (region == 0 || region == 2) {
      Geom sub = c.g;
      sub.h_begin = c.g.XhYZ;
      sub.h_end = c.g.XhYZ * (c.g.T - 1);
      if (sub.h_end > sub.h_begin) {
        EpiStore<S> e{T::view(out, c.g)};
        launch_dslash<R>(c, T::view(in, c.g), T::gauge(c), parity, dagger, e, s, &sub);
      }
      if (region == 0) return;
      region = 1;
    }
    const int fs = face_stride(c.g);
    const SlabRegion reg{region, c.g.XhYZ, c.g.T, c.g.Vh};
    const int n = reg.count();
    if (n <= 0) return;
    EpiStore<S> e{T::view(out, c.g)};
    const auto lf = T::link_face(c, link_halo, fs);
    const auto flo = T::face(halo_lo, fs), fhi = T::face(halo_hi, fs);
    auto go = [&](auto dag) {
      auto* k = dslash_slab_kernel<decltype(dag)::value, R, S, typename T::G, typename T::Fc, decltype(lf),
                                   EpiStore<S>>;
      static const int per_sm = resident_blocks(k, kDslashBlock);
      const int grid = wave_grid(n, kDslashBlock, c.num_sms, per_sm);
      k<<<grid, kDslashBlock, 0, s>>>(c.g, T::view(in, c.g), T::gauge(c), flo, fhi, lf, flip_lo, flip_hi, parity, reg,
                                      e);
    };
    if (dagger) go(std::true_type{});
    else go(std::false_type{});
  }

  static PrecOps make() {
    PrecOps o{};
    o.prec = (wd_prec)P;
    o.field_bytes = &field_bytes;
    o.dslash = &dslash;
    o.dslash_xpay = &dslash_xpay;
    o.import_lex = &import_lex;
    o.export_lex = &export_lex;
    o.from_f64 = &from_f64;
    o.to_f64 = &to_f64;
    o.norm2 = &norm2;
    o.zero = &zero;
    o.bicg_iteration = &bicg_iteration;
    o.bicg_update = &bicg_update;
    o.bicg_setup = &bicg_setup;
    o.cg_iteration = &cg_iteration;
    o.cg_update = &cg_update;
    o.cg_setup = &cg_setup;
    o.slab_face_bytes = &slab_face_bytes;
    o.slab_link_face_bytes = &slab_link_face_bytes;
    o.slab_pack_faces = &slab_pack_faces;
    o.slab_pack_link_face = &slab_pack_link_face;
    o.slab_dslash = &slab_dslash;
    return o;
  }
};

}  // namespace wd
