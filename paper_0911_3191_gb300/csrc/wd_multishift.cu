// Multi-shift solves over kappa (C ABI): M_kappa_k x_k = b for several kappa
// on one gauge field with one Krylov space.  This goes beyond arXiv:0911.3191
// (whose use case, Sec. 3, is many solves on one gauge field); it is the
// shifted-system Krylov method (Jegerlehner 1996; Frommer 2003) applied to the
// even-odd system of Sec. 3.
//
// The kappa family is a shifted family: with Q = -D_eo D_oe,
// M_hat(kappa) = 1 + kappa^2 Q, so for the seed kappa_s (the largest kappa,
// the slowest system) M_hat(kappa_k) = (kappa_k / kappa_s)^2 (B + tau_k) with
// B = M_hat(kappa_s) and tau_k = (kappa_s / kappa_k)^2 - 1 >= 0.  The Schur
// source b_hat_k = b_e + kappa_k D_eo b_o is a kappa-dependent combination of
// u = b_e and w = D_eo b_o, so the shifted family is solved for u (and for w
// when b_o is not zero): (B + tau_k) y_k = u, (B + tau_k) z_k = w, and
// x_e,k = (kappa_s / kappa_k)^2 (y_k + kappa_k z_k).
//
// GB300 layout of the work: the multi-shift BiCGstab runs in FP32 storage
// (two FP32 M_hat applications per iteration serve every kappa; per-shift
// vectors x_k, p_k updated by one fused kernel over all shifts; every scalar
// on the device, the loop one CUDA graph) down to a
// relative residual of 1e-7 (or the requested tol if larger); each kappa is
// then finished by the mixed-precision reliable-update solver of Alg. 2,
// started from x_k (its first step the FP64 residual b_hat - M_hat x_k), which
// brings the FP64 true residual to tol and rebuilds the odd half.  The recurrences for the shifted scalars are derived in
// the oracle's multishift module (test infrastructure), whose pins the tests
// run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "wd_kernels.cuh"

using namespace wd;

namespace {

using cplx = std::complex<double>;
constexpr int kMaxShifts = 32;
constexpr double kStageTol = 1e-7;  // FP32 multi-shift stage target (relative)

wd_status merr(wd_ctx* ctx, wd_status st, const std::string& m) {
  ctx->c.last_error = m;
  return st;
}

#define MS_CK(call)                                                                                        \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess)                                                                                 \
      return merr(ctx, e_ == cudaErrorMemoryAllocation ? WD_ERR_OOM : WD_ERR_CUDA,                         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                     \
  } while (0)
#define MS_ST(call)                           \
  do {                                        \
    wd_status s_ = (call);                    \
    if (s_ != WD_OK) return s_;               \
  } while (0)

// (<a, b>, |a|^2) with <a, b> = sum_sites conj(a) . b: per-site partials in
// FP32, the sites summed in FP64
struct OpDotNormF32 {
  static constexpr int NRED = 3;
  SpinorF32 a, b;
  RedScratch rs;
  FinStore fin;
  __device__ __forceinline__ void operator()(int h, double* red) const {
    float av[24], bv[24];
    a.load(h, av);
    b.load(h, bv);
    float re = 0.f, im = 0.f, nn = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re += av[2 * k] * bv[2 * k];
      re += av[2 * k + 1] * bv[2 * k + 1];
      im += av[2 * k] * bv[2 * k + 1];
      im -= av[2 * k + 1] * bv[2 * k];
      nn += av[2 * k] * av[2 * k];
      nn += av[2 * k + 1] * av[2 * k + 1];
    }
    red[0] += (double)re;
    red[1] += (double)im;
    red[2] += (double)nn;
  }
};

// out = a - c b (complex c)
struct OpSubScaledF32 {
  static constexpr int NRED = 0;
  SpinorF32 out, a, b;
  float cr, ci;
  __device__ __forceinline__ void operator()(int h, double*) const {
    float av[24], bv[24];
    a.load(h, av);
    b.load(h, bv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float br = bv[2 * k], bi = bv[2 * k + 1];
      av[2 * k] -= cr * br;
      av[2 * k] += ci * bi;
      av[2 * k + 1] -= cr * bi;
      av[2 * k + 1] -= ci * br;
    }
    out.store_f(h, av);
  }
};

// out = a x + b y (real a, b), FP64 fields
struct OpAxpbyF64 {
  static constexpr int NRED = 0;
  SpinorF64 out, x, y;
  double a, b;
  __device__ __forceinline__ void operator()(int h, double*) const {
    double xv[24], yv[24];
    x.load(h, xv);
    y.load(h, yv);
#pragma unroll
    for (int k = 0; k < 24; ++k) xv[k] = a * xv[k] + b * yv[k];
    out.store(h, xv);
  }
};

// Per-shift coefficients of one iteration (complex, as float2):
// x_k += ax p_k + as s;  p_k = c1 r_new + c2 p_k + c3 r + c4 s.
struct ShiftCoef {
  float2 ax, as, c1, c2, c3, c4;
  int active;
  int pad;
};
struct ShiftCoefs {
  ShiftCoef k[kMaxShifts];
};

// y += c x for the two complex numbers of a float4
__device__ __forceinline__ void cmad4(float4& y, float2 c, float4 x) {
  y.x += c.x * x.x;
  y.x -= c.y * x.y;
  y.y += c.x * x.y;
  y.y += c.y * x.x;
  y.z += c.x * x.z;
  y.z -= c.y * x.w;
  y.w += c.x * x.w;
  y.w += c.y * x.z;
}

// Device state of one shifted-family BiCGstab: the seed's scalars, the
// shifted recurrences (Jegerlehner's f, g and the product pi of the
// (1 + omega tau) factors), and the per-shift update coefficients the
// finaliser of each iteration writes for the fused update kernel.
struct MsCtl {
  double2 rho, alpha, omega;
  double stop;       // tol_rel |source|
  int iters, max_iter, done, failed, status, n, in_graph, loops;
  unsigned long long h_loop;
  double tau[kMaxShifts];
  double2 fz[kMaxShifts], gz[kMaxShifts], pz[kMaxShifts];
  int active[kMaxShifts];
  ShiftCoefs cf;
};

__device__ __forceinline__ double2 c_conj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_scale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double c_abs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ float2 c_f2(double2 z) { return make_float2((float)z.x, (float)z.y); }
__device__ __forceinline__ void ms_fail(MsCtl* m, int status) {
  if (!m->failed) m->status = status;
  m->failed = 1;
  m->done = 1;
}

// setup: rho = <r_tilde, r> (t = {<r, r_tilde>, |r|^2}), the stop
struct FinMsSetup {
  MsCtl* m;
  double tol_rel;
  __device__ void operator()(const double* t) const {
    m->rho = c_conj(make_double2(t[0], t[1]));
    if (!isfinite(t[2]) || !cfinite(m->rho)) ms_fail(m, WD_ERR_NUMERIC);
    m->stop = tol_rel * sqrt(t[2]);
  }
};

// alpha = rho / <r_tilde, v>  (t = {<v, r_tilde>, |v|^2})
struct FinMsAlpha {
  MsCtl* m;
  __device__ void operator()(const double* t) const {
    if (m->failed) return;
    const double2 rtv = c_conj(make_double2(t[0], t[1]));
    if (!cfinite(rtv)) { ms_fail(m, WD_ERR_NUMERIC); return; }
    if (c_abs(rtv) == 0.0 || c_abs(m->rho) == 0.0) { ms_fail(m, WD_ERR_BREAKDOWN); return; }
    m->alpha = cdiv(m->rho, rtv);
  }
};

// omega = <t, s> / <t, t>  (t = {<t, s>, |t|^2})
struct FinMsOmega {
  MsCtl* m;
  __device__ void operator()(const double* t) const {
    if (m->failed) return;
    const double2 ts = make_double2(t[0], t[1]);
    const double tt = t[2];
    if (!cfinite(ts) || !isfinite(tt)) { ms_fail(m, WD_ERR_NUMERIC); return; }
    if (tt == 0.0) { ms_fail(m, WD_ERR_BREAKDOWN); return; }
    m->omega = c_scale(1.0 / tt, ts);
    if (c_abs(m->omega) == 0.0) ms_fail(m, WD_ERR_BREAKDOWN);
  }
};

// end of iteration (t = {<r_new, r_tilde>, |r_new|^2}): beta, the shifted
// recurrences and update coefficients of every active shift, retirement of
// converged shifts, the stop test of the seed
struct FinMsIter {
  MsCtl* m;
  __device__ void operator()(const double* t) const {
    if (m->failed) return;
    m->iters += 1;
    const double2 rho_new = c_conj(make_double2(t[0], t[1]));
    const double rn = sqrt(t[2]);
    if (!isfinite(rn) || !cfinite(rho_new)) { ms_fail(m, WD_ERR_NUMERIC); return; }
    const double2 alpha = m->alpha, omega = m->omega;
    const double2 beta = cmul(cdiv(alpha, omega), cdiv(rho_new, m->rho));
    for (int k = 0; k < m->n; ++k) {
      ShiftCoef q{};
      if (m->active[k]) {
        const double sg = m->tau[k];
        const double2 fz = m->fz[k], gz = m->gz[k], pz = m->pz[k];
        const double2 f_next = c_add(fz, cmul(c_scale(sg, alpha), gz));
        const double2 alpha_s = cdiv(cmul(alpha, fz), f_next);
        const double2 one_ws = c_add(make_double2(1.0, 0.0), c_scale(sg, omega));
        const double2 omega_s = cdiv(omega, one_ws);
        const double2 pi_next = cmul(pz, one_ws);
        const double2 ratio = cdiv(fz, f_next);
        const double2 beta_s = cmul(beta, cmul(ratio, ratio));
        const double2 qq = cdiv(cmul(beta_s, omega_s), alpha_s);
        const double2 pf = cmul(pz, f_next);
        q.ax = c_f2(alpha_s);
        q.as = c_f2(cdiv(omega_s, pf));
        q.c1 = c_f2(cdiv(make_double2(1.0, 0.0), cmul(pi_next, f_next)));
        q.c2 = c_f2(beta_s);
        q.c3 = c_f2(cdiv(c_scale(-1.0, qq), cmul(pz, fz)));
        q.c4 = c_f2(cdiv(qq, pf));
        q.active = 1;
        m->gz[k] = c_add(f_next, cmul(beta, gz));
        m->fz[k] = f_next;
        m->pz[k] = pi_next;
      }
      m->cf.k[k] = q;
    }
    // the seed (k = 0) drives the iteration and stays active
    for (int k = 1; k < m->n; ++k)
      if (m->active[k] && rn <= m->stop * c_abs(cmul(m->pz[k], m->fz[k]))) m->active[k] = 0;
    m->rho = rho_new;
    if (rn <= m->stop || m->iters >= m->max_iter) m->done = 1;
  }
};

// (<a, b>, |a|^2) with the finaliser Fin
template <class Fin>
struct OpDotNormMs {
  static constexpr int NRED = 3;
  OpDotNormF32 d;
  Fin fin;
  RedScratch rs;
  __device__ __forceinline__ void operator()(int h, double* red) const { d(h, red); }
};

// out = a - c b with c read from the control block (alpha or omega)
struct OpSubScaledMs {
  static constexpr int NRED = 0;
  SpinorF32 out, a, b;
  const double2* c;
  const MsCtl* m;
  __device__ __forceinline__ void operator()(int h, double*) const {
    if (m->failed) return;
    OpSubScaledF32{out, a, b, (float)c->x, (float)c->y}(h, nullptr);
  }
};

// All shifts in one pass: per site and float4 chunk of the spinor the seed's
// r, r_new and s are read once and every active shift's x_k, p_k updated
// (fields of the shifts rs bytes apart), with the coefficients the
// finaliser wrote; then r <- r_new for the next iteration.
__global__ void __launch_bounds__(kBlasBlock) shift_update_kernel(int n, SpinorF32 xs, SpinorF32 ps, SpinorF32 r,
                                                                  SpinorF32 r_new, SpinorF32 s, const MsCtl* m) {
  if (m->failed) return;
  const int nshift = m->n;
  const int stride = r.stride;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
#pragma unroll 1
    for (int c = 0; c < 6; ++c) {
      const size_t o = (size_t)c * stride + h;
      const float4 rv = __ldg(r.p + o), nv = __ldg(r_new.p + o), sv = __ldg(s.p + o);
      for (int k = 0; k < nshift; ++k) {
        const ShiftCoef q = m->cf.k[k];
        if (!q.active) continue;
        float4* xk = (float4*)((char*)xs.p + (size_t)k * xs.rs) + o;
        float4* pk = (float4*)((char*)ps.p + (size_t)k * ps.rs) + o;
        const float4 pv = *pk;
        float4 xv = *xk;
        cmad4(xv, q.ax, pv);
        cmad4(xv, q.as, sv);
        *xk = xv;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        cmad4(t, q.c2, pv);
        cmad4(t, q.c4, sv);
        cmad4(t, q.c3, rv);
        cmad4(t, q.c1, nv);
        *pk = t;
      }
      r.p[o] = nv;
    }
  }
}

// last node of the WHILE body: continue while not done; the body count is
// bounded here on its own (max_iter + 16 executions)
__global__ void ms_loop_control_kernel(MsCtl* m) {
  m->loops += 1;
  if (m->loops > m->max_iter + 16 && !m->done) ms_fail(m, WD_ERR_NOT_CONVERGED);
  if (m->in_graph) cudaGraphSetConditional((cudaGraphConditionalHandle)m->h_loop, m->done ? 0u : 1u);
}

// one block: the control block is zeroed word by word in place (a local
// copy of it would live on the stack), then its fields are set
__global__ void ms_init_kernel(MsCtl* m, int n, const double* tau, int max_iter, unsigned long long h_loop) {
  static_assert(sizeof(MsCtl) % sizeof(unsigned) == 0, "MsCtl is a whole number of words");
  unsigned* w = reinterpret_cast<unsigned*>(m);
  for (int i = threadIdx.x; i < (int)(sizeof(MsCtl) / sizeof(unsigned)); i += blockDim.x) w[i] = 0u;
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    m->tau[k] = tau[k];
    m->fz[k] = m->gz[k] = m->pz[k] = make_double2(1.0, 0.0);
    m->active[k] = 1;
  }
  if (threadIdx.x == 0) {
    m->n = n;
    m->max_iter = max_iter;
    m->status = WD_OK;
    m->in_graph = 1;
    m->h_loop = h_loop;
  }
}

float2 f2(cplx z) { return make_float2((float)z.real(), (float)z.imag()); }

}  // namespace

namespace {

// FP32 work fields of one shifted family (even parity)
struct Family {
  void *r, *rt, *s, *t, *v, *rn;
  void* todd;  // odd FP32 temporary of M_hat
  void* xs;  // n solutions, fb apart
  void* ps;  // n directions, fb apart
};

// BiCGstab over the shifted family (B + tau_k) y_k = src, B = M_hat(kappa_s),
// tau_0 = 0 (the seed), run on the device: every scalar of the iteration
// lives in the control block m, written by the finalisers of the fused
// reductions, and the loop is one CUDA graph (a WHILE node over the
// iteration), so the host waits once per family instead of three times per
// iteration.  Returns when the seed's iterated residual reaches
// tol_rel |src| (the shifted systems, whose residuals are the seed's divided
// by |pi_k f_k| >= 1 in practice, stop being updated once they reach it).
wd_status family_solve(wd_ctx* ctx, const void* src, double kappa_s, const std::vector<double>& tau, int max_iter,
                       double tol_rel, Family& f, size_t fb, MsCtl* m, double* tau_dev, int& iters,
                       long long& launches) {
  Ctx& c = ctx->c;
  cudaStream_t st = c.stream;
  const Geom& g = c.g;
  const int n = (int)tau.size();
  const PrecOps* o32 = prec_ops(WD_F32);
  auto V = [&](const void* p, size_t rs = 0) { return Tr<WD_F32>::view(p, g, rs); };
  double* hp = c.host_pinned;
  MS_CK(cudaMemcpyAsync(f.r, src, fb, cudaMemcpyDeviceToDevice, st));
  MS_CK(cudaMemcpyAsync(f.rt, src, fb, cudaMemcpyDeviceToDevice, st));
  for (int k = 0; k < n; ++k) MS_CK(cudaMemcpyAsync((char*)f.ps + k * fb, src, fb, cudaMemcpyDeviceToDevice, st));
  MS_CK(cudaMemsetAsync(f.xs, 0, n * fb, st));
  MS_CK(cudaMemcpyAsync(tau_dev, tau.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));

  // the loop as a graph: WHILE(!done) { iteration; loop control }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct GraphGuard {
    cudaGraph_t& g;
    cudaGraphExec_t& e;
    ~GraphGuard() {
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
    }
  } guard{graph, exec};
  MS_CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle hl;
  MS_CK(cudaGraphConditionalHandleCreate(&hl, graph, 1, cudaGraphCondAssignDefault));
  ms_init_kernel<<<1, 128, 0, st>>>(m, n, tau_dev, max_iter, (unsigned long long)hl);
  launch_sites(c, g.Vh, OpDotNormMs<FinMsSetup>{OpDotNormF32{V(f.r), V(f.rt), c.red, FinStore{nullptr, 0}},
                                                FinMsSetup{m, tol_rel}, c.red},
               st);
  launches += 2;
  // a zero source needs no iteration (y = 0); a non-finite one is refused
  MS_CK(cudaMemcpyAsync(hp + 16, &m->stop, sizeof(double), cudaMemcpyDeviceToHost, st));
  MS_CK(cudaMemcpyAsync(hp + 17, &m->failed, sizeof(int), cudaMemcpyDeviceToHost, st));
  MS_CK(cudaStreamSynchronize(st));
  iters = 0;
  int failed0 = 0;
  memcpy(&failed0, hp + 17, sizeof(int));
  if (failed0) return merr(ctx, WD_ERR_NUMERIC, "multi-shift: source not finite");
  if (hp[16] == 0.0) return WD_OK;

  union Raw {  // zero-initialised node parameters (the type has no default constructor)
    cudaGraphNodeParams p;
    unsigned char bytes[sizeof(cudaGraphNodeParams)];
    Raw() { memset(bytes, 0, sizeof(bytes)); }
  } raw;
  cudaGraphNodeParams& wp = raw.p;
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hl;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  MS_CK(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaStream_t cs;
  MS_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t unused;
  MS_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  {
    const int gx = std::min((g.Vh + kBlasBlock - 1) / kBlasBlock, c.num_sms * 8);
    auto apply_B = [&](void* out, const void* in) {  // out = M_hat(kappa_s) in
      o32->dslash(c, f.todd, in, 1, 0, cs);
      o32->dslash_xpay(c, out, f.todd, in, -kappa_s * kappa_s, nullptr, 0, 0, cs);
    };
    apply_B(f.v, f.ps);  // v = B p_0
    launch_sites(c, g.Vh, OpDotNormMs<FinMsAlpha>{OpDotNormF32{V(f.v), V(f.rt), c.red, FinStore{nullptr, 0}},
                                                  FinMsAlpha{m}, c.red},
                 cs);
    launch_sites(c, g.Vh, OpSubScaledMs{V(f.s), V(f.r), V(f.v), &m->alpha, m}, cs);  // s = r - alpha v
    apply_B(f.t, f.s);                                                              // t = B s
    launch_sites(c, g.Vh, OpDotNormMs<FinMsOmega>{OpDotNormF32{V(f.t), V(f.s), c.red, FinStore{nullptr, 0}},
                                                  FinMsOmega{m}, c.red},
                 cs);
    launch_sites(c, g.Vh, OpSubScaledMs{V(f.rn), V(f.s), V(f.t), &m->omega, m}, cs);  // r_new = s - omega t
    launch_sites(c, g.Vh, OpDotNormMs<FinMsIter>{OpDotNormF32{V(f.rn), V(f.rt), c.red, FinStore{nullptr, 0}},
                                                 FinMsIter{m}, c.red},
                 cs);
    shift_update_kernel<<<gx, kBlasBlock, 0, cs>>>(g.Vh, V(f.xs, fb), V(f.ps, fb), V(f.r), V(f.rn), V(f.s), m);
    ms_loop_control_kernel<<<1, 1, 0, cs>>>(m);
  }
  const cudaError_t ce = cudaStreamEndCapture(cs, &unused);
  cudaStreamDestroy(cs);
  MS_CK(ce);
  MS_CK(cudaGraphInstantiate(&exec, graph, 0));
  MS_CK(cudaGraphLaunch(exec, st));
  MsCtl hm;
  MS_CK(cudaMemcpyAsync(&hm, m, sizeof(MsCtl), cudaMemcpyDeviceToHost, st));
  MS_CK(cudaStreamSynchronize(st));
  iters = hm.iters;
  launches += (long long)hm.loops * 11;
  if (hm.failed) {
    const char* what = hm.status == WD_ERR_BREAKDOWN ? "multi-shift: breakdown" : "multi-shift: NaN/Inf";
    return merr(ctx, (wd_status)(hm.status ? hm.status : WD_ERR_NUMERIC), what);
  }
  return WD_OK;
}

struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

}  // namespace

namespace {

// x: n FP64 full fields (even, odd) back to back; b: one FP64 full field;
// both device memory in the internal layout
wd_status multishift_core(wd_ctx* ctx, int n, char* x, const char* b, const double* kappas,
                          const wd_solve_params* params, wd_solve_info* infos) {
  for (int k = 0; k < n; ++k)
    if (!(kappas[k] > 0.0) || !std::isfinite(kappas[k]) || !(params->tol > 0.0) || params->max_iter < 1)
      return merr(ctx, WD_ERR_INVALID_ARG, "wd_solve_multishift: bad kappa, tol or max_iter");
  Ctx& c = ctx->c;
  if (!c.gauge_loaded) return merr(ctx, WD_ERR_INVALID_ARG, "wd_solve_multishift: no gauge field loaded");
  MS_ST(wd_internal_ensure_gauge(ctx, WD_F64));
  MS_ST(wd_internal_ensure_gauge(ctx, WD_F32));
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = c.stream;
  const Geom& g = c.g;
  const size_t f64 = Tr<WD_F64>::bytes(g.stride), f32 = Tr<WD_F32>::bytes(g.stride);
  DevBuf mem;
  mem.s = st;
  const size_t bytes64 = f64, bytes32 = (size_t)(8 + 3 * n) * f32;
  const size_t bytes_ctl = align256(sizeof(MsCtl)) + align256(kMaxShifts * sizeof(double));
  MS_CK(cudaMallocAsync(&mem.p, bytes_ctl + bytes64 + bytes32, st));
  char* q = (char*)mem.p;
  MsCtl* mctl = (MsCtl*)q;  q += align256(sizeof(MsCtl));
  double* tau_dev = (double*)q; q += align256(kMaxShifts * sizeof(double));
  char* w64 = q;    q += f64;       // D_eo b_o, and a conversion scratch
  Family fam{};
  fam.r = q;  q += f32;
  fam.rt = q; q += f32;
  fam.s = q;  q += f32;
  fam.t = q;  q += f32;
  fam.v = q;  q += f32;
  fam.rn = q; q += f32;
  fam.todd = q; q += f32;
  char* src32 = q; q += f32;
  char* ys = q; q += n * f32;
  char* zs = q; q += n * f32;
  fam.ps = q;
  auto V64 = [&](const void* p) { return Tr<WD_F64>::view(p, g); };
  long long launches = 0;
  const PrecOps* o64 = ops_f64();
  const PrecOps* o32 = prec_ops(WD_F32);
  double* hp = c.host_pinned;
  const char* b_e = b;
  const char* b_o = b + f64;
  o64->norm2(c, c.scalars + 20, b_e, st);
  o64->norm2(c, c.scalars + 21, b_o, st);
  launches += 2;
  MS_CK(cudaMemcpyAsync(hp + 20, c.scalars + 20, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  MS_CK(cudaStreamSynchronize(st));
  const double be2 = hp[20], bo2 = hp[21], b2 = be2 + bo2;
  if (!std::isfinite(b2)) return merr(ctx, WD_ERR_NUMERIC, "wd_solve_multishift: source not finite");
  // seed first: the largest kappa is the slowest system
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int bb) { return kappas[a] > kappas[bb]; });
  const double ks = kappas[order[0]];
  std::vector<double> tau(n);
  for (int i = 0; i < n; ++i) tau[i] = (ks / kappas[order[i]]) * (ks / kappas[order[i]]) - 1.0;
  const double stage_tol = std::max(params->tol, kStageTol);
  int it_u = 0, it_w = 0;
  if (be2 > 0.0) {
    o32->from_f64(c, src32, b_e, st);
    fam.xs = ys;
    MS_ST(family_solve(ctx, src32, ks, tau, params->max_iter, stage_tol, fam, f32, mctl, tau_dev, it_u, launches));
  } else {
    MS_CK(cudaMemsetAsync(ys, 0, n * f32, st));
  }
  if (bo2 > 0.0) {
    o64->dslash(c, w64, b_o, 0, 0, st);  // w = D_eo b_o
    o32->from_f64(c, src32, w64, st);
    launches += 2;
    fam.xs = zs;
    MS_ST(family_solve(ctx, src32, ks, tau, params->max_iter, stage_tol, fam, f32, mctl, tau_dev, it_w, launches));
  }
  const int ms_iters = it_u + it_w;
  wd_status worst = WD_OK;
  for (int i = 0; i < n; ++i) {
    const int k = order[i];
    const double kap = kappas[k], sc = (ks / kap) * (ks / kap);
    char* xfull = x + (size_t)k * 2 * f64;
    char* xe = xfull;
    // x_e = (kappa_s / kappa)^2 (y + kappa z) (Sec. 3)
    o32->to_f64(c, xe, ys + (size_t)i * f32, st);
    if (bo2 > 0.0) {
      o32->to_f64(c, w64, zs + (size_t)i * f32, st);
      launch_sites(c, g.Vh, OpAxpbyF64{V64(xe), V64(xe), V64(w64), sc, sc * kap}, st);
      launches += 3;
    } else {
      launch_sites(c, g.Vh, OpAxpbyF64{V64(xe), V64(xe), V64(xe), sc, 0.0}, st);
      launches += 2;
    }
    // the reliable-update BiCGstab finishes the system from x_e (its first
    // residual b_hat - M_hat x_e in FP64); it rebuilds x_o and reports the
    // full FP64 true residual of the returned x (S13)
    wd_solve_params p2 = *params;
    p2.solver = WD_BICGSTAB;
    p2.restart = 0;
    p2.initial_guess = 0;  // the start is x_e itself (wd_internal_solve_x0)
    wd_solve_info ie{};
    const wd_status se = wd_internal_solve_x0(ctx, xfull, b, kap, &p2, &ie);
    if (se != WD_OK && se != WD_ERR_NOT_CONVERGED) return se;
    launches += ie.kernel_launches;
    const double rel = ie.true_rel_residual;
    const wd_status sk = !std::isfinite(rel) ? WD_ERR_NUMERIC : (rel <= params->tol ? WD_OK : WD_ERR_NOT_CONVERGED);
    if (sk != WD_OK && worst == WD_OK) worst = sk;
    wd_solve_info& inf = infos[k];
    inf.iters = ms_iters + ie.iters;
    inf.reliable_updates = ie.reliable_updates;
    inf.true_rel_residual = rel;
    inf.iterated_rel_residual = ie.iterated_rel_residual;
    inf.status = sk;
  }
  MS_CK(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int k = 0; k < n; ++k) {
    infos[k].seconds = secs;
    infos[k].kernel_launches = launches;
  }
  if (worst != WD_OK) return merr(ctx, worst, "wd_solve_multishift: some kappa did not reach tol");
  return WD_OK;
}

}  // namespace

extern "C" wd_status wd_solve_multishift_device(wd_ctx* ctx, int n, void* x, const void* b, const double* kappas,
                                                const wd_solve_params* params, wd_solve_info* infos) {
  if (!ctx || n < 1 || n > kMaxShifts || !x || !b || !kappas || !params || !infos)
    return ctx ? merr(ctx, WD_ERR_INVALID_ARG, "wd_solve_multishift_device: bad args") : WD_ERR_INVALID_ARG;
  MS_CK(cudaSetDevice(ctx->c.device));
  return multishift_core(ctx, n, (char*)x, (const char*)b, kappas, params, infos);
}

extern "C" wd_status wd_solve_multishift(wd_ctx* ctx, int n, double* const* x, const double* b,
                                         const double* kappas, const wd_solve_params* params,
                                         wd_solve_info* infos) {
  if (!ctx || n < 1 || n > kMaxShifts || !x || !b || !kappas || !params || !infos)
    return ctx ? merr(ctx, WD_ERR_INVALID_ARG, "wd_solve_multishift: bad args") : WD_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k)
    if (!x[k]) return merr(ctx, WD_ERR_INVALID_ARG, "wd_solve_multishift: bad x");
  Ctx& c = ctx->c;
  MS_CK(cudaSetDevice(c.device));
  if (!c.gauge_loaded) return merr(ctx, WD_ERR_INVALID_ARG, "wd_solve_multishift: no gauge field loaded");
  const size_t f64 = Tr<WD_F64>::bytes(c.g.stride);
  DevBuf mem;
  mem.s = c.stream;
  MS_CK(cudaMallocAsync(&mem.p, (size_t)(n + 1) * 2 * f64, c.stream));
  char* bdev = (char*)mem.p;
  char* xdev = bdev + 2 * f64;
  MS_ST(wd_internal_import_full(ctx, bdev, bdev + f64, b));
  const wd_status st = multishift_core(ctx, n, xdev, bdev, kappas, params, infos);
  if (st != WD_OK && st != WD_ERR_NOT_CONVERGED) return st;
  for (int k = 0; k < n; ++k) MS_ST(wd_internal_export_full(ctx, x[k], xdev + (size_t)k * 2 * f64,
                                                            xdev + (size_t)k * 2 * f64 + f64));
  return st;
}
