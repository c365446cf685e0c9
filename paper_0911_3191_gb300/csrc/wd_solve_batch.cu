// Batched solves and the multi-RHS dslash entry points (C ABI).
//
// wd_solve_batch_device solves M_kappa_r x_r = b_r for n systems that share
// the gauge field, each with its own kappa (Sec. 3: many source vectors b; the
// 12 spin-colour sources of a propagator times several masses).  All systems
// run the reliable-update BiCGstab of Sec. 5.1/5.3 in lockstep: one
// multi-RHS dslash launch per stencil application, one SolverCtl per system,
// converged systems masked out, reliable updates only for the systems that
// asked.  The whole loop is one CUDA graph (WHILE over the iteration, IF over
// "some system needs a reliable update").  The multi-RHS dslash shape (RHS
// tile, grid) is chosen by timing candidates on first use (autotuner), cached
// per (lattice, precision, n) in the context and optionally in the file named
// by the WD_TUNE_CACHE environment variable.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "wd_batch.cuh"

using namespace wd;

namespace {

wd_status berr(wd_ctx* ctx, wd_status st, const std::string& msg) {
  if (ctx) ctx->c.last_error = msg;
  return st;
}

wd_status bcuda(wd_ctx* ctx, cudaError_t e, const char* what) {
  return berr(ctx, e == cudaErrorMemoryAllocation ? WD_ERR_OOM : WD_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define WB_CK(ctx, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return bcuda(ctx, e_, #call);   \
  } while (0)
#define WB_CK_LAUNCH(ctx) WB_CK(ctx, (cudaPeekAtLastError(), cudaGetLastError()))

constexpr int kMaxBatch = 256;

size_t fbytes(const Ctx& c, int prec) { return prec_ops(prec)->field_bytes(c.g.stride); }

void destroy_batch_graph(Ctx& c) {
  if (c.batch_exec) cudaGraphExecDestroy(c.batch_exec);
  if (c.batch_graph) cudaGraphDestroy(c.batch_graph);
  c.batch_exec = nullptr;
  c.batch_graph = nullptr;
}

int blas_gx(const Ctx& c, int n) {
  const int per_rhs = (c.num_sms * 8 + n - 1) / n;
  const int need = (c.g.Vh + kBlasBlock - 1) / kBlasBlock;
  return per_rhs < need ? (per_rhs > 0 ? per_rhs : 1) : need;
}

// Layout of the small allocation: ctl[n] | BatchCtl | partials | kappas[2n] | scal[4n]
struct SmallLayout {
  size_t ctl, bc, partials, kappas, scal, total;
};
SmallLayout small_layout(const Ctx& c, int n) {
  SmallLayout L;
  const int maxblk = c.num_sms * 16 > blas_gx(c, n) ? c.num_sms * 16 : blas_gx(c, n);
  L.ctl = 0;
  L.bc = align256(L.ctl + (size_t)n * sizeof(SolverCtl));
  L.partials = align256(L.bc + sizeof(BatchCtl));
  L.kappas = align256(L.partials + (size_t)maxblk * n * 4 * sizeof(double));
  L.scal = align256(L.kappas + (size_t)2 * n * sizeof(double));
  L.total = align256(L.scal + (size_t)4 * n * sizeof(double));
  return L;
}

BatchBufs batch_views(Ctx& c, int n, int prec) {
  BatchBufs b{};
  const SmallLayout L = small_layout(c, n);
  char* s = (char*)c.batch_small;
  b.ctl = (SolverCtl*)(s + L.ctl);
  b.bc = (BatchCtl*)(s + L.bc);
  b.partials = (double*)(s + L.partials);
  b.kappas = (double*)(s + L.kappas);
  b.scal = (double*)(s + L.scal);
  const size_t f64 = fbytes(c, WD_F64) * n, fin = fbytes(c, prec) * n;
  char* p = (char*)c.batch_block;
  b.b_hat = p; p += f64;
  b.xe = p; p += f64;
  b.tmp64 = p; p += f64;
  b.r_hat = p; p += fin;
  b.r_tilde = p; p += fin;
  b.p = p; p += fin;
  b.v = p; p += fin;
  b.t = p; p += fin;
  b.x_hat = p; p += fin;
  b.tmp = p; p += fin;
  return b;
}

wd_status ensure_batch(wd_ctx* ctx, int n, int prec) {
  Ctx& c = ctx->c;
  if (c.batch_block && c.batch_n == n && c.batch_prec == prec) return WD_OK;
  batch_release(c);
  const size_t need = 3 * fbytes(c, WD_F64) * n + 7 * fbytes(c, prec) * n;
  cudaError_t e = cudaMalloc(&c.batch_block, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.batch_block = nullptr;
    return bcuda(ctx, e, "batch workspace");
  }
  const SmallLayout L = small_layout(c, n);
  e = cudaMalloc(&c.batch_small, L.total);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.batch_small, 0, L.total, c.stream);  // ordered with the solve
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c.batch_host, (size_t)n * sizeof(SolverCtl) + 4 * n * 8 + 64);
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_release(c);
    return bcuda(ctx, e, "batch control");
  }
  c.batch_bytes = need;
  c.batch_n = n;
  c.batch_prec = prec;
  c.batch_tr = 0;
  c.batch_pack = 0;
  return WD_OK;
}

std::string tune_key(const Ctx& c, int n, int prec) {
  std::ostringstream k;
  // the link format and the temporal gauge change the cost of the multi-RHS
  // dslash, so a shape tuned for one is not reused for the other
  k << c.g.X << "x" << c.g.Y << "x" << c.g.Z << "x" << c.g.T << " prec" << prec << " n" << n << " sms" << c.num_sms
    << " links" << c.low_recon << " tfix" << c.g.tfix;
  return k.str();
}

// Autotuner: time the multi-RHS inner-precision dslash for every (RHS tile,
// grid) candidate on the batch's own fields and keep the fastest.
wd_status tune_batch(wd_ctx* ctx, int n, int prec, BatchBufs& b) {
  Ctx& c = ctx->c;
  if (c.batch_tr) return WD_OK;
  const std::string key = tune_key(c, n, prec);
  const char* cache = std::getenv("WD_TUNE_CACHE");
  if (cache) {
    std::ifstream f(cache);
    std::string line;
    while (std::getline(f, line)) {
      const size_t bar = line.find('|');
      if (bar != std::string::npos && line.substr(0, bar) == key) {
        std::istringstream v(line.substr(bar + 1));
        int tr = 0, grid = 0, pack = 0;
        const bool shape = static_cast<bool>(v >> tr >> grid);
        if (shape && !(v >> pack)) pack = 0;  // entries without the layout field: one system per thread
        if (shape && (tr == 0 || tr == 1 || tr == 2 || tr == 4 || tr == 8) && grid > 0 &&
            (pack == 0 || (pack == 1 && tr >= 2 && prec != WD_F64))) {
          c.batch_tr = tr ? tr : -1;
          c.batch_grid = grid;
          c.batch_pack = pack;
          return WD_OK;
        }
      }
    }
  }
  const PrecOps* o = prec_ops(prec);
  const int ntiles = (c.g.Vh + 31) / 32;
  BatchLaunch bl{n, 1, 1, blas_gx(c, n)};
  // defined (zero) inputs for the timing runs
  WB_CK(ctx, cudaMemsetAsync(b.r_hat, 0, fbytes(c, prec) * n, c.stream));
  cudaEvent_t e0, e1;
  WB_CK(ctx, cudaEventCreate(&e0));
  WB_CK(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_tr = 4, best_grid = c.num_sms * 4, best_pack = 0;
  // block shapes and register layouts: tr 0 is one system per block row (128
  // sites per block); tr 1..8 systems per 32-site link tile, one system per
  // thread, or (pack) two systems per thread in FP32x2 registers, tr / 2
  // thread rows
  const int trs[8] = {0, 1, 2, 4, 8, 2, 4, 8};
  const int packs[8] = {0, 0, 0, 0, 0, 1, 1, 1};
  const int ncand = prec == WD_F64 ? 5 : 8;
  const int mults[4] = {2, 4, 8, 16};
  const int nblk128 = (c.g.Vh + kDslashBlock - 1) / kDslashBlock;
  for (int ti = 0; ti < ncand; ++ti) {
    for (int mi = 0; mi < 4; ++mi) {
      int grid = c.num_sms * mults[mi];
      const int cap = trs[ti] ? ntiles : nblk128;
      if (grid > cap) grid = cap;
      bl.tr = trs[ti];
      bl.pack = packs[ti];
      bl.grid = grid;
      o->dslash_batch(c, bl, b.tmp, b.r_hat, 1, 0, c.stream);  // warm-up
      WB_CK(ctx, cudaEventRecord(e0, c.stream));
      for (int rep = 0; rep < 3; ++rep) o->dslash_batch(c, bl, b.tmp, b.r_hat, 1, 0, c.stream);
      WB_CK(ctx, cudaEventRecord(e1, c.stream));
      WB_CK(ctx, cudaEventSynchronize(e1));
      float ms = 0.f;
      WB_CK(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_tr = trs[ti];
        best_grid = grid;
        best_pack = packs[ti];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  WB_CK_LAUNCH(ctx);
  c.batch_tr = best_tr ? best_tr : -1;
  c.batch_grid = best_grid;
  c.batch_pack = best_pack;
  if (cache) {
    std::ofstream f(cache, std::ios::app);
    f << key << "|" << best_tr << " " << best_grid << " " << best_pack << "\n";
  }
  return WD_OK;
}

BatchLaunch launch_shape(const Ctx& c, int n) {
  const int ntiles = (c.g.Vh + 31) / 32;
  BatchLaunch bl{n, c.batch_tr ? std::max(c.batch_tr, 0) : 4, c.batch_tr ? c.batch_grid : c.num_sms * 4,
                 blas_gx(c, n)};
  if (bl.tr && bl.grid > ntiles) bl.grid = ntiles;
  bl.grid64 = rhs_grid64(c.g, c.num_sms);
  bl.pack = (c.batch_tr > 0) ? c.batch_pack : 0;
  return bl;
}

wd_status build_batch_graph(wd_ctx* ctx, int prec, BatchBufs& b, const BatchLaunch& bl) {
  Ctx& c = ctx->c;
  cudaError_t e = build_batch_loop_graph(c, prec, b, bl, &c.batch_graph, &c.batch_exec, &c.batch_hu, &c.batch_hl);
  if (e != cudaSuccess) return bcuda(ctx, e, "batched solver graph");
  return WD_OK;
}

// x, b: n FP64 full fields (even then odd) back to back, internal layout
wd_status solve_batch_device(wd_ctx* ctx, int n, void* x, const void* bsrc, const double* kappas,
                             const wd_solve_params* prm, wd_solve_info* infos) {
  Ctx& c = ctx->c;
  const auto t0 = std::chrono::steady_clock::now();
  wd_solve_params p{1e-10, 0.1, 10000, WD_BICGSTAB, WD_Q16, 1, 0, 0};
  if (prm) p = *prm;
  if (n < 1 || n > kMaxBatch) return berr(ctx, WD_ERR_INVALID_ARG, "batch size must be in [1, 256]");
  if (p.inner_precision < WD_F64 || p.inner_precision > WD_B16N)
    return berr(ctx, WD_ERR_INVALID_ARG, "bad inner_precision");
  if (p.solver != WD_BICGSTAB) return berr(ctx, WD_ERR_INVALID_ARG, "batched solves use BiCGstab");
  if (p.restart) return berr(ctx, WD_ERR_INVALID_ARG, "batched solves use reliable updates (restart = 0)");
  if (p.initial_guess) return berr(ctx, WD_ERR_INVALID_ARG, "batched solves start from zero (initial_guess = 0)");
  if (!(p.tol > 0.0) || p.max_iter <= 0) return berr(ctx, WD_ERR_INVALID_ARG, "bad tol or max_iter");
  if (p.inner_precision == WD_F64) p.delta = 0.0;
  else if (!(p.delta > 0.0 && p.delta < 1.0)) return berr(ctx, WD_ERR_INVALID_ARG, "delta must be in (0,1)");
  for (int r = 0; r < n; ++r)
    if (!std::isfinite(kappas[r])) return berr(ctx, WD_ERR_INVALID_ARG, "kappa must be finite");
  if (!c.gauge_loaded) return berr(ctx, WD_ERR_STATE, "no gauge field loaded");
  // the inner precision's gauge copy is derived from the FP64 copy on first use
  wd_status st = wd_internal_ensure_gauge(ctx, p.inner_precision);
  if (st != WD_OK) return st;
  st = ensure_batch(ctx, n, p.inner_precision);
  if (st != WD_OK) return st;
  BatchBufs b = batch_views(c, n, p.inner_precision);
  cudaStream_t s = c.stream;
  const Geom& g = c.g;
  const size_t f64 = fbytes(c, WD_F64);
  using T64 = Tr<WD_F64>;
  const SpinorF64 be = T64::view(bsrc, g, 2 * f64), bo = T64::view((const char*)bsrc + f64, g, 2 * f64);
  const SpinorF64 xe = T64::view(x, g, 2 * f64), xo = T64::view((char*)x + f64, g, 2 * f64);
  const SpinorF64 bhat = T64::view(b.b_hat, g, f64), xacc = T64::view(b.xe, g, f64);

  // kappa_r and -kappa_r for the epilogues
  std::vector<double> kk(2 * n);
  for (int r = 0; r < n; ++r) {
    kk[r] = kappas[r];
    kk[n + r] = -kappas[r];
  }
  WB_CK(ctx, cudaMemcpyAsync(b.kappas, kk.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice, s));
  WB_CK(ctx, cudaStreamSynchronize(s));

  if (!c.batch_tr) {
    if ((st = tune_batch(ctx, n, p.inner_precision, b)) != WD_OK) return st;
  }
  const BatchLaunch bl = launch_shape(c, n);
  const BatchArgs all{n, nullptr, 0, b.partials, nullptr};
  // |b_e|^2, |b_o|^2 per system
  launch_sites_batch(g, bl, OpNorm2<SpinorF64>{be, c.red, FinStore{b.scal, 1}}, all, s);
  launch_finalize<1>(bl, all, bl.blas_gx, FinStore{b.scal, 1}, b.bc, 0, 0, s);
  launch_sites_batch(g, bl, OpNorm2<SpinorF64>{bo, c.red, FinStore{b.scal + n, 1}}, all, s);
  launch_finalize<1>(bl, all, bl.blas_gx, FinStore{b.scal + n, 1}, b.bc, 0, 0, s);
  // b_hat_r = b_e,r + kappa_r D_eo b_o,r ; x accumulators zero
  EpiXpay<SpinorF64, SpinorF64> eb{bhat, be, Coef{0.0, b.kappas, 1}};
  launch_dslash_mrhs<double>(g, bl, bo, T64::gauge(c), 0, 0, eb, all, s);
  launch_sites_batch(g, bl, OpZero<SpinorF64>{xacc}, all, s);
  WB_CK_LAUNCH(ctx);

  const PrecOps* o = prec_ops(p.inner_precision);
  if (p.use_graph && !c.batch_exec) {
    if ((st = build_batch_graph(ctx, p.inner_precision, b, bl)) != WD_OK) return st;
  }
  batch_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(b.ctl, b.bc, n, p.tol, p.delta, p.max_iter, b.kappas, b.scal,
                                                    p.use_graph ? 1 : 0, p.use_graph ? c.batch_hu : 0,
                                                    p.use_graph ? c.batch_hl : 0);
  o->batch_setup(c, bl, b, s);
  WB_CK_LAUNCH(ctx);
  BatchCtl hb;
  if (p.use_graph) {
    WB_CK(ctx, cudaGraphLaunch(c.batch_exec, s));
  } else {
    for (int loop = 0; loop < p.max_iter + 16; ++loop) {
      o->batch_iteration(c, bl, b, s);
      WB_CK_LAUNCH(ctx);
      WB_CK(ctx, cudaMemcpyAsync(&hb, b.bc, sizeof(hb), cudaMemcpyDeviceToHost, s));
      WB_CK(ctx, cudaStreamSynchronize(s));
      if (hb.any_update) {
        o->batch_update(c, bl, b, s);
        WB_CK_LAUNCH(ctx);
      }
      batch_loop_control_kernel<<<1, 1, 0, s>>>(b.bc, b.ctl, n);
      WB_CK(ctx, cudaMemcpyAsync(&hb, b.bc, sizeof(hb), cudaMemcpyDeviceToHost, s));
      WB_CK(ctx, cudaStreamSynchronize(s));
      if (hb.all_done) break;
    }
  }
  // x_e,r from the accumulators; x_o,r = b_o,r + kappa_r D_oe x_e,r; the full
  // FP64 true residuals |b_r - M x_r|^2 (S13)
  launch_sites_batch(g, bl, OpConvert<SpinorF64, SpinorF64>{xe, xacc}, all, s);
  EpiXpay<SpinorF64, SpinorF64> ex{xo, bo, Coef{0.0, b.kappas, 1}};
  launch_dslash_mrhs<double>(g, bl, xe, T64::gauge(c), 1, 0, ex, all, s);
  const Coef nk{0.0, b.kappas + n, 1};
  EpiResid<SpinorF64, SpinorF64, SpinorF64, FinStore> re{xe, false, be, xe, nk, c.red, FinStore{b.scal + 2 * n, 1}};
  launch_dslash_mrhs<double>(g, bl, xo, T64::gauge(c), 0, 0, re, all, s);
  launch_finalize<1>(bl, all, mrhs_grid<double>(bl), FinStore{b.scal + 2 * n, 1}, b.bc, 0, 0, s);
  EpiResid<SpinorF64, SpinorF64, SpinorF64, FinStore> ro{xo, false, bo, xo, nk, c.red, FinStore{b.scal + 3 * n, 1}};
  launch_dslash_mrhs<double>(g, bl, xe, T64::gauge(c), 1, 0, ro, all, s);
  launch_finalize<1>(bl, all, mrhs_grid<double>(bl), FinStore{b.scal + 3 * n, 1}, b.bc, 0, 0, s);
  WB_CK_LAUNCH(ctx);
  SolverCtl* hc = (SolverCtl*)c.batch_host;
  double* hs = (double*)((char*)c.batch_host + (size_t)n * sizeof(SolverCtl));
  WB_CK(ctx, cudaMemcpyAsync(hc, b.ctl, n * sizeof(SolverCtl), cudaMemcpyDeviceToHost, s));
  WB_CK(ctx, cudaMemcpyAsync(hs, b.scal, 4 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  WB_CK(ctx, cudaStreamSynchronize(s));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  wd_status worst = WD_OK;
  for (int r = 0; r < n; ++r) {
    const double b2 = hs[r] + hs[n + r], r2 = hs[2 * n + r] + hs[3 * n + r];
    wd_status sr = (wd_status)hc[r].status;
    if (sr == WD_OK && !hc[r].done) sr = WD_ERR_NOT_CONVERGED;
    if (b2 > 0.0 && !std::isfinite(r2)) sr = WD_ERR_NUMERIC;
    // the reported full residual of the reconstructed x decides convergence
    if (sr == WD_OK && b2 > 0.0 && r2 > p.tol * p.tol * b2) sr = WD_ERR_NOT_CONVERGED;
    if (infos) {
      infos[r].iters = hc[r].iter + hc[r].updates;
      infos[r].reliable_updates = hc[r].updates;
      infos[r].true_rel_residual = b2 > 0.0 ? std::sqrt(r2 / b2) : 0.0;
      infos[r].iterated_rel_residual = b2 > 0.0 ? std::sqrt(hc[r].rr / b2) : 0.0;
      infos[r].seconds = secs;
      infos[r].status = sr;
      infos[r].kernel_launches = 0;
    }
    if (sr != WD_OK && worst == WD_OK) worst = sr;
  }
  if (worst != WD_OK) berr(ctx, worst, "at least one system of the batch did not converge cleanly");
  return worst;
}

}  // namespace

namespace wd {

#define WB_RET(call)                 \
  do {                               \
    cudaError_t e_ = (call);         \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

cudaError_t build_batch_loop_graph(const Ctx& c, int prec, BatchBufs& b, const BatchLaunch& bl, cudaGraph_t* graph,
                                   cudaGraphExec_t* exec, unsigned long long* h_update, unsigned long long* h_loop) {
  const PrecOps* o = prec_ops(prec);
  cudaGraph_t g = nullptr;
  WB_RET(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hl, hu;
  WB_RET(cudaGraphConditionalHandleCreate(&hl, g, 1, cudaGraphCondAssignDefault));
  union Raw {
    cudaGraphNodeParams p;
    unsigned char bytes[sizeof(cudaGraphNodeParams)];
    Raw() { memset(bytes, 0, sizeof(bytes)); }
  } wraw, iraw;
  cudaGraphNodeParams& wp = wraw.p;
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hl;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  WB_RET(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  WB_RET(cudaGraphConditionalHandleCreate(&hu, body, 0, cudaGraphCondAssignDefault));
  cudaStream_t cs;
  WB_RET(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t unused;
  WB_RET(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  o->batch_iteration(c, bl, b, cs);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  WB_RET(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
  WB_RET(cudaStreamEndCapture(cs, &unused));
  cudaGraphNodeParams& ip = iraw.p;
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hu;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  WB_RET(cudaGraphAddNode(&inode, body, tail.data(), nullptr, tail.size(), &ip));
  cudaGraph_t ubody = ip.conditional.phGraph_out[0];
  WB_RET(cudaStreamBeginCaptureToGraph(cs, ubody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  o->batch_update(c, bl, b, cs);
  WB_RET(cudaStreamEndCapture(cs, &unused));
  WB_RET(cudaStreamBeginCaptureToGraph(cs, body, &inode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  batch_loop_control_kernel<<<1, 1, 0, cs>>>(b.bc, b.ctl, bl.nrhs);
  WB_RET(cudaStreamEndCapture(cs, &unused));
  WB_RET(cudaStreamDestroy(cs));
  WB_RET(cudaGraphInstantiate(exec, g, 0));
  *graph = g;
  *h_update = hu;
  *h_loop = hl;
  return cudaSuccess;
}

void batch_release(Ctx& c) {
  destroy_batch_graph(c);
  if (c.batch_block) cudaFree(c.batch_block);
  if (c.batch_small) cudaFree(c.batch_small);
  if (c.batch_host) cudaFreeHost(c.batch_host);
  c.batch_block = nullptr;
  c.batch_small = nullptr;
  c.batch_host = nullptr;
  c.batch_n = 0;
  c.batch_prec = -1;
  c.batch_tr = 0;
  c.batch_pack = 0;
}
}  // namespace wd

extern "C" {

wd_status wd_dslash_batch(wd_ctx* ctx, void* out, const void* in, int nrhs, wd_parity out_parity, int dagger,
                          wd_prec prec) {
  if (!ctx || !out || !in || out == in || nrhs < 1 || nrhs > kMaxBatch || (out_parity != 0 && out_parity != 1) ||
      prec < WD_F64 || prec > WD_B16N)
    return berr(ctx, WD_ERR_INVALID_ARG, "wd_dslash_batch: bad args");
  Ctx& c = ctx->c;
  WB_CK(ctx, cudaSetDevice(c.device));
  wd_status st = wd_internal_ensure_gauge(ctx, prec);
  if (st != WD_OK) return st;
  BatchLaunch bl{nrhs, 4, c.num_sms * 4, blas_gx(c, nrhs)};
  if (c.batch_tr && c.batch_n == nrhs && c.batch_prec == prec) {
    bl.tr = std::max(c.batch_tr, 0);
    bl.grid = c.batch_grid;
    bl.pack = c.batch_tr > 0 ? c.batch_pack : 0;
  }
  const int ntiles = (c.g.Vh + 31) / 32;
  if (bl.tr && bl.grid > ntiles) bl.grid = ntiles;
  prec_ops(prec)->dslash_batch(c, bl, out, in, out_parity, dagger ? 1 : 0, c.stream);
  WB_CK_LAUNCH(ctx);
  return WD_OK;
}

wd_status wd_solve_batch_device(wd_ctx* ctx, int n, void* x, const void* b, const double* kappas,
                                const wd_solve_params* params, wd_solve_info* infos) {
  if (!ctx || !x || !b || !kappas || x == b) return berr(ctx, WD_ERR_INVALID_ARG, "wd_solve_batch_device: bad args");
  WB_CK(ctx, cudaSetDevice(ctx->c.device));
  return solve_batch_device(ctx, n, x, b, kappas, params, infos);
}

wd_status wd_solve_batch(wd_ctx* ctx, int n, double* const* x, const double* const* b, const double* kappas,
                         const wd_solve_params* params, wd_solve_info* infos) {
  if (!ctx || !x || !b || !kappas || n < 1 || n > kMaxBatch)
    return berr(ctx, WD_ERR_INVALID_ARG, "wd_solve_batch: bad args");
  for (int r = 0; r < n; ++r)
    if (!x[r] || !b[r]) return berr(ctx, WD_ERR_INVALID_ARG, "wd_solve_batch: null field pointer");
  Ctx& c = ctx->c;
  WB_CK(ctx, cudaSetDevice(c.device));
  const size_t full = 2 * fbytes(c, WD_F64);
  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, 2 * full * n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bcuda(ctx, e, "wd_solve_batch fields");
  }
  char* bf = (char*)dev;
  char* xf = bf + full * n;
  wd_status st = WD_OK;
  for (int r = 0; r < n && st == WD_OK; ++r) {
    st = wd_internal_import_full(ctx, bf + r * full, bf + r * full + full / 2, b[r]);
  }
  wd_status rs = st;
  if (st == WD_OK) rs = solve_batch_device(ctx, n, xf, bf, kappas, params, infos);
  if (rs == WD_OK || rs == WD_ERR_NOT_CONVERGED || rs == WD_ERR_BREAKDOWN || rs == WD_ERR_NUMERIC) {
    for (int r = 0; r < n; ++r) {
      wd_status s2 = wd_internal_export_full(ctx, x[r], xf + r * full, xf + r * full + full / 2);
      if (s2 != WD_OK) {
        rs = s2;
        break;
      }
    }
  }
  cudaFree(dev);
  return rs;
}

}  // extern "C"
