// Serving: continuous batching of solve requests (C ABI wd_server_*).
//
// Requests (a source b, kappa, tol) arrive for one of several resident gauge
// fields, possibly of different lattice volumes.  Each gauge field has a pool:
// its own context and CUDA stream, and -- while it has work -- a batch of
// solver slots in one device allocation, iterated in lockstep by the batched
// reliable-update BiCGstab (wd_batch.cuh) as a CUDA graph that pauses every
// `iters_per_step` iterations.  Between steps the host retires converged
// slots (FP64 reconstruction and true residual on the device, solution copied
// to the caller's buffer), admits queued requests into free slots (setup of
// one slot while the others keep their Krylov state), and releases the slot
// memory of idle pools so that other pools can grow.  Every allocation is
// charged against a device-memory budget; pools on different streams overlap
// on the device.  A request's iteration is the same kernel sequence whether it
// runs alone or in a mix, so its result does not depend on its neighbours
// beyond rounding of the reductions' block partition.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "wd_batch.cuh"

using namespace wd;

namespace {

struct Request {
  long long id;
  int pool;
  const double* b;
  double* x;
  double kappa, tol;
  int state;  // 0 queued, 1 active, 3 solution download in flight, 2 finished
  int slot;
  wd_solve_info info;
  std::chrono::steady_clock::time_point t_submit;
  SolverCtl final_ctl;           // the slot's control block when it retired
  int scal_idx = -1;             // entry of wd_server::scal_pinned with its four norms
  cudaEvent_t done_ev = nullptr; // recorded after the solution download
};

struct Pool {
  wd_ctx* ctx = nullptr;
  int dims[4] = {0, 0, 0, 0};
  size_t fixed_bytes = 0;  // gauge copies, staging, scratch
  int capacity = 0;        // slots (0: no workspace)
  void* ws = nullptr;      // slot fields
  void* small = nullptr;   // ctl array, BatchCtl, partials, kappas, scalars
  size_t ws_bytes = 0;
  BatchBufs bb{};
  void* bfull = nullptr;   // per slot FP64 full source field (inside ws)
  BatchLaunch bl{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long hu = 0, hl = 0;
  std::vector<long long> slot_req;  // -1 free
  std::deque<long long> queue;
  SolverCtl* hctl = nullptr;        // pinned mirror of the ctl array
  bool launched = false;            // a step of iterations is in flight
  int trace_idx = -1;               // its record in the server's trace (WD_SERVER_TRACE)
  cudaEvent_t start_ev = nullptr;   // recorded before the step's iterations
  cudaEvent_t done_ev = nullptr;    // recorded after them
  // the source of the next queued request, uploaded on a stream of its own
  // while the pool's steps run (host layout, one full field)
  void* pf_buf = nullptr;
  cudaStream_t pf_stream = nullptr;
  cudaEvent_t pf_done = nullptr;    // the upload into pf_buf has completed
  cudaEvent_t pf_free = nullptr;    // the admission has read pf_buf
  long long pf_req = -1;            // request whose source is in pf_buf (or on its way)
  cudaEvent_t turn_ev = nullptr;    // trace: recorded before the retire and admit work
  cudaEvent_t seg_ev[4] = {nullptr, nullptr, nullptr, nullptr};  // trace: ends of the turnover segments
  bool seg_used = false;            // trace: a retire and an admission ran in this turnover
  double t_seen = 0.0;              // trace: when the last step was seen complete
};

}  // namespace

// A caller's host buffer, page-locked by the server (cudaHostRegister) so
// that uploads and downloads run asynchronously; released when no pending
// request uses it.  Buffers the caller had already page-locked are used as
// they are.
struct Pin {
  size_t bytes = 0;
  int refs = 0;
  bool registered = false;
};

// One completed step of a pool, for the optional trace (WD_SERVER_TRACE)
struct StepRecord {
  double t_launch;  // seconds since the server was created, when the step was launched
  double t_end;     // ... when the step was seen complete
  int pool;
  int capacity;     // slots of the pool's workspace
  int active;       // slots holding a request during the step
  int admitted;     // requests admitted just before the step
  double step_ms;   // device time of the step (events around its iterations)
  double turn_ms;   // device time from the previous step's end to this one's start (retire, admit)
  double host_ms;   // host time from seeing the previous step complete to this launch
  double seg_ms[4]; // of turn_ms: retire kernels, export + download, upload + import, admission kernels
};

struct wd_server {
  wd_server_params p;
  std::vector<Pool> pools;
  std::map<long long, Request> reqs;
  std::map<const void*, Pin> pins;
  // pinned host entries (4 doubles: |b_e|^2, |b_o|^2, |r_e|^2, |r_o|^2) that
  // retired requests' norms are downloaded into; free list of entries
  double* scal_pinned = nullptr;
  std::vector<int> scal_free;
  size_t used = 0;
  long long next_id = 1;
  std::string err;
  wd_server_stats st{};
  // optional trace of every completed step, written as CSV to the file named
  // by WD_SERVER_TRACE when the server is destroyed (empty: no trace)
  std::string trace_path;
  std::vector<StepRecord> trace;
  long long pins_registered = 0, pins_pageable = 0;  // host buffers page-locked / left pageable
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

wd_status serr(wd_server* s, wd_status st, const std::string& m) {
  if (s) s->err = m;
  return st;
}

void pin(wd_server* s, const void* p, size_t bytes) {
  Pin& pn = s->pins[p];
  if (pn.refs++ > 0) return;
  pn.bytes = bytes;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost) return;  // already pinned
  cudaGetLastError();
  pn.registered = cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterDefault) == cudaSuccess;
  if (!pn.registered) cudaGetLastError();  // pageable: transfers stay correct, just synchronous
  ++(pn.registered ? s->pins_registered : s->pins_pageable);
}

void unpin(wd_server* s, const void* p) {
  auto it = s->pins.find(p);
  if (it == s->pins.end()) return;
  if (--it->second.refs > 0) return;
  if (it->second.registered) cudaHostUnregister(const_cast<void*>(p));
  s->pins.erase(it);
}

#define WS_CK(s, call)                                                                                    \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess)                                                                                \
      return serr(s, e_ == cudaErrorMemoryAllocation ? WD_ERR_OOM : WD_ERR_CUDA,                          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                    \
  } while (0)

size_t fbytes(const Ctx& c, int prec) { return prec_ops(prec)->field_bytes(c.g.stride); }

size_t slot_bytes(const Ctx& c, int prec) {
  return 2 * fbytes(c, WD_F64) + 3 * fbytes(c, WD_F64) + 7 * fbytes(c, prec);
}

int blas_gx_for(const Ctx& c, int n) {
  const int per = (c.num_sms * 8 + n - 1) / n;
  const int need = (c.g.Vh + kBlasBlock - 1) / kBlasBlock;
  return std::max(1, std::min(per, need));
}

// Launch shape for a capacity of n slots.  rhs_tile > 0 (or 0 with more than
// two slots): right-hand sides per block no more than the slots (a block's
// threads for absent systems idle), and enough blocks that the sites of one
// system alone fill the device.  rhs_tile -1 (or 0 with one or two slots):
// one system per block row, the single-system grid, blocks of absent systems
// return at once.  (Choosing the shape per step from the systems present,
// with one graph per shape, measured no faster on the serving stream.)
BatchLaunch pool_shape(const Ctx& c, int n, int rhs_tile) {
  const int ntiles = (c.g.Vh + 31) / 32;
  int tr = 1;
  if (rhs_tile > 0) {
    tr = rhs_tile;
  } else {
    while (tr < n && tr < 4) tr *= 2;
    if (rhs_tile < 0 || n <= 2) tr = 0;
  }
  BatchLaunch bl{n, tr, tr ? std::min(c.num_sms * (64 / tr), ntiles) : rhs_grid64(c.g, c.num_sms),
                 blas_gx_for(c, n)};
  bl.grid64 = rhs_grid64(c.g, c.num_sms);
  return bl;
}

size_t small_bytes(const Ctx& c, int n, int rhs_tile) {
  const BatchLaunch bl = pool_shape(c, n, rhs_tile);
  const int maxblk = std::max(std::max(bl.grid, bl.grid64), bl.blas_gx);
  return align256((size_t)n * sizeof(SolverCtl)) + align256(sizeof(BatchCtl)) +
         align256((size_t)maxblk * n * 4 * sizeof(double)) + align256((size_t)2 * n * 8) + align256((size_t)4 * n * 8);
}

__global__ void slot_init_kernel(SolverCtl* ctl, double tol, double delta, int max_iter, double kappa,
                                 const double* bnorm2) {
  SolverCtl c;
  memset(&c, 0, sizeof(c));
  c.rho = c.rho_prev = c.alpha = c.omega = make_double2(1.0, 0.0);
  c.beta = make_double2(0.0, 0.0);
  const double b2 = bnorm2[0] + bnorm2[1];
  c.stop2 = tol * tol * b2;
  c.delta = delta;
  c.kappa = kappa;
  c.neg_kappa2 = -kappa * kappa;
  c.max_iter = max_iter;
  c.status = WD_OK;
  if (!isfinite(b2)) {
    c.status = WD_ERR_NUMERIC;
    c.done = 1;
  } else if (b2 == 0.0) {
    c.done = 1;
  }
  *ctl = c;
}

__global__ void mark_free_kernel(SolverCtl* ctl, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) {
    ctl[r].done = 1;
    ctl[r].do_update = 0;
  }
}

__global__ void batch_reset_kernel(BatchCtl* bc, int step_limit, int in_graph, unsigned long long hu,
                                   unsigned long long hl) {
  for (int k = 0; k < 4; ++k) bc->counter[k] = 0;
  bc->any_update = 0;
  bc->all_done = 0;
  bc->in_graph = in_graph;
  bc->loops = 0;
  bc->max_loops = 1 << 30;  // slots carry their own max_iter
  bc->step_loops = 0;
  bc->step_limit = step_limit;
  bc->h_update = hu;
  bc->h_loop = hl;
}

void release_workspace(Pool& pl, size_t& used) {
  if (pl.exec) cudaGraphExecDestroy(pl.exec);
  if (pl.graph) cudaGraphDestroy(pl.graph);
  pl.exec = nullptr;
  pl.graph = nullptr;
  if (pl.ws) cudaFree(pl.ws);
  if (pl.small) cudaFree(pl.small);
  if (pl.hctl) cudaFreeHost(pl.hctl);
  pl.ws = pl.small = nullptr;
  pl.hctl = nullptr;
  used -= pl.ws_bytes;
  pl.ws_bytes = 0;
  pl.capacity = 0;
  pl.slot_req.clear();
}

// Workspace for `cap` slots: the batch views of wd_batch.cuh plus one FP64
// full source field per slot.
wd_status alloc_workspace(wd_server* sv, Pool& pl, int cap) {
  Ctx& c = pl.ctx->c;
  const int prec = sv->p.inner_precision;
  const size_t f64 = fbytes(c, WD_F64), fin = fbytes(c, prec);
  const size_t ws = slot_bytes(c, prec) * cap, sm = small_bytes(c, cap, sv->p.rhs_tile);
  WS_CK(sv, cudaMalloc(&pl.ws, ws));
  if (cudaMalloc(&pl.small, sm) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(pl.ws);
    pl.ws = nullptr;
    return serr(sv, WD_ERR_OOM, "slot control allocation failed");
  }
  // on the pool's stream: a plain cudaMemset runs on the legacy default
  // stream, which is not ordered with the pool's non-blocking stream and could
  // land after the slots' control blocks are initialised
  WS_CK(sv, cudaMemsetAsync(pl.small, 0, sm, c.stream));
  WS_CK(sv, cudaMallocHost((void**)&pl.hctl, (size_t)cap * sizeof(SolverCtl)));
  pl.ws_bytes = ws + sm;
  sv->used += pl.ws_bytes;
  pl.capacity = cap;
  pl.slot_req.assign(cap, -1);
  // carve the views
  char* s = (char*)pl.small;
  BatchBufs& b = pl.bb;
  b.ctl = (SolverCtl*)s;
  s += align256((size_t)cap * sizeof(SolverCtl));
  b.bc = (BatchCtl*)s;
  s += align256(sizeof(BatchCtl));
  b.partials = (double*)s;
  {
    const BatchLaunch bl = pool_shape(c, cap, sv->p.rhs_tile);
    s += align256((size_t)std::max(std::max(bl.grid, bl.grid64), bl.blas_gx) * cap * 4 * sizeof(double));
  }
  b.kappas = (double*)s;
  s += align256((size_t)2 * cap * 8);
  b.scal = (double*)s;
  char* p = (char*)pl.ws;
  pl.bfull = p; p += 2 * f64 * cap;
  b.b_hat = p; p += f64 * cap;
  b.xe = p; p += f64 * cap;
  b.tmp64 = p; p += f64 * cap;
  b.r_hat = p; p += fin * cap;
  b.r_tilde = p; p += fin * cap;
  b.p = p; p += fin * cap;
  b.v = p; p += fin * cap;
  b.t = p; p += fin * cap;
  b.x_hat = p; p += fin * cap;
  b.tmp = p; p += fin * cap;
  pl.bl = pool_shape(c, cap, sv->p.rhs_tile);
  mark_free_kernel<<<(cap + 127) / 128, 128, 0, c.stream>>>(b.ctl, cap);
  WS_CK(sv, cudaGetLastError());
  if (sv->p.use_graph) {
    cudaError_t e = build_batch_loop_graph(c, prec, b, pl.bl, &pl.graph, &pl.exec, &pl.hu, &pl.hl);
    if (e != cudaSuccess) return serr(sv, WD_ERR_CUDA, std::string("pool graph: ") + cudaGetErrorString(e));
  }
  WS_CK(sv, cudaStreamSynchronize(c.stream));
  return WD_OK;
}

// single-slot views (batch fields at slot r)
SolveBufs slot_bufs(Pool& pl, int r, int prec) {
  Ctx& c = pl.ctx->c;
  const size_t f64 = fbytes(c, WD_F64), fin = fbytes(c, prec);
  SolveBufs s{};
  s.ctl = pl.bb.ctl + r;
  s.b_hat = (char*)pl.bb.b_hat + r * f64;
  s.x = (char*)pl.bb.xe + r * f64;
  s.r = nullptr;
  s.tmp64 = (char*)pl.bb.tmp64 + r * f64;
  s.r_hat = (char*)pl.bb.r_hat + r * fin;
  s.r_tilde = (char*)pl.bb.r_tilde + r * fin;
  s.p = (char*)pl.bb.p + r * fin;
  s.v = (char*)pl.bb.v + r * fin;
  s.t = (char*)pl.bb.t + r * fin;
  s.x_hat = (char*)pl.bb.x_hat + r * fin;
  s.tmp = (char*)pl.bb.tmp + r * fin;
  return s;
}

// admission of one request into slot r: source upload, Schur source, control
// block, quantised residual; the other slots keep their Krylov state
using Clock = std::chrono::steady_clock;
double since(Clock::time_point t0) { return std::chrono::duration<double>(Clock::now() - t0).count(); }

wd_status admit(wd_server* sv, Pool& pl, Request& q, int r) {
  const auto t0 = Clock::now();
  ++sv->st.admitted;
  struct Acc {
    wd_server* s;
    Clock::time_point t;
    ~Acc() { s->st.admit_seconds += since(t); }
  } acc{sv, t0};
  Ctx& c = pl.ctx->c;
  const int prec = sv->p.inner_precision;
  const size_t f64 = fbytes(c, WD_F64);
  char* bf = (char*)pl.bfull + 2 * f64 * r;
  const bool seg = !sv->trace_path.empty() && pl.seg_ev[1];
  if (seg) WS_CK(sv, cudaEventRecord(pl.seg_ev[2], c.stream));
  if (pl.pf_req == q.id) {  // uploaded ahead: convert from the prefetch buffer
    WS_CK(sv, cudaStreamWaitEvent(c.stream, pl.pf_done, 0));
    ops_f64()->import_lex(c, bf, (const double*)pl.pf_buf, 0, c.stream);
    ops_f64()->import_lex(c, bf + f64, (const double*)pl.pf_buf, 1, c.stream);
    WS_CK(sv, cudaEventRecord(pl.pf_free, c.stream));
    pl.pf_req = -1;
  } else {
    wd_status st = wd_internal_import_full(pl.ctx, bf, bf + f64, q.b);
    if (st != WD_OK) return serr(sv, st, std::string("source upload: ") + wd_last_error(pl.ctx));
  }
  if (seg) {
    WS_CK(sv, cudaEventRecord(pl.seg_ev[3], c.stream));
    pl.seg_used = true;
  }
  const PrecOps* o64 = ops_f64();
  SolveBufs s = slot_bufs(pl, r, prec);
  double* sc = pl.bb.scal + 4 * r;
  o64->norm2(c, sc + 0, bf, c.stream);
  o64->norm2(c, sc + 1, bf + f64, c.stream);
  o64->dslash_xpay(c, s.b_hat, bf + f64, bf, q.kappa, nullptr, 0, 0, c.stream);
  o64->zero(c, s.x, c.stream);
  slot_init_kernel<<<1, 1, 0, c.stream>>>(s.ctl, q.tol, prec == WD_F64 ? 0.0 : sv->p.delta, sv->p.max_iter, q.kappa,
                                          sc);
  prec_ops(prec)->bicg_setup(c, s, s.b_hat, c.stream);
  WS_CK(sv, cudaGetLastError());
  pl.slot_req[r] = q.id;
  q.state = 1;
  q.slot = r;
  return WD_OK;
}

wd_status finish(wd_server* sv, Request& q);

// retirement of slot r: x_e, x_o = b_o + kappa D_oe x_e, the full FP64 true
// residual, and the solution downloaded to the caller's buffer; all stream
// ordered (the slot can take a new request at once).  The request finishes
// when its event, recorded after the download, has completed (finish()).
wd_status retire(wd_server* sv, Pool& pl, Request& q, int r, const SolverCtl& hc) {
  ++sv->st.retired;
  struct Acc {
    wd_server* s;
    Clock::time_point t;
    ~Acc() { s->st.retire_seconds += since(t); }
  } acc{sv, Clock::now()};
  Ctx& c = pl.ctx->c;
  const int prec = sv->p.inner_precision;
  const size_t f64 = fbytes(c, WD_F64);
  const char* bf = (const char*)pl.bfull + 2 * f64 * r;
  SolveBufs s = slot_bufs(pl, r, prec);
  using T64 = Tr<WD_F64>;
  const Geom& g = c.g;
  ops_f64()->dslash_xpay(c, s.tmp64, s.x, bf + f64, q.kappa, nullptr, 1, 0, c.stream);  // x_o in tmp64
  double* sc = pl.bb.scal + 4 * r;
  const Coef ck{-q.kappa, nullptr};
  EpiResid<SpinorF64, SpinorF64, SpinorF64, FinStore> ee{T64::view(nullptr, g), false, T64::view(bf, g),
                                                         T64::view(s.x, g), ck, c.red, FinStore{sc + 2, 1}};
  launch_dslash<double>(c, T64::view(s.tmp64, g), T64::gauge(c), 0, 0, ee, c.stream);
  EpiResid<SpinorF64, SpinorF64, SpinorF64, FinStore> eo{T64::view(nullptr, g), false, T64::view(bf + f64, g),
                                                         T64::view(s.tmp64, g), ck, c.red, FinStore{sc + 3, 1}};
  launch_dslash<double>(c, T64::view(s.x, g), T64::gauge(c), 1, 0, eo, c.stream);
  WS_CK(sv, cudaGetLastError());
  // the request's four norms into its own pinned entry
  if (!sv->scal_pinned) {
    constexpr int kEntries = 4096;
    WS_CK(sv, cudaMallocHost((void**)&sv->scal_pinned, (size_t)kEntries * 4 * sizeof(double)));
    for (int k = kEntries - 1; k >= 0; --k) sv->scal_free.push_back(k);
  }
  if (sv->scal_free.empty()) {  // more downloads in flight than entries: wait for them
    WS_CK(sv, cudaDeviceSynchronize());
    for (auto& kv : sv->reqs)
      if (kv.second.state == 3) finish(sv, kv.second);
  }
  q.scal_idx = sv->scal_free.back();
  sv->scal_free.pop_back();
  WS_CK(sv, cudaMemcpyAsync(sv->scal_pinned + 4 * q.scal_idx, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                            c.stream));
  if (!sv->trace_path.empty()) {
    for (cudaEvent_t& e : pl.seg_ev)
      if (!e) WS_CK(sv, cudaEventCreate(&e));
    WS_CK(sv, cudaEventRecord(pl.seg_ev[0], c.stream));
  }
  const wd_status st = wd_internal_export_full_async(pl.ctx, q.x, s.x, s.tmp64);
  if (st != WD_OK) return serr(sv, st, std::string("solution download: ") + wd_last_error(pl.ctx));
  if (!sv->trace_path.empty()) WS_CK(sv, cudaEventRecord(pl.seg_ev[1], c.stream));
  q.final_ctl = hc;
  if (!q.done_ev) WS_CK(sv, cudaEventCreateWithFlags(&q.done_ev, cudaEventDisableTiming));
  WS_CK(sv, cudaEventRecord(q.done_ev, c.stream));
  q.state = 3;
  pl.slot_req[r] = -1;
  mark_free_kernel<<<1, 1, 0, c.stream>>>(pl.bb.ctl + r, 1);
  WS_CK(sv, cudaGetLastError());
  return WD_OK;
}

// a retired request whose download has completed: fill in its info
wd_status finish(wd_server* sv, Request& q) {
  const cudaError_t e = cudaEventQuery(q.done_ev);
  if (e == cudaErrorNotReady) return WD_OK;
  if (e != cudaSuccess) return serr(sv, WD_ERR_CUDA, std::string("request download: ") + cudaGetErrorString(e));
  const double* h = sv->scal_pinned + 4 * q.scal_idx;
  const SolverCtl& hc = q.final_ctl;
  const double b2 = h[0] + h[1], r2 = h[2] + h[3];
  wd_status rs = (wd_status)hc.status;
  if (rs == WD_OK && !hc.done) rs = WD_ERR_NOT_CONVERGED;
  if (b2 > 0.0 && !std::isfinite(r2)) rs = WD_ERR_NUMERIC;
  // the reported full residual of the reconstructed x decides convergence
  if (rs == WD_OK && b2 > 0.0 && r2 > q.tol * q.tol * b2) rs = WD_ERR_NOT_CONVERGED;
  q.info.iters = hc.iter + hc.updates;
  q.info.reliable_updates = hc.updates;
  q.info.true_rel_residual = b2 > 0.0 ? std::sqrt(r2 / b2) : 0.0;
  q.info.iterated_rel_residual = b2 > 0.0 ? std::sqrt(hc.rr / b2) : 0.0;
  q.info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - q.t_submit).count();
  q.info.status = rs;
  q.info.kernel_launches = 0;
  q.state = 2;
  sv->scal_free.push_back(q.scal_idx);
  q.scal_idx = -1;
  cudaEventDestroy(q.done_ev);
  q.done_ev = nullptr;
  unpin(sv, q.b);
  unpin(sv, q.x);
  return WD_OK;
}

// Upload the source of the pool's next queued request into its prefetch
// buffer, on the prefetch stream, so that the copy overlaps the pool's steps
// (the admission then only converts it); after the previous admission has
// read the buffer.
wd_status prefetch(wd_server* s, Pool& pl) {
  if (!pl.pf_buf || pl.pf_req >= 0 || pl.queue.empty()) return WD_OK;
  const Request& q = s->reqs[pl.queue.front()];
  const size_t bytes = (size_t)2 * pl.ctx->c.g.Vh * 24 * sizeof(double);
  WS_CK(s, cudaStreamWaitEvent(pl.pf_stream, pl.pf_free, 0));
  WS_CK(s, cudaMemcpyAsync(pl.pf_buf, q.b, bytes, cudaMemcpyHostToDevice, pl.pf_stream));
  WS_CK(s, cudaEventRecord(pl.pf_done, pl.pf_stream));
  pl.pf_req = q.id;
  return WD_OK;
}

// One pool: retire finished slots, release idle memory, admit, launch.
// did_work: a step completed, memory moved, a request was admitted or a step
// launched (a pool that only waits for memory does nothing)
wd_status pool_progress(wd_server* s, Pool& pl, int& waiting_for_memory, bool& did_work) {
  const int prec = s->p.inner_precision;
  Ctx& c = pl.ctx->c;
  did_work = false;
  if (pl.launched) {
    did_work = true;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pl.start_ev, pl.done_ev) == cudaSuccess) s->st.gpu_step_seconds += 1e-3 * ms;
    else cudaGetLastError();
    if (!s->trace_path.empty() && pl.trace_idx >= 0) {
      StepRecord& rec = s->trace[pl.trace_idx];
      rec.t_end = pl.t_seen = since(s->t0);
      rec.step_ms = ms;
      float tm = 0.f;
      if (pl.turn_ev && cudaEventElapsedTime(&tm, pl.turn_ev, pl.start_ev) == cudaSuccess) rec.turn_ms = tm;
      else cudaGetLastError();
      if (pl.seg_used) {
        const cudaEvent_t a[4] = {pl.turn_ev, pl.seg_ev[0], pl.seg_ev[2], pl.seg_ev[3]};
        const cudaEvent_t b[4] = {pl.seg_ev[0], pl.seg_ev[1], pl.seg_ev[3], pl.start_ev};
        for (int k = 0; k < 4; ++k) {
          float sm = 0.f;
          if (cudaEventElapsedTime(&sm, a[k], b[k]) == cudaSuccess) rec.seg_ms[k] = sm;
          else cudaGetLastError();
        }
        pl.seg_used = false;
      }
      if (!pl.turn_ev) WS_CK(s, cudaEventCreate(&pl.turn_ev));
      WS_CK(s, cudaEventRecord(pl.turn_ev, c.stream));
    }
    // retire the slots whose system finished during the step just completed
    WS_CK(s, cudaMemcpyAsync(pl.hctl, pl.bb.ctl, pl.capacity * sizeof(SolverCtl), cudaMemcpyDeviceToHost, c.stream));
    WS_CK(s, cudaStreamSynchronize(c.stream));
    for (int r = 0; r < pl.capacity; ++r) {
      if (pl.slot_req[r] < 0 || !pl.hctl[r].done) continue;
      wd_status st = retire(s, pl, s->reqs[pl.slot_req[r]], r, pl.hctl[r]);
      if (st != WD_OK) return st;
    }
    pl.launched = false;
  }
  bool busy = false;
  for (long long id : pl.slot_req) busy |= (id >= 0);
  if (pl.capacity && !busy && pl.queue.empty()) {
    // the retirements just enqueued still read the slot fields
    WS_CK(s, cudaStreamSynchronize(c.stream));
    release_workspace(pl, s->used);
    did_work = true;
  }
  if (!pl.queue.empty() && !pl.capacity) {
    // slot memory: what the budget has left, shared with the other pools that wait
    const size_t left = s->p.budget_bytes ? (s->p.budget_bytes > s->used ? s->p.budget_bytes - s->used : 0)
                                          : (size_t)-1;
    const size_t share = s->p.budget_bytes ? left / (size_t)std::max(1, waiting_for_memory) : left;
    int cap = s->p.max_slots;
    while (cap > 0 && s->p.budget_bytes && slot_bytes(c, prec) * cap + small_bytes(c, cap, s->p.rhs_tile) > share)
      --cap;
    if (cap < 1 && s->p.budget_bytes && slot_bytes(c, prec) + small_bytes(c, 1, s->p.rhs_tile) <= left) cap = 1;
    if (cap >= 1) {
      --waiting_for_memory;
      wd_status st = alloc_workspace(s, pl, cap);
      if (st != WD_OK) return st;
      did_work = true;
    }
  }
  int admitted = 0;
  for (int r = 0; r < pl.capacity && !pl.queue.empty(); ++r) {
    if (pl.slot_req[r] >= 0) continue;
    const long long id = pl.queue.front();
    pl.queue.pop_front();
    wd_status st = admit(s, pl, s->reqs[id], r);
    if (st != WD_OK) return st;
    ++admitted;
  }
  int n = 0;
  for (long long id : pl.slot_req) n += (id >= 0);
  if (!n) return WD_OK;
  // up to iters_per_step lockstep iterations, then an event marks the end
  if (!pl.start_ev) WS_CK(s, cudaEventCreate(&pl.start_ev));
  if (!pl.done_ev) WS_CK(s, cudaEventCreate(&pl.done_ev));
  WS_CK(s, cudaEventRecord(pl.start_ev, c.stream));
  batch_reset_kernel<<<1, 1, 0, c.stream>>>(pl.bb.bc, s->p.iters_per_step, s->p.use_graph ? 1 : 0, pl.hu, pl.hl);
  WS_CK(s, cudaGetLastError());
  if (s->p.use_graph) {
    WS_CK(s, cudaGraphLaunch(pl.exec, c.stream));
  } else {
    const PrecOps* o = prec_ops(prec);
    BatchCtl hb;
    for (int it = 0; it < s->p.iters_per_step; ++it) {
      o->batch_iteration(c, pl.bl, pl.bb, c.stream);
      WS_CK(s, cudaMemcpyAsync(&hb, pl.bb.bc, sizeof(hb), cudaMemcpyDeviceToHost, c.stream));
      WS_CK(s, cudaStreamSynchronize(c.stream));
      if (hb.any_update) o->batch_update(c, pl.bl, pl.bb, c.stream);
      batch_loop_control_kernel<<<1, 1, 0, c.stream>>>(pl.bb.bc, pl.bb.ctl, pl.capacity);
      WS_CK(s, cudaMemcpyAsync(&hb, pl.bb.bc, sizeof(hb), cudaMemcpyDeviceToHost, c.stream));
      WS_CK(s, cudaStreamSynchronize(c.stream));
      if (hb.all_done) break;
    }
  }
  WS_CK(s, cudaEventRecord(pl.done_ev, c.stream));
  pl.launched = true;
  if (wd_status pst = prefetch(s, pl); pst != WD_OK) return pst;
  if (!s->trace_path.empty()) {
    pl.trace_idx = (int)s->trace.size();
    const double now = since(s->t0);
    s->trace.push_back(StepRecord{now, 0.0, (int)(&pl - s->pools.data()), pl.capacity, n, admitted, 0.0, 0.0,
                                  pl.t_seen > 0.0 ? 1e3 * (now - pl.t_seen) : 0.0, {0.0, 0.0, 0.0, 0.0}});
  }
  did_work = true;
  ++s->st.steps;
  return WD_OK;
}

}  // namespace

extern "C" {

wd_status wd_server_create(wd_server** out, const wd_server_params* p) {
  if (!out || !p) return WD_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->max_slots < 1 || p->max_slots > 256 || p->iters_per_step < 1 || p->inner_precision < WD_F64 ||
      p->inner_precision > WD_B16N || p->max_iter < 1)
    return WD_ERR_INVALID_ARG;
  if (p->inner_precision != WD_F64 && !(p->delta > 0.0 && p->delta < 1.0)) return WD_ERR_INVALID_ARG;
  if (p->gauge_flags & ~(WD_GAUGE_TEMPORAL | WD_GAUGE_RECON8)) return WD_ERR_INVALID_ARG;
  if (!(p->rhs_tile >= -1 && p->rhs_tile <= 2) && p->rhs_tile != 4) return WD_ERR_INVALID_ARG;
  wd_server* s = new (std::nothrow) wd_server();
  if (!s) return WD_ERR_OOM;
  s->p = *p;
  if (const char* tp = std::getenv("WD_SERVER_TRACE")) s->trace_path = tp;
  *out = s;
  return WD_OK;
}

wd_status wd_server_destroy(wd_server* s) {
  if (!s) return WD_OK;
  if (!s->trace_path.empty()) {
    if (FILE* f = std::fopen(s->trace_path.c_str(), "w")) {
      std::fprintf(f, "# host buffers page-locked %lld, left pageable %lld\n", s->pins_registered,
                   s->pins_pageable);
      std::fprintf(f,
                   "t_launch_s,t_end_s,pool,dims,capacity,active,admitted,step_ms,turn_ms,host_ms,"
                   "retire_ms,download_ms,upload_ms,admit_ms\n");
      for (const StepRecord& r : s->trace) {
        const Pool& pl = s->pools[r.pool];
        std::fprintf(f, "%.6f,%.6f,%d,%dx%dx%dx%d,%d,%d,%d,%.4f,%.4f,%.4f,%.4f,%.4f,%.4f,%.4f\n", r.t_launch,
                     r.t_end, r.pool, pl.dims[0], pl.dims[1], pl.dims[2], pl.dims[3], r.capacity, r.active,
                     r.admitted, r.step_ms, r.turn_ms, r.host_ms, r.seg_ms[0], r.seg_ms[1], r.seg_ms[2],
                     r.seg_ms[3]);
      }
      std::fclose(f);
    }
  }
  for (Pool& pl : s->pools) {
    if (pl.ctx) cudaStreamSynchronize(pl.ctx->c.stream);
    if (pl.pf_stream) cudaStreamSynchronize(pl.pf_stream);  // before the host buffers are unregistered
  }
  for (auto& kv : s->reqs) {
    if (kv.second.state == 3) finish(s, kv.second);
    if (kv.second.done_ev) cudaEventDestroy(kv.second.done_ev);
  }
  for (auto& kv : s->pins)
    if (kv.second.registered) cudaHostUnregister(const_cast<void*>(kv.first));
  s->pins.clear();
  if (s->scal_pinned) cudaFreeHost(s->scal_pinned);
  for (Pool& pl : s->pools) {
    if (pl.ctx) cudaStreamSynchronize(pl.ctx->c.stream);
    release_workspace(pl, s->used);
    if (pl.done_ev) cudaEventDestroy(pl.done_ev);
    if (pl.start_ev) cudaEventDestroy(pl.start_ev);
    if (pl.pf_stream) {
      cudaStreamSynchronize(pl.pf_stream);
      cudaStreamDestroy(pl.pf_stream);
    }
    if (pl.pf_done) cudaEventDestroy(pl.pf_done);
    if (pl.pf_free) cudaEventDestroy(pl.pf_free);
    if (pl.pf_buf) cudaFree(pl.pf_buf);
    if (pl.turn_ev) cudaEventDestroy(pl.turn_ev);
    for (cudaEvent_t e : pl.seg_ev)
      if (e) cudaEventDestroy(e);
    if (pl.ctx) {
      cudaStream_t st = pl.ctx->c.stream;
      wd_destroy(pl.ctx);
      if (st) cudaStreamDestroy(st);
    }
  }
  delete s;
  return WD_OK;
}

const char* wd_server_last_error(const wd_server* s) { return s ? s->err.c_str() : "null server"; }

wd_status wd_server_add_gauge(wd_server* s, const int dims[4], int t_antiperiodic, const double* U, int recon,
                              int* gauge_id) {
  if (!s || !dims || !U || !gauge_id) return serr(s, WD_ERR_INVALID_ARG, "wd_server_add_gauge: bad args");
  cudaStream_t st;
  WS_CK(s, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  Pool pl;
  wd_status r = wd_create(&pl.ctx, dims, t_antiperiodic, st);
  if (r != WD_OK) {
    cudaStreamDestroy(st);
    return serr(s, r, "wd_server_add_gauge: bad lattice");
  }
  Ctx& c = pl.ctx->c;
  memcpy(pl.dims, dims, sizeof(pl.dims));
  // resident cost: FP64 and inner gauge copies, staging of one host field,
  // scratch; charged before anything is allocated
  const size_t links = (size_t)8 * c.g.stride;
  size_t inner_gauge = 0;
  const int ip = s->p.inner_precision;
  if (ip == WD_F32) inner_gauge = links * 48;
  else if (ip != WD_F64) inner_gauge = links * 24;
  pl.fixed_bytes = links * (recon / 2) * 16 + inner_gauge + (size_t)2 * c.g.Vh * 24 * 8 + ((size_t)c.num_sms * 128 * 8);
  if (s->p.gauge_flags & WD_GAUGE_TEMPORAL) pl.fixed_bytes += (size_t)2 * 9 * c.g.stride * 16;  // G (import / export)
  pl.fixed_bytes += (size_t)2 * c.g.Vh * 24 * 8;  // prefetch buffer of the next request's source
  if (s->p.budget_bytes && s->used + pl.fixed_bytes > s->p.budget_bytes) {
    wd_destroy(pl.ctx);
    cudaStreamDestroy(st);
    return serr(s, WD_ERR_BUDGET, "gauge field does not fit the memory budget");
  }
  r = wd_load_gauge_opt(pl.ctx, U, 0, recon, s->p.gauge_flags);
  if (r == WD_OK) r = wd_internal_ensure_gauge(pl.ctx, ip);
  if (r != WD_OK) {
    std::string m = wd_last_error(pl.ctx);
    wd_destroy(pl.ctx);
    cudaStreamDestroy(st);
    return serr(s, r, "wd_server_add_gauge: " + m);
  }
  {
    cudaError_t e = cudaMalloc(&pl.pf_buf, (size_t)2 * c.g.Vh * 24 * 8);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl.pf_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl.pf_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl.pf_free, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(pl.pf_free, st);  // the buffer starts free
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (pl.pf_free) cudaEventDestroy(pl.pf_free);
      if (pl.pf_done) cudaEventDestroy(pl.pf_done);
      if (pl.pf_stream) cudaStreamDestroy(pl.pf_stream);
      if (pl.pf_buf) cudaFree(pl.pf_buf);
      wd_destroy(pl.ctx);
      cudaStreamDestroy(st);
      return serr(s, e == cudaErrorMemoryAllocation ? WD_ERR_OOM : WD_ERR_CUDA,
                  std::string("wd_server_add_gauge: prefetch buffer: ") + cudaGetErrorString(e));
    }
  }
  s->used += pl.fixed_bytes;
  s->pools.push_back(std::move(pl));
  *gauge_id = (int)s->pools.size() - 1;
  return WD_OK;
}

wd_status wd_server_submit(wd_server* s, int gauge_id, const double* b, double* x, double kappa, double tol,
                           long long* request_id) {
  if (!s || !b || !x || !request_id || gauge_id < 0 || gauge_id >= (int)s->pools.size() || !(tol > 0.0) ||
      !std::isfinite(kappa))
    return serr(s, WD_ERR_INVALID_ARG, "wd_server_submit: bad args");
  {
    // a request whose single slot could never fit the budget is refused now
    const Pool& pl = s->pools[gauge_id];
    size_t fixed = 0;
    for (const Pool& q : s->pools) fixed += q.fixed_bytes;
    if (s->p.budget_bytes &&
        fixed + slot_bytes(pl.ctx->c, s->p.inner_precision) + small_bytes(pl.ctx->c, 1, s->p.rhs_tile) >
            s->p.budget_bytes)
      return serr(s, WD_ERR_BUDGET, "one solver slot for this lattice exceeds the memory budget");
  }
  const size_t field = (size_t)2 * s->pools[gauge_id].ctx->c.g.Vh * 24 * sizeof(double);
  pin(s, b, field);
  pin(s, x, field);
  Request q{};
  q.id = s->next_id++;
  q.pool = gauge_id;
  q.b = b;
  q.x = x;
  q.kappa = kappa;
  q.tol = tol;
  q.state = 0;
  q.slot = -1;
  q.t_submit = std::chrono::steady_clock::now();
  s->reqs[q.id] = q;
  s->pools[gauge_id].queue.push_back(q.id);
  *request_id = q.id;
  return WD_OK;
}

wd_status wd_server_step(wd_server* s, int* active_out, int* queued_out) {
  if (!s) return WD_ERR_INVALID_ARG;
  // Pools progress independently: a pool whose step is still running on its
  // stream is left alone, so requests on small lattices are not held behind
  // long steps on large ones.  If no pool can make progress, wait for the
  // first running pool to finish its step, then progress again.
  for (int pass = 0; pass < 2; ++pass) {
    int waiting = 0;
    for (Pool& pl : s->pools) waiting += (!pl.queue.empty() && !pl.capacity);
    bool progressed = false;
    for (Pool& pl : s->pools) {
      if (pl.launched) {
        const cudaError_t q = cudaEventQuery(pl.done_ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return serr(s, WD_ERR_CUDA, std::string("pool step: ") + cudaGetErrorString(q));
      } else if (pl.queue.empty()) {
        bool busy = false;
        for (long long id : pl.slot_req) busy |= (id >= 0);
        if (!busy && !pl.capacity) continue;
      }
      bool did = false;
      wd_status st = pool_progress(s, pl, waiting, did);
      if (st != WD_OK) return st;
      progressed |= did;
    }
    if (progressed || pass == 1) break;
    // wait for whichever running pool finishes its step first
    const auto tw = Clock::now();
    for (;;) {
      int running = 0;
      bool ready = false;
      for (Pool& pl : s->pools) {
        if (!pl.launched) continue;
        ++running;
        if (cudaEventQuery(pl.done_ev) != cudaErrorNotReady) ready = true;
      }
      if (!running || ready) break;
      if (since(tw) > 600.0) return serr(s, WD_ERR_TIMEOUT, "no pool finished its step within 600 s");
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    s->st.wait_seconds += since(tw);
  }
  int active = 0, queued = 0;
  for (Pool& pl : s->pools) {
    queued += (int)pl.queue.size();
    for (long long id : pl.slot_req) active += (id >= 0);
  }
  if (active_out) *active_out = active;
  if (queued_out) *queued_out = queued;
  return WD_OK;
}

wd_status wd_server_poll(wd_server* s, long long request_id, int* finished, wd_solve_info* info) {
  if (!s || !finished) return WD_ERR_INVALID_ARG;
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return serr(s, WD_ERR_INVALID_ARG, "unknown request id");
  if (it->second.state == 3) {
    const wd_status st = finish(s, it->second);
    if (st != WD_OK) return st;
  }
  *finished = it->second.state == 2;
  if (*finished && info) *info = it->second.info;
  return WD_OK;
}

size_t wd_server_memory_in_use(const wd_server* s) { return s ? s->used : 0; }

wd_status wd_server_get_stats(const wd_server* s, wd_server_stats* out) {
  if (!s || !out) return WD_ERR_INVALID_ARG;
  *out = s->st;
  return WD_OK;
}

}  // extern "C"
