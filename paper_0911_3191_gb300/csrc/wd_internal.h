// Host-side internals shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/wilson_dirac.h"
#include "wd_device.cuh"

namespace wd {

// Device-resident state of one Krylov solve.  Every scalar of the iteration
// lives here, written by the finalisers of the fused reductions, so the loop
// needs no host round trip (Sec. 5: the whole solver runs on the GPU).
struct SolverCtl {
  double2 rho, rho_prev, alpha, omega, beta;  // BiCGstab (beta.x also CG's beta)
  double cg_alpha;   // CG step
  double rr;         // |r_hat|^2, the iterated residual (CG: normal residual)
  double rr_prev;    // CG: |r_hat|^2 of the previous iteration
  double maxr;       // M(r_hat) of Alg. 2: max |r_hat| since the last update
  double stop2;      // (tol |b|)^2, b the full source
  double delta;      // reliable-update threshold of Alg. 2
  double r2_true;    // |b_hat - M_hat x|^2 at the last reliable update
  double target2;    // CG: current target for the normal residual
  double neg_kappa2; // -kappa^2
  double kappa;      // kappa
  int iter;          // k + l of Alg. 2
  int max_iter;
  int updates;       // l of Alg. 2
  int status;        // wd_status
  int done;          // 1 once the loop must stop
  int do_update;     // 1 when this iteration ends with a reliable update
  int forced;        // the update was forced by apparent convergence or max_iter
  int in_graph;      // 1: running inside the solver graph (set the conditionals)
  int restart;       // 1: defect correction (Alg. 1): every update restarts the Krylov space
  int loops;         // WHILE-body executions, counted by the loop control kernel
  int pad;
  unsigned long long h_update;  // graph conditional handles (used when in_graph)
  unsigned long long h_loop;
};

struct Ctx;
struct BatchLaunch;
struct BatchBufs;

// Per-precision operations, one table per storage precision.
struct PrecOps {
  wd_prec prec;
  size_t (*field_bytes)(int stride);
  // S3: out = D in (plain) or out = x + a D in (xpay); a read from *a_dev if non-null
  void (*dslash)(const Ctx&, void* out, const void* in, int out_parity, int dagger, cudaStream_t);
  void (*dslash_xpay)(const Ctx&, void* out, const void* in, const void* x, double a, const double* a_dev,
                      int out_parity, int dagger, cudaStream_t);
  // S2 / S13: host-layout FP64 lexicographic field <-> single-parity field
  void (*import_lex)(const Ctx&, void* field, const double* lex_dev, int parity, cudaStream_t);
  void (*export_lex)(const Ctx&, double* lex_dev, const void* field, int parity, cudaStream_t);
  // S10: FP64 single-parity field <-> this precision
  void (*from_f64)(const Ctx&, void* out, const void* in_f64, cudaStream_t);
  void (*to_f64)(const Ctx&, void* out_f64, const void* in, cudaStream_t);
  void (*norm2)(const Ctx&, double* out_dev, const void* field, cudaStream_t);
  void (*zero)(const Ctx&, void* field, cudaStream_t);
  // S6 BiCGstab iteration and S9 reliable update with this inner precision
  void (*bicg_iteration)(const Ctx&, struct SolveBufs&, cudaStream_t);
  void (*bicg_update)(const Ctx&, struct SolveBufs&, cudaStream_t);
  // setup from the FP64 even residual src (b_hat, or b_hat - M_hat x0)
  void (*bicg_setup)(const Ctx&, struct SolveBufs&, const void* src, cudaStream_t);
  // S7 CG on the normal equations, and its reliable update
  void (*cg_iteration)(const Ctx&, struct SolveBufs&, cudaStream_t);
  void (*cg_update)(const Ctx&, struct SolveBufs&, cudaStream_t);
  void (*cg_setup)(const Ctx&, struct SolveBufs&, cudaStream_t);
  // S11: multi-RHS dslash and the batched BiCGstab with this inner precision
  void (*dslash_batch)(const Ctx&, const BatchLaunch&, void* out, const void* in, int parity, int dagger,
                       cudaStream_t);
  void (*batch_setup)(const Ctx&, const BatchLaunch&, BatchBufs&, cudaStream_t);
  void (*batch_iteration)(const Ctx&, const BatchLaunch&, BatchBufs&, cudaStream_t);
  void (*batch_update)(const Ctx&, const BatchLaunch&, BatchBufs&, cudaStream_t);
  // T-slab decomposition (Sec. 6): projected boundary faces, the link face
  // of the last slice, and the dslash of a slab region reading received halos
  size_t (*slab_face_bytes)(const Ctx&);
  size_t (*slab_link_face_bytes)(const Ctx&);
  void (*slab_pack_faces)(const Ctx&, void* lo, void* hi, const void* in, int dagger, cudaStream_t);
  void (*slab_pack_link_face)(const Ctx&, void* face, cudaStream_t);
  void (*slab_dslash)(const Ctx&, void* out, const void* in, const void* halo_lo, const void* halo_hi,
                      const void* link_halo, int flip_lo, int flip_hi, int parity, int dagger, int region,
                      cudaStream_t);
};

const PrecOps* ops_f64();
const PrecOps* ops_f32();
const PrecOps* ops_q16();
const PrecOps* ops_h16();
const PrecOps* ops_b16();
const PrecOps* prec_ops(int prec);

// Workspace of one solve.  FP64 fields (Alg. 2: source b_hat, solution x,
// residual r, and the odd temporary of the even-odd matrix) plus the inner
// precision fields (BiCGstab 7, CG 5; Sec. 5.3).
struct SolveBufs {
  SolverCtl* ctl;       // device
  void* b_hat;          // F64 even
  void* x;              // F64 even, the accumulated solution
  void* r;              // F64 even (CG: true residual before M_hat^dag)
  void* tmp64;          // F64 odd
  void* r_hat;          // inner: r_hat (BiCGstab: also s)
  void* r_tilde;        // inner: BiCGstab shadow residual
  void* p;              // inner
  void* v;              // inner: BiCGstab v, CG w
  void* t;              // inner: BiCGstab t
  void* x_hat;          // inner (or FP32, xhat_f32): solution since the last reliable update
  void* tmp;            // inner odd temporary
  int xhat_f32;         // x_hat kept in FP32 under a 16-bit inner precision
};

struct Ctx {
  Geom g;
  int dims[4];
  cudaStream_t stream;
  int device;
  int num_sms;
  // gauge copies (nullptr until loaded / derived)
  int recon;            // reals per FP64 link: 12 or 18
  int low_recon;        // FP32 / 16-bit link storage: 12 reals or 8 numbers (App. A.2)
  void* gauge[5];       // by wd_prec: F64 double2; F32 float4; 16-bit: uint4 part
  void* gauge4[5];      // 16-bit: uint2 part
  bool gauge_loaded;
  // temporal gauge (wd_load_gauge_opt): G(x) as [parity][9][stride] double2,
  // or nullptr; c.g.tfix is set with it
  double2* gfix;
  // reduction scratch
  RedScratch red;
  int max_red_blocks;
  double* scalars;      // small device scratch (API reductions)
  double* host_pinned;  // pinned host mirror of small results
  // workspace for the API
  void* tmp_odd[5];     // odd temporary per precision (apply_M)
  double* lex_staging;  // V x 24 doubles (host transfers)
  size_t lex_staging_bytes;
  // solver workspace
  SolveBufs sb;
  int sb_prec, sb_solver;
  void* sb_block;
  size_t sb_bytes;
  void* sb_full[2];     // F64 full fields for host solves (b, x)
  cudaGraphExec_t graph_exec;
  cudaGraph_t graph;
  int graph_prec, graph_solver, graph_xhat;
  unsigned long long graph_hu, graph_hl;  // conditional handles of the graph
  // batched solves (S11): workspace, graph and tuned launch shapes
  void* batch_block;
  size_t batch_bytes;
  int batch_n, batch_prec;
  void* batch_small;      // ctl array, BatchCtl, partials, kappas, scalars
  cudaGraphExec_t batch_exec;
  cudaGraph_t batch_graph;
  unsigned long long batch_hu, batch_hl;
  int batch_tr, batch_grid;  // tuned multi-RHS dslash shape for (batch_n, batch_prec);
                             // batch_tr 0: not tuned, -1: one system per block row
  int batch_pack;            // 1: two systems per thread (FP32x2 registers)
  double* batch_host;     // pinned mirror of per-system results
  std::string last_error;
};

void batch_release(Ctx& c);  // frees the batched-solve workspace (wd_solve_batch.cu)

// helpers
inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace wd

struct wd_ctx {
  wd::Ctx c;
};

// derive the gauge copy of precision prec from the FP64 copy if missing
wd_status wd_internal_ensure_gauge(wd_ctx* ctx, int prec);
// host FP64 field (host layout) <- two single-parity FP64 device fields
wd_status wd_internal_export_full(wd_ctx* ctx, double* host, const void* even, const void* odd);
wd_status wd_internal_import_full(wd_ctx* ctx, void* even, void* odd, const double* host);
wd_status wd_internal_export_full_async(wd_ctx* ctx, double* host, const void* even, const void* odd);
// wd_solve_device (BiCGstab) started from the even half of x_full instead of
// zero: the iteration begins with the FP64 residual b_hat - M_hat x0_e (a
// reliable update at iteration 0); the odd half of x_full is overwritten
wd_status wd_internal_solve_x0(wd_ctx* ctx, void* x_full, const void* b_full, double kappa,
                               const wd_solve_params* params, wd_solve_info* info);
