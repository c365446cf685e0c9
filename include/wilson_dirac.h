/*
 * wilson_dirac.h -- C ABI of the GB300 Wilson-Dirac library.
 *
 * Even-odd preconditioned Wilson-Dirac operator ("dslash"), and BiCGstab and
 * CG-on-the-normal-equations solvers with the reliable-update mixed-precision
 * scheme of Clark, Babich, Barros, Brower and Rebbi, "Solving lattice QCD
 * systems of equations using mixed precision solvers on GPUs"
 * (arXiv:0911.3191).  Section references below are to that paper.
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: dims = {X, Y, Z, T}, all even, X >= 2; V = XYZT, Vh = V/2.
 *   Site (x,y,z,t) has lexicographic index x + X(y + Y(z + Z t)) and parity
 *   (x+y+z+t) mod 2.  Direction mu = 0,1,2,3 <-> x,y,z,t (gamma_4 is the
 *   temporal one).  Boundaries are periodic; with t_antiperiodic every hop
 *   across t = T-1 <-> 0 carries a factor -1 (the paper leaves the boundary
 *   open; Sec. 4.3 mentions only a boundary surface term).
 * Host fields (FP64, DeGrand-Rossi spin basis, App. B):
 *   spinor: [site][spin 4][colour 3][re, im]  = 24 doubles per site
 *   gauge : [site][mu 4][row 3][col 3][re, im] = 72 doubles per site,
 *           U_mu(x) is the link from x to x + mu.
 * Device fields (internal layout, one parity, "single-parity field"): the
 *   Vh sites of one parity in even-odd order (Sec. 4.1), structure of arrays
 *   so that consecutive threads read consecutive 16-byte words:
 *     WD_F64 : 12 arrays of double2  (192 B/site)
 *     WD_F32 :  6 arrays of float4   ( 96 B/site)
 *     WD_Q16 :  3 arrays of 8 x int16 codes + 1 array of float norms (Sec. 4.6)
 *     WD_H16N:  3 arrays of 8 x fp16 + float norms
 *     WD_B16N:  3 arrays of 8 x bf16 + float norms       (52 B/site each)
 *   The byte size of one single-parity field is wd_field_bytes(ctx, prec).
 *   A "full field" is the even field followed by the odd field (2x bytes).
 *   16-bit storage: per site norm = max |f_k| over the 24 FP32 values f_k;
 *     Q16 code q_k = rint(f_k * (32767/norm)), value q_k * (norm/32767);
 *     H16N/B16N hold fp16/bf16(f_k / norm), value h_k * norm; norm 0 -> 0.
 *   Arithmetic on 16-bit fields is FP32; all global sums are FP64.
 * Operators (Sec. 3):
 *   D psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                   + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
 *   D^dag    = the same with the two projectors exchanged (= gamma5 D gamma5).
 *   M_kappa  = 1 - kappa D   (= 2 kappa times the paper's M, kappa = 1/(2(4+m)))
 *   M_hat    = 1 - kappa^2 D_eo D_oe on the even sites.
 *
 * Ownership and ordering: the context owns every device buffer it allocates
 * (gauge copies, solver workspace, staging); the caller owns the buffers it
 * passes in.  All work is ordered on the context's CUDA stream; calls that
 * return host results (wd_norm2, wd_solve*, host-side import/export)
 * synchronise that stream before returning.  A context is used by one host
 * thread at a time.
 *
 * Errors: every call returns a wd_status and never aborts the process;
 * wd_last_error(ctx) gives a one-line description of the last failure.
 */
#ifndef WILSON_DIRAC_H
#define WILSON_DIRAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_ctx wd_ctx;

typedef enum {
  WD_OK = 0,
  WD_ERR_INVALID_ARG = 1, /* bad pointer, size, enum or dims                 */
  WD_ERR_OOM = 2,         /* device allocation failed                        */
  WD_ERR_CUDA = 3,        /* a CUDA runtime call failed                      */
  WD_ERR_NOT_CONVERGED = 4, /* max_iter reached, or the reported FP64 true
                               residual above tol; x and info are still written */
  WD_ERR_BREAKDOWN = 5,   /* Krylov breakdown (rho, <r0,v> or <t,t> = 0)      */
  WD_ERR_NUMERIC = 6,     /* NaN or Inf met in a reduction                    */
  WD_ERR_TIMEOUT = 7,     /* a bounded device wait gave up                    */
  WD_ERR_BUDGET = 8,      /* request exceeds the configured memory budget     */
  WD_ERR_STATE = 9        /* call out of order (e.g. no gauge field loaded)   */
} wd_status;

typedef enum { WD_F64 = 0, WD_F32 = 1, WD_Q16 = 2, WD_H16N = 3, WD_B16N = 4 } wd_prec;
typedef enum { WD_BICGSTAB = 0, WD_CGNR = 1 } wd_solver;
typedef enum { WD_EVEN = 0, WD_ODD = 1 } wd_parity;
typedef enum { WD_M_FULL = 0, WD_M_SCHUR_EVEN = 1 } wd_operator;

/* Create a context for one lattice (Sec. 4.1: fields split by parity).
 * dims: {X,Y,Z,T}, each even and >= 2, with Vh < 2^31.  cuda_stream: a
 * cudaStream_t (NULL = the legacy default stream).  *out receives the handle. */
wd_status wd_create(wd_ctx **out, const int dims[4], int t_antiperiodic, void *cuda_stream);

/* Free every device buffer the context owns, then the context. NULL is allowed. */
wd_status wd_destroy(wd_ctx *ctx);

/* Change the stream later work is ordered on. */
wd_status wd_set_stream(wd_ctx *ctx, void *cuda_stream);

/* Bytes of one single-parity device field of precision prec (0 on bad args). */
size_t wd_field_bytes(const wd_ctx *ctx, wd_prec prec);

/* Load the gauge field (Sec. 3: SU(3) links U_mu(x)).  U: host layout above,
 * FP64, on the host (is_device = 0) or the device (is_device = 1).  recon =
 * 12 stores the first two rows of every link and rebuilds the third as
 * c = (a x b)^* (App. A.1; exact for SU(3) links); recon = 18 stores all
 * nine entries (FP64 only).  Lower-precision copies (FP32; Q16 codes
 * rint(u*32767); fp16; bf16) are derived from the FP64 copy on first use.
 * Replaces any previous gauge field. */
wd_status wd_load_gauge(wd_ctx *ctx, const double *U, int is_device, int recon);

/* Options of wd_load_gauge_opt (bitwise or). */
typedef enum {
  /* Sec. 4.3: load the links in the temporal gauge.  The library applies
   * G(x, t) = U_4(x, 0) U_4(x, 1) ... U_4(x, t-1) (G = 1 on t = 0),
   * U'_mu(x) = G(x) U_mu(x) G(x + mu)^dag; then every temporal link is the
   * unit matrix except on the last time slice t = T-1 (where U'_4 is the
   * product of U_4 around the time direction), and the dslash reads no
   * temporal link and does no temporal SU(3) multiply away from that slice.
   * Since D[U'] = G D[U] G^dag, the context's device fields hold G psi:
   * wd_field_import applies G (after the App. B basis change) and
   * wd_field_export applies G^dag, so every result seen through the host
   * layout is that of the untransformed U (to the FP64 rounding of G, about
   * 1e-15 relative).  G stays on the device (144 bytes per site, FP64). */
  WD_GAUGE_TEMPORAL = 1,
  /* App. A.2: the FP32 and 16-bit link copies hold 8 numbers per link
   * {arg a1, arg c1, a2, a3, b1} instead of 12 reals, and the kernels rebuild
   * the link from them (square roots and sine / cosine); the FP64 copy keeps
   * `recon` reals.  Links with |a1| = 1 (the parametrisation's singularity,
   * e.g. unit links) cannot be stored: the first use of a lower precision then
   * fails with WD_ERR_INVALID_ARG (temporal links of WD_GAUGE_TEMPORAL off the
   * last slice are never read and are exempt). */
  WD_GAUGE_RECON8 = 2
} wd_gauge_flags;

/* wd_load_gauge with options (flags: wd_gauge_flags, 0 = wd_load_gauge).
 * Device fields imported before this call belong to the previous gauge field
 * and must be imported again. */
wd_status wd_load_gauge_opt(wd_ctx *ctx, const double *U, int is_device, int recon, int flags);

/* Host <-> device field transfer with reorder and precision conversion
 * (Sec. 4.1 layout; Sec. 4.6 16-bit storage; App. B: fields cross in the
 * DeGrand-Rossi basis).  lex: V x 24 doubles, host (is_device = 0) or device.
 * Import reads the sites of `parity` from lex and writes the single-parity
 * device field `field`.  Export writes those sites of lex (others untouched). */
wd_status wd_field_import(wd_ctx *ctx, void *field, const double *lex, int is_device, wd_parity parity, wd_prec prec);
wd_status wd_field_export(wd_ctx *ctx, double *lex, const void *field, int is_device, wd_parity parity, wd_prec prec);

/* Dslash (Sec. 3, "the application of D to a spinor field"; Sec. 4):
 * out = D_{p,1-p} in (dagger: D^dag), where in is the single-parity field of
 * parity 1-p and out that of parity p = out_parity.  out and in must not
 * overlap.  Both fields are device fields of precision prec. */
wd_status wd_dslash(wd_ctx *ctx, void *out, const void *in, wd_parity out_parity, int dagger, wd_prec prec);

/* out = x + a * D_{p,1-p} in  (x of parity p; x may alias out). */
wd_status wd_dslash_xpay(wd_ctx *ctx, void *out, const void *in, const void *x, double a, wd_parity out_parity,
                         int dagger, wd_prec prec);

/* ---- T-slab domain decomposition (Sec. 6 names multi-GPU operation as the
 * next step).  A context created with dims {X, Y, Z, nt} holds one slab of a
 * lattice {X, Y, Z, T}: the nt time slices t0 .. t0 + nt - 1 of one rank, nt
 * even and t0 even, so local and global site parities agree.  Its links are
 * the slab's own (wd_load_gauge with the slab's sites; general links: no
 * temporal gauge, 12-real FP32 / 16-bit copies).  A dslash on the slab needs
 * from each time neighbour one boundary slice of the input spinor, projected
 * by the temporal hop's projector (1 -+ gamma_4): in the internal basis this
 * is a half spinor, 12 reals per site, the same half the temporal hop of the
 * stencil reads.  The first slice's backward hop also needs U_4 on the lower
 * neighbour's last slice (the "link face", once per gauge field).
 * The caller moves the faces between ranks (the Python binding uses
 * torch.distributed point-to-point messages: NCCL on GPUs, gloo on CPUs; with
 * one rank the halos are the rank's own opposite faces) into buffers in the
 * receiving GPU's own memory, and passes them to wd_dslash_slab.
 *
 * Face buffers are device buffers of wd_slab_face_bytes / wd_slab_link_face_bytes
 * bytes, owned by the caller.  Both sizes depend on the context's dims and,
 * for the link face, on its FP64 link storage (12 or 18 reals). */
size_t wd_slab_face_bytes(const wd_ctx *ctx, wd_prec prec);
size_t wd_slab_link_face_bytes(const wd_ctx *ctx, wd_prec prec);

/* Project the boundary slices of the single-parity input field `in` (the
 * field a following wd_dslash_slab reads):
 *   face_lo <- slice 0, for the lower neighbour's forward temporal hop,
 *   face_hi <- slice nt-1, for the upper neighbour's backward temporal hop,
 * each the half spinor that hop projects onto for D (dagger = 0) or D^dag.
 * Stored words are copied unchanged (16-bit codes keep their site norm). */
wd_status wd_slab_pack_faces(wd_ctx *ctx, void *face_lo, void *face_hi, const void *in, int dagger, wd_prec prec);

/* U_4 of the slab's last slice, both parities, in the precision-prec link
 * copy's own words, for the upper neighbour's link halo. */
wd_status wd_slab_pack_link_face(wd_ctx *ctx, void *link_face, wd_prec prec);

/* out = D_{p,1-p} in on the slab (dagger: D^dag), p = out_parity, for the
 * output sites of `region`: 0 = interior slices 1 .. nt-2 (needs no halo, so
 * it can run while the faces travel), 1 = the two boundary slices, 2 = all.
 * halo_lo: the lower neighbour's face_hi; halo_hi: the upper neighbour's
 * face_lo; link_halo: the lower neighbour's link face (all three may be NULL
 * for region 0).  flip_lo / flip_hi: nonzero when that halo crosses the
 * global t = T-1 <-> 0 boundary of an antiperiodic time direction (a factor
 * -1).  Errors: WD_ERR_INVALID_ARG for bad pointers, an odd or too small nt,
 * the temporal gauge or 8-number links. */
wd_status wd_dslash_slab(wd_ctx *ctx, void *out, const void *in, const void *halo_lo, const void *halo_hi,
                         const void *link_halo, int flip_lo, int flip_hi, wd_parity out_parity, int dagger,
                         wd_prec prec, int region);

/* Apply the Wilson-Dirac matrix (Sec. 3).  WD_M_FULL: out = M_kappa in on full
 * fields (even then odd).  WD_M_SCHUR_EVEN: out = M_hat in on even fields
 * (Sec. 3 Schur complement); the odd temporary is context workspace.
 * dagger applies M_kappa^dag / M_hat^dag.  out and in must not overlap. */
wd_status wd_apply_M(wd_ctx *ctx, void *out, const void *in, double kappa, wd_operator which, int dagger,
                     wd_prec prec);

/* |field|^2 over one single-parity field, summed in FP64 in a fixed order
 * (Sec. 5.1: global sums in double precision).  Result written to *result. */
wd_status wd_norm2(wd_ctx *ctx, double *result, const void *field, wd_prec prec);

typedef struct {
  double tol;          /* stop when |b - M x| <= tol |b| (FP64 true residual)      */
  double delta;        /* reliable-update threshold, ulp_inner < delta < 1 (Sec. 5.3) */
  int max_iter;        /* bound on inner iterations (reliable updates included)    */
  int solver;          /* wd_solver                                                */
  int inner_precision; /* wd_prec of the Krylov iteration; WD_F64 = pure FP64      */
  int use_graph;       /* 1: whole solve loop runs as one CUDA graph with device-side
                          conditional nodes; 0: host-driven loop                   */
  int restart;         /* 0: reliable updates (Alg. 2).  1: defect correction
                          (Alg. 1): each inner solve runs to eps_in = delta
                          relative to its starting residual, then x += p,
                          r = b - A x in FP64 and the Krylov iteration restarts
                          (not for batched solves; needs a lower inner precision) */
  int xhat_f32;        /* 1: x_hat, the solution accumulated between reliable
                          updates, is kept in FP32 when the inner precision is
                          16-bit (Sec. 5.3 keeps it in the inner precision, the
                          default 0); single solves only                        */
  int initial_guess;   /* 1: start from the x passed in (its even half; the odd
                          half is rebuilt from it): the accumulator holds x_e
                          and the first step is the FP64 residual b_hat -
                          M_hat x_e, a reliable update at iteration 0; an x
                          that already meets tol returns after no iteration.
                          BiCGstab with reliable updates (restart 0) only;
                          single solves only.  0 (default): start from zero */
} wd_solve_params;

typedef struct {
  int iters;                /* k + l of Alg. 2: iterations incl. reliable updates */
  int reliable_updates;     /* l                                                  */
  double true_rel_residual; /* |b - M x| / |b|, FP64, recomputed on the full lattice */
  double iterated_rel_residual; /* last iterated (inner) residual / |b|           */
  double seconds;           /* wall time of the call                             */
  int status;               /* wd_status of the solve                            */
  long long kernel_launches; /* kernels this call ran on the device (graph nodes included) */
} wd_solve_info;

/* Solve M_kappa x = b (Sec. 5): even-odd Schur system b_hat = b_e + kappa
 * D_eo b_o, M_hat x_e = b_hat by BiCGstab or CG on M_hat^dag M_hat, then
 * x_o = b_o + kappa D_oe x_e.  With inner_precision != WD_F64 the iteration
 * runs in that precision and the reliable-update scheme of Alg. 2 keeps the
 * solution x, the source and the true residual in FP64 (Sec. 5.3).
 * x, b: host FP64 fields in the host layout (V x 24 doubles).  On return x
 * holds the solution and *info is filled even when not converged (status
 * WD_ERR_NOT_CONVERGED / WD_ERR_BREAKDOWN / WD_ERR_NUMERIC).  WD_OK means
 * info->true_rel_residual, the full FP64 residual of the returned x, is at
 * most tol; the device loop stops on the Schur residual of its last reliable
 * update, and a returned x whose full residual is above tol gives
 * WD_ERR_NOT_CONVERGED (the same rule holds for the batched solves and the
 * server). */
wd_status wd_solve(wd_ctx *ctx, double *x, const double *b, double kappa, const wd_solve_params *params,
                   wd_solve_info *info);

/* As wd_solve, with x and b device FP64 full fields in the internal layout
 * (already resident on the device; no host transfer). */
wd_status wd_solve_device(wd_ctx *ctx, void *x, const void *b, double kappa, const wd_solve_params *params,
                          wd_solve_info *info);

/* Multi-right-hand-side dslash: out_r = D_{p,1-p} in_r (dagger: D^dag) for
 * r = 0..nrhs-1, 1 <= nrhs <= 256.  in and out each hold nrhs single-parity
 * fields of precision prec back to back (field r at byte offset
 * r * wd_field_bytes(ctx, prec)).  One launch: every link is read from device
 * memory once and applied to all right-hand sides (Sec. 3: one matrix, many
 * source vectors).  The launch shape is the one the autotuner chose for the
 * last batched solve of this nrhs and precision, else a default. */
wd_status wd_dslash_batch(wd_ctx *ctx, void *out, const void *in, int nrhs, wd_parity out_parity, int dagger,
                          wd_prec prec);

/* Solve M_kappa_r x_r = b_r for n systems sharing the loaded gauge field
 * (1 <= n <= 256), each with its own kappas[r] (host array): the 12
 * spin-colour sources of a propagator times several masses.  Even-odd Schur
 * BiCGstab with the reliable-update mixed precision of Alg. 2 (Sec. 5), all
 * systems in lockstep in one CUDA graph; converged systems stop doing work;
 * reliable updates are batched over the systems that need one.
 * params->solver must be WD_BICGSTAB.  The multi-RHS dslash shape (RHS tile
 * and grid) is chosen by timing on the first call for (lattice, precision,
 * n), and cached in the context and, when the environment variable
 * WD_TUNE_CACHE names a file, in that file.  infos[r] is filled for every
 * system; the return value is WD_OK when all converged, else the first
 * failing status.
 * wd_solve_batch_device: x and b are n FP64 full fields (even then odd, the
 *   internal layout) back to back, system r at byte offset
 *   r * 2 * wd_field_bytes(ctx, WD_F64).
 * wd_solve_batch: x[r], b[r] are host FP64 fields in the host layout. */
wd_status wd_solve_batch_device(wd_ctx *ctx, int n, void *x, const void *b, const double *kappas,
                                const wd_solve_params *params, wd_solve_info *infos);
wd_status wd_solve_batch(wd_ctx *ctx, int n, double *const *x, const double *const *b, const double *kappas,
                         const wd_solve_params *params, wd_solve_info *infos);

/* Multi-shift solve over kappa (beyond the paper, whose use case, Sec. 3, is
 * many solves on one gauge field): M_kappa_k x_k = b for one source and n
 * kappas (1 <= n <= 32) with one Krylov space.  With the seed kappa_s = the
 * largest kappa, M_hat(kappa_k) = (kappa_k / kappa_s)^2 (M_hat(kappa_s) +
 * tau_k), tau_k = (kappa_s / kappa_k)^2 - 1, a shifted family; the Schur
 * sources b_e + kappa_k D_eo b_o are combinations of b_e and D_eo b_o, each
 * solved for all shifts at once (a second family only when b_o != 0).  The
 * multi-shift BiCGstab runs in FP32 storage to a relative residual of 1e-7
 * (or tol if larger); each kappa is then finished by the solver of wd_solve
 * (params->inner_precision, Alg. 2) started from the multi-shift solution
 * (its first step the FP64 Schur residual of that solution) to the FP64 true
 * residual tol.  params->solver is not used (the refinement is BiCGstab).
 * x[k]: host FP64 fields in the host layout (V x 24 doubles), written; b:
 * host FP64 source; kappas: host array.  infos[k].iters counts the shared
 * multi-shift iterations plus that kappa's refinement iterations;
 * .seconds and .kernel_launches are those of the whole call.  Returns WD_OK
 * when every kappa reached tol, WD_ERR_NOT_CONVERGED otherwise (infos filled),
 * WD_ERR_BREAKDOWN / WD_ERR_NUMERIC when the shared iteration fails. */
wd_status wd_solve_multishift(wd_ctx *ctx, int n, double *const *x, const double *b, const double *kappas,
                              const wd_solve_params *params, wd_solve_info *infos);
/* As wd_solve_multishift with device fields in the internal layout: b one
 * FP64 full field (even then odd); x n FP64 full fields back to back, kappa k
 * at byte offset k * 2 * wd_field_bytes(ctx, WD_F64). */
wd_status wd_solve_multishift_device(wd_ctx *ctx, int n, void *x, const void *b, const double *kappas,
                                     const wd_solve_params *params, wd_solve_info *infos);

/* ---- Serving: continuous batching of solve requests ----------------------
 * A server keeps several gauge fields resident (possibly of different
 * lattice volumes), queues solve requests against them and runs them as
 * slots of batched, lockstep reliable-update BiCGstab solves (Sec. 5 and the
 * batched solver above).  Requests that arrive while others are running are
 * admitted at the next step as slots and memory free up; every device
 * allocation is charged against budget_bytes.  Each gauge field has its own
 * CUDA stream, so solves on different volumes overlap on the device.  A
 * request's iterates follow the same kernel sequence alone and in a mix. */
typedef struct wd_server wd_server;

typedef struct {
  size_t budget_bytes; /* device memory for gauge fields and solver slots; 0 = no limit */
  int max_slots;       /* concurrent solves per gauge field, 1..256                   */
  int iters_per_step;  /* lockstep iterations per wd_server_step between admissions   */
  int inner_precision; /* wd_prec of the inner iteration                              */
  double delta;        /* reliable-update threshold (Alg. 2)                          */
  int max_iter;        /* per request                                                 */
  int use_graph;       /* 1: each step's iterations run as one CUDA graph             */
  int gauge_flags;     /* wd_gauge_flags for every gauge field (wd_load_gauge_opt)    */
  int rhs_tile;        /* inner multi-RHS dslash: systems sharing a link tile (1, 2 or
                          4), -1 one system per block row, 0 chosen from the pool's
                          capacity                                                    */
} wd_server_params;

wd_status wd_server_create(wd_server **out, const wd_server_params *params);
wd_status wd_server_destroy(wd_server *server);

/* Make a gauge field resident (host layout, FP64; recon 12 or 18 as in
 * wd_load_gauge).  Its copies, staging, scratch and a prefetch buffer (one
 * host-layout FP64 field: the next queued request's source is uploaded into it
 * on a stream of its own while the field's current solves run) are charged
 * against the budget (WD_ERR_BUDGET if they do not fit).  *gauge_id names it
 * in requests. */
wd_status wd_server_add_gauge(wd_server *server, const int dims[4], int t_antiperiodic, const double *U, int recon,
                              int *gauge_id);

/* Queue M_kappa x = b to |b - M x| <= tol |b| on gauge field gauge_id.  b and
 * x are host FP64 fields in the host layout that the caller keeps alive until
 * the request has finished; x is written when it finishes.  The server
 * page-locks b and x (cudaHostRegister; buffers already page-locked are used
 * as they are) so that their transfers overlap other work, and releases them
 * when no unfinished request uses them.  Buffers allocated page-locked
 * (cudaHostAlloc) transfer fastest: on GB300 a registered 4 GB buffer moved at
 * 20-190 GB/s from copy to copy, an allocated one at 190 GB/s.  WD_ERR_BUDGET
 * if even one slot for this lattice can never fit the budget. */
wd_status wd_server_submit(wd_server *server, int gauge_id, const double *b, double *x, double kappa, double tol,
                           long long *request_id);

/* One scheduling round: retire the requests that finished during the previous
 * round (reconstruction, FP64 true residual, x copied out), release the slot
 * memory of idle gauge fields, admit queued requests into free slots within the
 * budget, then run up to iters_per_step lockstep iterations on every gauge field
 * with active slots (concurrently, one stream each) and wait for them.
 * *active / *queued receive the numbers of running and waiting requests. */
wd_status wd_server_step(wd_server *server, int *active, int *queued);

/* *finished = 1 and *info filled once the request has been retired. */
wd_status wd_server_poll(wd_server *server, long long request_id, int *finished, wd_solve_info *info);

/* Device bytes currently charged against the budget. */
size_t wd_server_memory_in_use(const wd_server *server);

/* Counters of a server since its creation: host seconds spent admitting
 * requests (source upload, Schur source, slot setup), retiring them (FP64
 * reconstruction, true residual, solution download) and waiting for a step
 * when no pool could progress; device seconds of the pools' steps (summed
 * over pools, which run concurrently); steps launched; requests admitted /
 * retired. */
typedef struct {
  double admit_seconds, retire_seconds, wait_seconds, gpu_step_seconds;
  long long steps, admitted, retired;
} wd_server_stats;
wd_status wd_server_get_stats(const wd_server *server, wd_server_stats *out);
/* Step trace: when the environment variable WD_SERVER_TRACE names a file at
 * wd_server_create, the server records every step (launch and completion
 * times, pool, capacity, active slots, admissions, device time of the step
 * and of the retire / download / upload / admission work before it) and
 * writes them as CSV to that file in wd_server_destroy. */
const char *wd_server_last_error(const wd_server *server);

/* |field|^2 of one single-parity device field, in FP64, for callers that
 * cannot allocate device memory.  (The paper has no counterpart; this is a
 * service of the library.)  Such callers -- code whose host framework owns all
 * device memory through its own pool and forbids allocations on its hot path,
 * or code about to capture its work into a CUDA graph -- cannot create a
 * wd_ctx, because wd_create allocates.  This call needs no context and
 * allocates nothing: the reduction's scratch (one partial sum per block plus a
 * ticket counter) is a static device array of the library, about 512 KB on
 * every GPU that loads it, kept until the process exits.
 *   result : DEVICE pointer to one double, written on `cuda_stream`; the call
 *            returns without synchronising, so read it after the stream.
 *   field  : single-parity device field of precision prec for lattice dims
 *            (layout as above).
 *   dims   : {X,Y,Z,T}, each even and >= 2, with at most 16,777,216 sites per
 *            parity (the scratch holds 65,536 partial sums of 256 sites);
 *            larger lattices are rejected with WD_ERR_INVALID_ARG.
 *   err    : optional buffer of err_len bytes for a one-line error message.
 * The first call in each CUDA context (the device's primary context for
 * runtime-API callers; a driver-API caller's own context; a new primary
 * context after cudaDeviceReset) looks up the scratch address in that context
 * and caches it under the context's unique id; make that first call before
 * any stream capture.  All calls share the scratch, whose counter is cleared
 * on the stream before each launch: calls that overlap on the GPU (other
 * streams, other host threads) race and must not be issued.
 * Errors: WD_ERR_INVALID_ARG for null pointers, a bad precision, odd or too
 * large dims (nothing is launched); WD_ERR_CUDA when no context can be made
 * current or a launch fails. */
wd_status wd_norm2_noalloc(double *result, const void *field, const int dims[4], wd_prec prec, void *cuda_stream,
                           char *err, size_t err_len);

/* Description of the last failure on ctx ("" if none); static string for NULL. */
const char *wd_last_error(const wd_ctx *ctx);
const char *wd_status_string(wd_status s);

#ifdef __cplusplus
}
#endif
#endif /* WILSON_DIRAC_H */
