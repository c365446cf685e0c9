// C ABI of the Wilson-Dirac library (declared in include/wilson_dirac.h).
//
// The context owns the gauge copies, the reduction scratch and the solver
// workspace; all work is ordered on the context's stream.  The solver loop
// (Alg. 2 of Sec. 5.3 around BiCGstab or CG, Sec. 5.1) runs either as one
// CUDA graph -- a WHILE conditional node whose body is one Krylov iteration
// followed by an IF conditional node holding the FP64 reliable update, both
// conditions set on the device by the reduction finalisers -- or, with
// use_graph = 0, as a host loop that reads the device control block each
// iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cstdlib>
#include <fstream>
#include <sstream>

#include "wd_batch.cuh"

namespace wd {

// Last node of the WHILE body: continue while not done.  The body count is
// bounded here on its own (max_iter + 16 executions), whatever the
// finalisers did, so the device loop always terminates.
__global__ void loop_control_kernel(SolverCtl* ctl) {
  ctl->loops += 1;
  if (ctl->loops > ctl->max_iter + 16 && !ctl->done) {
    ctl->done = 1;
    if (ctl->status == WD_OK) ctl->status = WD_ERR_NOT_CONVERGED;
  }
  if (ctl->in_graph) cudaGraphSetConditional((cudaGraphConditionalHandle)ctl->h_loop, ctl->done ? 0u : 1u);
}

__global__ void init_ctl_kernel(SolverCtl* ctl, double tol, double delta, int max_iter, double kappa,
                                const double* bnorm2, int in_graph, unsigned long long h_update,
                                unsigned long long h_loop, int restart) {
  SolverCtl c;
  memset(&c, 0, sizeof(c));
  const double one = 1.0;
  c.rho = c.rho_prev = c.alpha = c.omega = make_double2(one, 0.0);
  c.beta = make_double2(0.0, 0.0);
  c.stop2 = tol * tol * (bnorm2[0] + bnorm2[1]);
  c.delta = delta;
  c.kappa = kappa;
  c.neg_kappa2 = -kappa * kappa;
  c.max_iter = max_iter;
  c.status = WD_OK;
  c.in_graph = in_graph;
  c.restart = restart;
  c.h_update = h_update;
  c.h_loop = h_loop;
  *ctl = c;
}

// an initial guess that meets the tolerance: no iteration
__global__ void mark_done_kernel(SolverCtl* ctl) {
  ctl->status = WD_OK;
  ctl->done = 1;
}

// ---- gauge field: host layout -> even-odd structure of arrays (S1)
__global__ void gauge_pack_f64_kernel(Geom g, const double* lex, double2* out, int nc) {
  const int n = 2 * g.Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int parity = i / g.Vh, h = i - parity * g.Vh;
    int x, y, z, t;
    site_coords(g, h, parity, x, y, z, t);
    const size_t s = (size_t)x + (size_t)g.X * (y + (size_t)g.Y * (z + (size_t)g.Z * t));
    for (int mu = 0; mu < 4; ++mu) {
      const double2* src = reinterpret_cast<const double2*>(lex + (s * 4 + mu) * 18);
      double2* dst = out + (size_t)(parity * 4 + mu) * nc * g.stride + h;
      for (int c = 0; c < nc; ++c) dst[(size_t)c * g.stride] = src[c];
    }
  }
}

// ---- temporal gauge (Sec. 4.3), FP64 on the host-layout links in place.
// 3x3 complex, row-major: c = a b, c = a b^dag.
__device__ __forceinline__ void m3_mul(const double2* a, const double2* b, double2* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double2 x = a[i * 3 + k], y = b[k * 3 + j];
        re += x.x * y.x;
        re -= x.y * y.y;
        im += x.x * y.y;
        im += x.y * y.x;
      }
      c[i * 3 + j] = make_double2(re, im);
    }
}
__device__ __forceinline__ void m3_mul_dag(const double2* a, const double2* b, double2* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < 3; ++k) {  // a_ik conj(b_jk)
        const double2 x = a[i * 3 + k], y = b[j * 3 + k];
        re += x.x * y.x;
        re += x.y * y.y;
        im += x.y * y.x;
        im -= x.x * y.y;
      }
      c[i * 3 + j] = make_double2(re, im);
    }
}

// G(x, 0) = 1, G(x, t + 1) = G(x, t) U_4(x, t): one thread per spatial site
// walks the time direction.  G: [lexicographic site][9].
__global__ void temporal_gauge_g_kernel(Geom g, const double* lex, double2* G) {
  const long long ns = (long long)g.X * g.Y * g.Z;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < ns;
       s += (long long)gridDim.x * blockDim.x) {
    double2 m[9], n[9];
    for (int k = 0; k < 9; ++k) m[k] = make_double2((k % 4 == 0) ? 1.0 : 0.0, 0.0);
    for (int t = 0; t < g.T; ++t) {
      const size_t site = (size_t)s + (size_t)ns * t;
      for (int k = 0; k < 9; ++k) G[site * 9 + k] = m[k];
      if (t + 1 < g.T) {
        m3_mul(m, reinterpret_cast<const double2*>(lex + (site * 4 + 3) * 18), n);
        for (int k = 0; k < 9; ++k) m[k] = n[k];
      }
    }
  }
}

// U'_mu(x) = G(x) U_mu(x) G(x + mu)^dag: the temporal links become 1 except
// on t = T-1, where U'_4 = G(x, T-1) U_4(x, T-1) (G(x, 0) = 1).
__global__ void temporal_gauge_apply_kernel(Geom g, double* lex, const double2* G) {
  const size_t V = (size_t)2 * g.Vh;
  for (size_t site = blockIdx.x * (size_t)blockDim.x + threadIdx.x; site < V; site += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(site % g.X);
    const int y = (int)((site / g.X) % g.Y);
    const int z = (int)((site / ((size_t)g.X * g.Y)) % g.Z);
    const int t = (int)(site / ((size_t)g.X * g.Y * g.Z));
    const size_t step[3] = {1, (size_t)g.X, (size_t)g.X * g.Y};
    const bool last[3] = {x == g.X - 1, y == g.Y - 1, z == g.Z - 1};
    const size_t wrap[3] = {(size_t)(g.X - 1), (size_t)(g.Y - 1) * g.X, (size_t)(g.Z - 1) * g.X * g.Y};
    const double2* gx = G + site * 9;
    double2 tmp[9], out[9];
    for (int mu = 0; mu < 3; ++mu) {
      const size_t nb = last[mu] ? site - wrap[mu] : site + step[mu];
      double2* u = reinterpret_cast<double2*>(lex + (site * 4 + mu) * 18);
      m3_mul(gx, u, tmp);
      m3_mul_dag(tmp, G + nb * 9, out);
      for (int k = 0; k < 9; ++k) u[k] = out[k];
    }
    double2* u4 = reinterpret_cast<double2*>(lex + (site * 4 + 3) * 18);
    if (t == g.T - 1) {
      m3_mul(gx, u4, out);
      for (int k = 0; k < 9; ++k) u4[k] = out[k];
    } else {
      for (int k = 0; k < 9; ++k) u4[k] = make_double2((k % 4 == 0) ? 1.0 : 0.0, 0.0);
    }
  }
}

// G (lexicographic) -> [parity][9][stride] at even-odd indices
__global__ void temporal_gauge_pack_kernel(Geom g, const double2* G, double2* out) {
  const int n = 2 * g.Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int parity = i / g.Vh, h = i - parity * g.Vh;
    int x, y, z, t;
    site_coords(g, h, parity, x, y, z, t);
    const size_t s = (size_t)x + (size_t)g.X * (y + (size_t)g.Y * (z + (size_t)g.Z * t));
    for (int k = 0; k < 9; ++k) out[(size_t)(parity * 9 + k) * g.stride + h] = G[s * 9 + k];
  }
}

// FP64 copy (first two rows) -> FP32 / 16-bit copies
__global__ void gauge_f64_to_f32_kernel(Geom g, const double2* in, int nc, float4* out) {
  const int n = 8 * g.Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int pm = i / g.Vh, h = i - pm * g.Vh;
    double r[12];
    for (int c = 0; c < 6; ++c) {
      double2 d = in[((size_t)pm * nc + c) * g.stride + h];
      r[2 * c] = d.x;
      r[2 * c + 1] = d.y;
    }
    for (int c = 0; c < 3; ++c)
      out[((size_t)pm * 3 + c) * g.stride + h] =
          make_float4(__double2float_rn(r[4 * c]), __double2float_rn(r[4 * c + 1]), __double2float_rn(r[4 * c + 2]),
                      __double2float_rn(r[4 * c + 3]));
  }
}

template <Fmt16 F>
__device__ __forceinline__ uint32_t link16(double u) {
  const float f = __double2float_rn(u);
  if constexpr (F == Fmt16::Q16) return (uint32_t)(uint16_t)(int16_t)rintf(__fmul_rn(f, 32767.f));
  else if constexpr (F == Fmt16::H16) return (uint32_t)__half_as_ushort(__float2half_rn(f));
  else return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f));
}

template <Fmt16 F>
__global__ void gauge_f64_to_16_kernel(Geom g, const double2* in, int nc, uint4* out8, uint2* out4) {
  const int n = 8 * g.Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int pm = i / g.Vh, h = i - pm * g.Vh;
    uint32_t w[6];
    for (int c = 0; c < 6; ++c) {
      double2 d = in[((size_t)pm * nc + c) * g.stride + h];
      w[c] = link16<F>(d.x) | (link16<F>(d.y) << 16);
    }
    out8[(size_t)pm * g.stride + h] = make_uint4(w[0], w[1], w[2], w[3]);
    out4[(size_t)pm * g.stride + h] = make_uint2(w[4], w[5]);
  }
}

// Batch loop control, last node of the batched WHILE body: continue while a
// system is unconverged; bounded on its own at max_iter + 16 executions.
__global__ void batch_loop_control_kernel(BatchCtl* bc, const SolverCtl* ctl_in, int nrhs) {
  SolverCtl* ctl = const_cast<SolverCtl*>(ctl_in);
  int all = 1;
  for (int r = 0; r < nrhs; ++r)
    if (!ctl[r].done) all = 0;
  bc->loops += 1;
  bc->step_loops += 1;
  if (!all && bc->loops > bc->max_loops) {
    for (int r = 0; r < nrhs; ++r)
      if (!ctl[r].done) {
        ctl[r].done = 1;
        if (ctl[r].status == WD_OK) ctl[r].status = WD_ERR_NOT_CONVERGED;
      }
    all = 1;
  }
  bc->all_done = all;
  const int cont = !all && bc->step_loops < bc->step_limit;
  if (bc->in_graph) cudaGraphSetConditional((cudaGraphConditionalHandle)bc->h_loop, cont ? 1u : 0u);
}

__global__ void batch_init_kernel(SolverCtl* ctl, BatchCtl* bc, int nrhs, double tol, double delta, int max_iter,
                                  const double* kappas, const double* bnorm2, int in_graph,
                                  unsigned long long h_update, unsigned long long h_loop) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrhs) {
    SolverCtl c;
    memset(&c, 0, sizeof(c));
    c.rho = c.rho_prev = c.alpha = c.omega = make_double2(1.0, 0.0);
    c.beta = make_double2(0.0, 0.0);
    const double b2 = bnorm2[r] + bnorm2[nrhs + r];
    c.stop2 = tol * tol * b2;
    c.delta = delta;
    c.kappa = kappas[r];
    c.neg_kappa2 = -kappas[r] * kappas[r];
    c.max_iter = max_iter;
    c.status = WD_OK;
    if (!isfinite(b2)) {
      c.status = WD_ERR_NUMERIC;
      c.done = 1;
    } else if (b2 == 0.0) {
      c.done = 1;  // zero source: x = 0
    }
    ctl[r] = c;
  }
  if (r == 0) {
    for (int k = 0; k < 4; ++k) bc->counter[k] = 0;
    bc->any_update = 0;
    bc->all_done = 0;
    bc->in_graph = in_graph;
    bc->loops = 0;
    bc->max_loops = max_iter + 16;
    bc->step_loops = 0;
    bc->step_limit = max_iter + 16;
    bc->h_update = h_update;
    bc->h_loop = h_loop;
  }
}

const PrecOps* prec_ops(int p) {
  switch (p) {
    case WD_F64: return ops_f64();
    case WD_F32: return ops_f32();
    case WD_Q16: return ops_q16();
    case WD_H16N: return ops_h16();
    case WD_B16N: return ops_b16();
    default: return nullptr;
  }
}

}  // namespace wd

using namespace wd;

namespace {

wd_status set_err(wd_ctx* ctx, wd_status st, const std::string& msg) {
  if (ctx) ctx->c.last_error = msg;
  return st;
}

wd_status cuda_err(wd_ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_err(ctx, e == cudaErrorMemoryAllocation ? WD_ERR_OOM : WD_ERR_CUDA, m);
}

#define WD_CK(ctx, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call); \
  } while (0)

#define WD_CK_LAUNCH(ctx, what) WD_CK(ctx, (cudaPeekAtLastError(), cudaGetLastError()))

bool valid_prec(int p) { return p >= WD_F64 && p <= WD_B16N; }

size_t field_bytes(const Ctx& c, int prec) { return prec_ops(prec)->field_bytes(c.g.stride); }

template <class T>
wd_status dev_alloc(wd_ctx* ctx, T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return WD_OK;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_err(ctx, e, "cudaMalloc");
  }
  return WD_OK;
}

void dev_free(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

int grid_for(const Ctx& c, int n, int block) {
  int b = (n + block - 1) / block;
  int cap = c.num_sms * 8;
  return b < cap ? b : cap;
}

// FP64 copy -> the 8 numbers of App. A.2 per link: {arg a1, arg c1, a2, a3,
// b1}.  FP32: two float4 [p][mu][2][stride]; 16-bit: one uint4 [p][mu][stride],
// the angles as fixed-point codes rint(32767 angle / pi) in every 16-bit
// format, a2, a3, b1 in the format's own encoding.  Counts in *nsing
// the links that the dslash reads and that sit at the parametrisation's
// singularity |a1| = 1 (N = sqrt(|a2|^2 + |a3|^2) below 1e-6); temporal links
// of the temporal gauge off the last slice are never read.
template <int P>
__global__ void gauge_f64_to_8_kernel(Geom g, const double2* in, int nc, void* out, unsigned* nsing) {
  const int n = 8 * g.Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int pm = i / g.Vh, h = i - pm * g.Vh;
    const int parity = pm >> 2, mu = pm & 3;
    double2 r[6];
    for (int c = 0; c < 6; ++c) r[c] = in[((size_t)pm * nc + c) * g.stride + h];
    double2 c1;
    if (nc == 9) {
      c1 = in[((size_t)pm * nc + 6) * g.stride + h];
    } else {  // c1 = conj(a2 b3 - a3 b2)
      const double re = r[1].x * r[5].x - r[1].y * r[5].y - (r[2].x * r[4].x - r[2].y * r[4].y);
      const double im = r[1].x * r[5].y + r[1].y * r[5].x - (r[2].x * r[4].y + r[2].y * r[4].x);
      c1 = make_double2(re, -im);
    }
    const double n2 = r[1].x * r[1].x + r[1].y * r[1].y + r[2].x * r[2].x + r[2].y * r[2].y;
    int x, y, z, t;
    site_coords(g, h, parity, x, y, z, t);
    const bool read = !(g.tfix && mu == 3 && t != g.T - 1);
    if (read && n2 < 1e-12) atomicAdd(nsing, 1u);
    const double q[8] = {atan2(r[0].y, r[0].x), atan2(c1.y, c1.x), r[1].x, r[1].y, r[2].x, r[2].y, r[3].x, r[3].y};
    if constexpr (P == WD_F32) {
      float4* o = reinterpret_cast<float4*>(out);
      o[((size_t)pm * 2) * g.stride + h] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
      o[((size_t)pm * 2 + 1) * g.stride + h] = make_float4((float)q[4], (float)q[5], (float)q[6], (float)q[7]);
    } else {
      constexpr Fmt16 F = (P == WD_Q16) ? Fmt16::Q16 : (P == WD_H16N) ? Fmt16::H16 : Fmt16::B16;
      const double ip = 0.31830988618379067154;  // 1/pi
      uint32_t w[4];
      // the angles as 16-bit fixed point in every format, the rest in the format's own
      w[0] = link16<Fmt16::Q16>(q[0] * ip) | (link16<Fmt16::Q16>(q[1] * ip) << 16);
      for (int k = 1; k < 4; ++k) w[k] = link16<F>(q[2 * k]) | (link16<F>(q[2 * k + 1]) << 16);
      reinterpret_cast<uint4*>(out)[(size_t)pm * g.stride + h] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

wd_status ensure_gauge(wd_ctx* ctx, int prec) {
  Ctx& c = ctx->c;
  if (!c.gauge_loaded) return set_err(ctx, WD_ERR_STATE, "no gauge field loaded (call wd_load_gauge first)");
  if (c.gauge[prec]) return WD_OK;
  const size_t links = (size_t)8 * c.g.stride;
  const int nc = c.recon / 2;
  const double2* src = (const double2*)c.gauge[WD_F64];
  const int grid = grid_for(c, 8 * c.g.Vh, 256);
  wd_status st;
  if (c.low_recon == 8 && prec != WD_F64) {
    const size_t bytes = links * (prec == WD_F32 ? 2 * sizeof(float4) : sizeof(uint4));
    if ((st = dev_alloc(ctx, &c.gauge[prec], bytes)) != WD_OK) return st;
    unsigned* nsing = reinterpret_cast<unsigned*>(c.scalars);
    WD_CK(ctx, cudaMemsetAsync(nsing, 0, sizeof(unsigned), c.stream));
    if (prec == WD_F32) gauge_f64_to_8_kernel<WD_F32><<<grid, 256, 0, c.stream>>>(c.g, src, nc, c.gauge[prec], nsing);
    else if (prec == WD_Q16) gauge_f64_to_8_kernel<WD_Q16><<<grid, 256, 0, c.stream>>>(c.g, src, nc, c.gauge[prec], nsing);
    else if (prec == WD_H16N) gauge_f64_to_8_kernel<WD_H16N><<<grid, 256, 0, c.stream>>>(c.g, src, nc, c.gauge[prec], nsing);
    else gauge_f64_to_8_kernel<WD_B16N><<<grid, 256, 0, c.stream>>>(c.g, src, nc, c.gauge[prec], nsing);
    WD_CK_LAUNCH(ctx, "gauge conversion (8 numbers)");
    unsigned h_nsing = 0;
    WD_CK(ctx, cudaMemcpyAsync(&h_nsing, nsing, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    WD_CK(ctx, cudaStreamSynchronize(c.stream));
    if (h_nsing) {
      dev_free(c.gauge[prec]);
      return set_err(ctx, WD_ERR_INVALID_ARG,
                     "8-number link storage: " + std::to_string(h_nsing) +
                         " links have |a1| = 1 (the parametrisation's singularity, App. A.2)");
    }
    return WD_OK;
  }
  if (prec == WD_F32) {
    if ((st = dev_alloc(ctx, &c.gauge[prec], links * 3 * sizeof(float4))) != WD_OK) return st;
    gauge_f64_to_f32_kernel<<<grid, 256, 0, c.stream>>>(c.g, src, nc, (float4*)c.gauge[prec]);
  } else {
    if ((st = dev_alloc(ctx, &c.gauge[prec], links * sizeof(uint4))) != WD_OK) return st;
    if ((st = dev_alloc(ctx, &c.gauge4[prec], links * sizeof(uint2))) != WD_OK) return st;
    uint4* o8 = (uint4*)c.gauge[prec];
    uint2* o4 = (uint2*)c.gauge4[prec];
    if (prec == WD_Q16) gauge_f64_to_16_kernel<Fmt16::Q16><<<grid, 256, 0, c.stream>>>(c.g, src, nc, o8, o4);
    else if (prec == WD_H16N) gauge_f64_to_16_kernel<Fmt16::H16><<<grid, 256, 0, c.stream>>>(c.g, src, nc, o8, o4);
    else gauge_f64_to_16_kernel<Fmt16::B16><<<grid, 256, 0, c.stream>>>(c.g, src, nc, o8, o4);
  }
  WD_CK_LAUNCH(ctx, "gauge conversion");
  return WD_OK;
}

wd_status ensure_staging(wd_ctx* ctx) {
  Ctx& c = ctx->c;
  const size_t need = (size_t)2 * c.g.Vh * 24 * sizeof(double);
  if (c.lex_staging && c.lex_staging_bytes >= need) return WD_OK;
  dev_free((void*&)c.lex_staging);
  wd_status st = dev_alloc(ctx, &c.lex_staging, need);
  c.lex_staging_bytes = st == WD_OK ? need : 0;
  return st;
}

wd_status ensure_tmp_odd(wd_ctx* ctx, int prec) {
  Ctx& c = ctx->c;
  if (c.tmp_odd[prec]) return WD_OK;
  return dev_alloc(ctx, &c.tmp_odd[prec], field_bytes(c, prec));
}

void destroy_graph(Ctx& c) {
  if (c.graph_exec) cudaGraphExecDestroy(c.graph_exec);
  if (c.graph) cudaGraphDestroy(c.graph);
  c.graph_exec = nullptr;
  c.graph = nullptr;
  c.graph_prec = c.graph_solver = -1;
}

// workspace of one solve (Sec. 5.3 field count: 4 FP64 + 7 / 5 inner fields)
wd_status ensure_solver(wd_ctx* ctx, int solver, int prec) {
  Ctx& c = ctx->c;
  if (c.sb_block && c.sb_prec == prec && c.sb_solver == solver) return WD_OK;
  destroy_graph(c);
  dev_free(c.sb_block);
  if (!c.sb.ctl) {
    wd_status st = dev_alloc(ctx, &c.sb.ctl, sizeof(SolverCtl));
    if (st != WD_OK) return st;
  }
  const size_t f64 = field_bytes(c, WD_F64), fin = field_bytes(c, prec);
  const size_t fx = std::max(fin, field_bytes(c, WD_F32));  // x_hat may be FP32
  const int n_inner = (solver == WD_BICGSTAB) ? 7 : 5;
  c.sb_bytes = 4 * f64 + (n_inner - 1) * fin + fx;
  wd_status st = dev_alloc(ctx, &c.sb_block, c.sb_bytes);
  if (st != WD_OK) return st;
  char* p = (char*)c.sb_block;
  c.sb.b_hat = p; p += f64;
  c.sb.x = p; p += f64;
  c.sb.r = p; p += f64;
  c.sb.tmp64 = p; p += f64;
  c.sb.r_hat = p; p += fin;
  c.sb.p = p; p += fin;
  c.sb.v = p; p += fin;
  c.sb.x_hat = p; p += fx;
  c.sb.tmp = p; p += fin;
  if (solver == WD_BICGSTAB) {
    c.sb.r_tilde = p; p += fin;
    c.sb.t = p; p += fin;
  } else {
    c.sb.r_tilde = nullptr;
    c.sb.t = nullptr;
  }
  c.sb_prec = prec;
  c.sb_solver = solver;
  return WD_OK;
}

cudaGraphNodeParams make_conditional_params() {
  union Raw {
    cudaGraphNodeParams p;
    unsigned char bytes[sizeof(cudaGraphNodeParams)];
    Raw() { memset(bytes, 0, sizeof(bytes)); }
  } raw;
  return raw.p;
}

// WHILE(!done) { iteration; IF(update) { reliable update }; loop control }
wd_status build_graph(wd_ctx* ctx, int solver, int prec, unsigned long long* h_update, unsigned long long* h_loop) {
  Ctx& c = ctx->c;
  const PrecOps* ops = prec_ops(prec);
  cudaGraph_t g = nullptr;
  WD_CK(ctx, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hl, hu;
  WD_CK(ctx, cudaGraphConditionalHandleCreate(&hl, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp = make_conditional_params();
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hl;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  WD_CK(ctx, cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  WD_CK(ctx, cudaGraphConditionalHandleCreate(&hu, body, 0, cudaGraphCondAssignDefault));

  cudaStream_t cs;
  WD_CK(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t unused;
  // the Krylov iteration
  WD_CK(ctx, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  if (solver == WD_BICGSTAB) ops->bicg_iteration(c, c.sb, cs);
  else ops->cg_iteration(c, c.sb, cs);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  WD_CK(ctx, cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
  WD_CK(ctx, cudaStreamEndCapture(cs, &unused));
  // IF(update) { reliable update }
  cudaGraphNodeParams ip = make_conditional_params();
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hu;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  WD_CK(ctx, cudaGraphAddNode(&inode, body, tail.data(), nullptr, tail.size(), &ip));
  cudaGraph_t ubody = ip.conditional.phGraph_out[0];
  WD_CK(ctx, cudaStreamBeginCaptureToGraph(cs, ubody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  if (solver == WD_BICGSTAB) ops->bicg_update(c, c.sb, cs);
  else ops->cg_update(c, c.sb, cs);
  WD_CK(ctx, cudaStreamEndCapture(cs, &unused));
  // loop control
  WD_CK(ctx, cudaStreamBeginCaptureToGraph(cs, body, &inode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  loop_control_kernel<<<1, 1, 0, cs>>>(c.sb.ctl);
  WD_CK(ctx, cudaStreamEndCapture(cs, &unused));
  WD_CK(ctx, cudaStreamDestroy(cs));
  cudaGraphExec_t exec;
  WD_CK(ctx, cudaGraphInstantiate(&exec, g, 0));
  c.graph = g;
  c.graph_exec = exec;
  c.graph_prec = prec;
  c.graph_solver = solver;
  c.graph_xhat = c.sb.xhat_f32;
  *h_update = hu;
  *h_loop = hl;
  return WD_OK;
}

wd_status solve_device(wd_ctx* ctx, void* x_full, const void* b_full, double kappa, const wd_solve_params* prm,
                       wd_solve_info* info, bool x0 = false) {
  Ctx& c = ctx->c;
  const auto t0 = std::chrono::steady_clock::now();
  wd_solve_params p{1e-10, 0.1, 10000, WD_BICGSTAB, WD_F64, 1, 0, 0};
  if (prm) p = *prm;
  if (!valid_prec(p.inner_precision)) return set_err(ctx, WD_ERR_INVALID_ARG, "bad inner_precision");
  if (p.xhat_f32 != 0 && p.xhat_f32 != 1) return set_err(ctx, WD_ERR_INVALID_ARG, "xhat_f32 must be 0 or 1");
  if (p.restart && p.inner_precision == WD_F64)
    return set_err(ctx, WD_ERR_INVALID_ARG, "defect correction needs a lower inner precision");
  if (p.solver != WD_BICGSTAB && p.solver != WD_CGNR) return set_err(ctx, WD_ERR_INVALID_ARG, "bad solver");
  if (p.initial_guess != 0 && p.initial_guess != 1)
    return set_err(ctx, WD_ERR_INVALID_ARG, "initial_guess must be 0 or 1");
  x0 = x0 || p.initial_guess;
  if (x0 && (p.solver != WD_BICGSTAB || p.restart))
    return set_err(ctx, WD_ERR_INVALID_ARG, "an initial guess needs BiCGstab with reliable updates");
  if (!(p.tol > 0.0) || p.max_iter <= 0) return set_err(ctx, WD_ERR_INVALID_ARG, "bad tol or max_iter");
  if (p.inner_precision == WD_F64) p.delta = 0.0;  // pure FP64: update only to confirm convergence
  else if (!(p.delta > 0.0 && p.delta < 1.0)) return set_err(ctx, WD_ERR_INVALID_ARG, "delta must be in (0,1)");
  wd_status st;
  if ((st = ensure_gauge(ctx, WD_F64)) != WD_OK) return st;
  if ((st = ensure_gauge(ctx, p.inner_precision)) != WD_OK) return st;
  if ((st = ensure_solver(ctx, p.solver, p.inner_precision)) != WD_OK) return st;
  const PrecOps* o64 = ops_f64();
  const PrecOps* oin = prec_ops(p.inner_precision);
  SolveBufs& sb = c.sb;
  sb.xhat_f32 = p.xhat_f32;
  cudaStream_t s = c.stream;
  const size_t f64 = field_bytes(c, WD_F64);
  const char* b_e = (const char*)b_full;
  const char* b_o = b_e + f64;
  char* x_e = (char*)x_full;
  char* x_o = x_e + f64;

  // |b|^2 (both parities), b_hat = b_e + kappa D_eo b_o, |b_hat|^2
  o64->norm2(c, c.scalars + 0, b_e, s);
  o64->norm2(c, c.scalars + 1, b_o, s);
  // a source without odd sites (an even-site point source) has b_hat = b_e
  // exactly: its D_eo b_o is skipped
  WD_CK(ctx, cudaMemcpyAsync(c.host_pinned + 1, c.scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  WD_CK(ctx, cudaStreamSynchronize(s));
  const bool odd_zero = c.host_pinned[1] == 0.0;
  if (odd_zero) WD_CK(ctx, cudaMemcpyAsync(sb.b_hat, b_e, f64, cudaMemcpyDeviceToDevice, s));
  else o64->dslash_xpay(c, sb.b_hat, b_o, b_e, kappa, nullptr, 0, 0, s);
  o64->norm2(c, c.scalars + 2, sb.b_hat, s);
  const void* setup_src = sb.b_hat;
  if (x0) {
    // start from x0_e: the accumulator holds it and the iteration starts from
    // r0 = b_hat - M_hat x0_e in FP64 (tmp64 = D_oe x0_e, then the even rows),
    // kept in the FP64 residual buffer, which BiCGstab does not use otherwise
    using T64 = Tr<WD_F64>;
    WD_CK(ctx, cudaMemcpyAsync(sb.x, x_e, f64, cudaMemcpyDeviceToDevice, s));
    EpiStore<SpinorF64> e0{T64::view(sb.tmp64, c.g)};
    launch_dslash<double>(c, T64::view(sb.x, c.g), T64::gauge(c), 1, 0, e0, s);
    EpiResid<SpinorF64, SpinorF64, SpinorF64, FinStore> e1{T64::view(sb.r, c.g), true, T64::view(sb.b_hat, c.g),
                                                           T64::view(sb.x, c.g), Coef{-kappa * kappa, nullptr},
                                                           c.red, FinStore{c.scalars + 6, 1}};
    launch_dslash<double>(c, T64::view(sb.tmp64, c.g), T64::gauge(c), 0, 0, e1, s);
    setup_src = sb.r;
  } else {
    o64->zero(c, sb.x, s);
  }
  WD_CK_LAUNCH(ctx, "solve setup");

  unsigned long long hu = 0, hl = 0;
  if (p.use_graph) {
    if (!(c.graph_exec && c.graph_prec == p.inner_precision && c.graph_solver == p.solver &&
          c.graph_xhat == p.xhat_f32)) {
      destroy_graph(c);
      if ((st = build_graph(ctx, p.solver, p.inner_precision, &c.graph_hu, &c.graph_hl)) != WD_OK) return st;
    }
    hu = c.graph_hu;
    hl = c.graph_hl;
  }
  init_ctl_kernel<<<1, 1, 0, s>>>(sb.ctl, p.tol, p.delta, p.max_iter, kappa, c.scalars, p.use_graph ? 1 : 0, hu,
                                  hl, p.restart ? 1 : 0);
  if (p.solver == WD_BICGSTAB) oin->bicg_setup(c, sb, setup_src, s);
  else oin->cg_setup(c, sb, s);
  WD_CK_LAUNCH(ctx, "solver setup");

  // a zero source needs no iteration, nor does an initial guess that already
  // meets the tolerance
  WD_CK(ctx, cudaMemcpyAsync(c.host_pinned, c.scalars, 7 * sizeof(double), cudaMemcpyDeviceToHost, s));
  WD_CK(ctx, cudaStreamSynchronize(s));
  const double b2 = c.host_pinned[0] + c.host_pinned[1];
  const bool start_converged = x0 && c.host_pinned[6] <= p.tol * p.tol * b2;
  SolverCtl hc;
  if (!(b2 > 0.0)) {
    o64->zero(c, x_e, s);
    o64->zero(c, x_o, s);
    WD_CK(ctx, cudaStreamSynchronize(s));
    if (info) {
      memset(info, 0, sizeof(*info));
      info->status = std::isfinite(b2) ? WD_OK : WD_ERR_NUMERIC;
    }
    return std::isfinite(b2) ? WD_OK : set_err(ctx, WD_ERR_NUMERIC, "source is not finite");
  }

  if (start_converged) {
    mark_done_kernel<<<1, 1, 0, s>>>(sb.ctl);
  } else if (p.use_graph) {
    WD_CK(ctx, cudaGraphLaunch(c.graph_exec, s));
  } else {
    for (;;) {
      if (p.solver == WD_BICGSTAB) oin->bicg_iteration(c, sb, s);
      else oin->cg_iteration(c, sb, s);
      WD_CK_LAUNCH(ctx, "iteration");
      WD_CK(ctx, cudaMemcpyAsync(&hc, sb.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
      WD_CK(ctx, cudaStreamSynchronize(s));
      if (hc.done) break;
      if (hc.do_update) {
        if (p.solver == WD_BICGSTAB) oin->bicg_update(c, sb, s);
        else oin->cg_update(c, sb, s);
        WD_CK_LAUNCH(ctx, "reliable update");
        WD_CK(ctx, cudaMemcpyAsync(&hc, sb.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
        WD_CK(ctx, cudaStreamSynchronize(s));
        if (hc.done) break;
      }
    }
  }

  // x_e from the accumulator, x_o = b_o + kappa D_oe x_e (Sec. 3: the full
  // solution is reconstructed from the Schur solution)
  WD_CK(ctx, cudaMemcpyAsync(x_e, sb.x, f64, cudaMemcpyDeviceToDevice, s));
  // S13: full FP64 true residual |b - M x|.  The odd rows come with x_o
  // itself: one FP64 D_oe x_e gives x_o = b_o + kappa D_oe x_e and
  // r_o = b_o - (x_o - kappa D_oe x_e); the even rows need D_eo x_o.
  {
    using T64 = Tr<WD_F64>;
    EpiReconResid<FinStore> eo{T64::view(x_o, c.g), T64::view(b_o, c.g), Coef{kappa, nullptr}, c.red,
                               FinStore{c.scalars + 5, 1}};
    launch_dslash<double>(c, T64::view(x_e, c.g), T64::gauge(c), 1, 0, eo, s);
    const Coef ck{-kappa, nullptr};
    EpiResid<SpinorF64, SpinorF64, SpinorF64, FinStore> ee{T64::view(nullptr, c.g), false, T64::view(b_e, c.g),
                                                           T64::view(x_e, c.g), ck, c.red, FinStore{c.scalars + 4, 1}};
    launch_dslash<double>(c, T64::view(x_o, c.g), T64::gauge(c), 0, 0, ee, s);
  }
  WD_CK_LAUNCH(ctx, "reconstruction");
  WD_CK(ctx, cudaMemcpyAsync(&hc, sb.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
  WD_CK(ctx, cudaMemcpyAsync(c.host_pinned, c.scalars, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  WD_CK(ctx, cudaStreamSynchronize(s));
  const double r2 = c.host_pinned[4] + c.host_pinned[5];
  wd_status result = (wd_status)hc.status;
  if (result == WD_OK && !hc.done) result = WD_ERR_NOT_CONVERGED;
  if (!std::isfinite(r2)) result = WD_ERR_NUMERIC;
  // the device stops on the Schur residual of its last reliable update; the
  // full residual of the reconstructed x is the one reported, and it decides
  if (result == WD_OK && r2 > p.tol * p.tol * b2) result = WD_ERR_NOT_CONVERGED;
  if (info) {
    info->iters = hc.iter + hc.updates;
    info->reliable_updates = hc.updates;
    info->true_rel_residual = std::sqrt(r2 / b2);
    info->iterated_rel_residual = std::sqrt(hc.rr / b2);
    info->status = result;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // setup: 3 norms, b_hat, zero x, control init, solver setup (4 kernels,
    // CG: 2 dslash + 2 zero); per iteration: BiCGstab 7 (CG 5) + loop control;
    // per reliable update: BiCGstab 4 (5 with a lower inner precision: the
    // quantisation pass), CG 5; end: x_o with the odd residual,
    // and the even residual dslash
    // (an initial guess: its two residual dslashes instead of the zeroing,
    // and the control update when it already meets the tolerance)
    const long long setup = 3 + (odd_zero ? 0 : 1) + (x0 ? 2 : 1) + 1 + 4 + (start_converged ? 1 : 0);
    const long long per_it = (p.solver == WD_BICGSTAB ? 7 : 5) + (p.use_graph ? 1 : 0);
    const long long per_up = (p.solver == WD_BICGSTAB) ? (p.inner_precision == WD_F64 ? 4 : 5) : 5;
    info->kernel_launches = setup + (long long)hc.iter * per_it + (long long)hc.updates * per_up + 2;
  }
  if (result != WD_OK) {
    char m[160];
    snprintf(m, sizeof m, "solve ended with status %d after %d iterations (true residual %.3e)", (int)result,
             hc.iter + hc.updates, std::sqrt(r2 / b2));
    set_err(ctx, result, m);
  }
  return result;
}

}  // namespace

// both parities of a device FP64 field -> host lexicographic array, one
// device-to-host copy, stream-ordered and not waited for (asynchronous when
// the host array is page-locked)
wd_status wd_internal_export_full_async(wd_ctx* ctx, double* host, const void* even, const void* odd) {
  Ctx& c = ctx->c;
  wd_status st = ensure_staging(ctx);
  if (st != WD_OK) return st;
  const PrecOps* o = ops_f64();
  o->export_lex(c, c.lex_staging, even, 0, c.stream);
  o->export_lex(c, c.lex_staging, odd, 1, c.stream);
  WD_CK_LAUNCH(ctx, "export");
  WD_CK(ctx, cudaMemcpyAsync(host, c.lex_staging, (size_t)2 * c.g.Vh * 24 * sizeof(double), cudaMemcpyDeviceToHost,
                             c.stream));
  return WD_OK;
}

wd_status wd_internal_export_full(wd_ctx* ctx, double* host, const void* even, const void* odd) {
  Ctx& c = ctx->c;
  wd_status st = ensure_staging(ctx);
  if (st != WD_OK) return st;
  const PrecOps* o = ops_f64();
  o->export_lex(c, c.lex_staging, even, 0, c.stream);
  o->export_lex(c, c.lex_staging, odd, 1, c.stream);
  WD_CK_LAUNCH(ctx, "export");
  WD_CK(ctx, cudaMemcpyAsync(host, c.lex_staging, (size_t)2 * c.g.Vh * 24 * sizeof(double), cudaMemcpyDeviceToHost,
                             c.stream));
  WD_CK(ctx, cudaStreamSynchronize(c.stream));
  return WD_OK;
}

// host lexicographic FP64 field -> both parities of a device FP64 field, one
// host-to-device copy, stream-ordered.  For pageable host memory the copy has
// read the array when this returns; for page-locked memory it is still in
// flight, and the array may be reused only once the stream has reached this
// point (an event or a synchronisation)
wd_status wd_internal_import_full(wd_ctx* ctx, void* even, void* odd, const double* host) {
  Ctx& c = ctx->c;
  wd_status st = ensure_staging(ctx);
  if (st != WD_OK) return st;
  WD_CK(ctx, cudaMemcpyAsync(c.lex_staging, host, (size_t)2 * c.g.Vh * 24 * sizeof(double), cudaMemcpyHostToDevice,
                             c.stream));
  const PrecOps* o = ops_f64();
  o->import_lex(c, even, c.lex_staging, 0, c.stream);
  o->import_lex(c, odd, c.lex_staging, 1, c.stream);
  WD_CK_LAUNCH(ctx, "import");
  return WD_OK;
}

wd_status wd_internal_solve_x0(wd_ctx* ctx, void* x_full, const void* b_full, double kappa,
                               const wd_solve_params* params, wd_solve_info* info) {
  if (!ctx || !x_full || !b_full || x_full == b_full) return WD_ERR_INVALID_ARG;
  return solve_device(ctx, x_full, b_full, kappa, params, info, true);
}

wd_status wd_internal_ensure_gauge(wd_ctx* ctx, int prec) {
  if (!ctx || prec < WD_F64 || prec > WD_B16N) return WD_ERR_INVALID_ARG;
  return ensure_gauge(ctx, prec);
}

extern "C" {

const char* wd_status_string(wd_status s) {
  switch (s) {
    case WD_OK: return "ok";
    case WD_ERR_INVALID_ARG: return "invalid argument";
    case WD_ERR_OOM: return "out of device memory";
    case WD_ERR_CUDA: return "CUDA error";
    case WD_ERR_NOT_CONVERGED: return "not converged";
    case WD_ERR_BREAKDOWN: return "Krylov breakdown";
    case WD_ERR_NUMERIC: return "NaN or Inf";
    case WD_ERR_TIMEOUT: return "device wait timed out";
    case WD_ERR_BUDGET: return "memory budget exceeded";
    case WD_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* wd_last_error(const wd_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

wd_status wd_create(wd_ctx** out, const int dims[4], int t_antiperiodic, void* cuda_stream) {
  if (!out || !dims) return WD_ERR_INVALID_ARG;
  *out = nullptr;
  long long v = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || (dims[m] & 1)) return WD_ERR_INVALID_ARG;
    v *= dims[m];
  }
  if (v / 2 > (1LL << 30)) return WD_ERR_INVALID_ARG;
  wd_ctx* ctx = new (std::nothrow) wd_ctx();
  if (!ctx) return WD_ERR_OOM;
  Ctx& c = ctx->c;
  c.g = make_geom(dims, t_antiperiodic);
  memcpy(c.dims, dims, sizeof(c.dims));
  c.stream = (cudaStream_t)cuda_stream;
  c.recon = 12;
  c.low_recon = 12;
  c.sb_prec = c.sb_solver = -1;
  c.graph_prec = c.graph_solver = -1;
  wd_status st = WD_OK;
  cudaError_t e = cudaGetDevice(&c.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
  if (e != cudaSuccess) {
    delete ctx;
    return WD_ERR_CUDA;
  }
  c.max_red_blocks = c.num_sms * 16;
  if ((st = dev_alloc(ctx, &c.red.partials, (size_t)c.max_red_blocks * 8 * sizeof(double))) != WD_OK ||
      (st = dev_alloc(ctx, &c.red.counter, 256)) != WD_OK ||
      (st = dev_alloc(ctx, &c.scalars, 64 * sizeof(double))) != WD_OK) {
    wd_destroy(ctx);
    return st;
  }
  if (cudaMemset(c.red.counter, 0, 256) != cudaSuccess || cudaMemset(c.scalars, 0, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&c.host_pinned, 64 * sizeof(double)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    wd_destroy(ctx);
    return WD_ERR_CUDA;
  }
  *out = ctx;
  return WD_OK;
}

wd_status wd_destroy(wd_ctx* ctx) {
  if (!ctx) return WD_OK;
  Ctx& c = ctx->c;
  cudaStreamSynchronize(c.stream);
  destroy_graph(c);
  for (int p = 0; p < 5; ++p) {
    dev_free(c.gauge[p]);
    dev_free(c.gauge4[p]);
    dev_free(c.tmp_odd[p]);
  }
  dev_free((void*&)c.red.partials);
  dev_free((void*&)c.red.counter);
  dev_free((void*&)c.scalars);
  dev_free((void*&)c.lex_staging);
  dev_free(c.sb_block);
  dev_free((void*&)c.sb.ctl);
  dev_free(c.sb_full[0]);
  dev_free(c.sb_full[1]);
  dev_free((void*&)c.gfix);
  batch_release(c);
  if (c.host_pinned) cudaFreeHost(c.host_pinned);
  delete ctx;
  return WD_OK;
}

wd_status wd_set_stream(wd_ctx* ctx, void* stream) {
  if (!ctx) return WD_ERR_INVALID_ARG;
  ctx->c.stream = (cudaStream_t)stream;
  return WD_OK;
}

size_t wd_field_bytes(const wd_ctx* ctx, wd_prec prec) {
  if (!ctx || !valid_prec(prec)) return 0;
  return field_bytes(ctx->c, prec);
}

wd_status wd_load_gauge(wd_ctx* ctx, const double* U, int is_device, int recon) {
  return wd_load_gauge_opt(ctx, U, is_device, recon, 0);
}

wd_status wd_load_gauge_opt(wd_ctx* ctx, const double* U, int is_device, int recon, int flags) {
  if (!ctx || !U || (recon != 12 && recon != 18) || (flags & ~(WD_GAUGE_TEMPORAL | WD_GAUGE_RECON8)))
    return set_err(ctx, WD_ERR_INVALID_ARG, "wd_load_gauge: bad args");
  const int temporal_gauge = (flags & WD_GAUGE_TEMPORAL) ? 1 : 0;
  Ctx& c = ctx->c;
  WD_CK(ctx, cudaSetDevice(c.device));
  WD_CK(ctx, cudaStreamSynchronize(c.stream));
  destroy_graph(c);
  batch_release(c);
  for (int p = 0; p < 5; ++p) {
    dev_free(c.gauge[p]);
    dev_free(c.gauge4[p]);
  }
  dev_free((void*&)c.gfix);
  c.gauge_loaded = false;
  c.g.tfix = 0;
  const size_t lex_bytes = (size_t)2 * c.g.Vh * 72 * sizeof(double);
  const double* src = U;
  double* staging = nullptr;
  double2* glex = nullptr;
  wd_status st = WD_OK;
  // the temporal gauge transforms the links in place: always on a copy
  if (!is_device || temporal_gauge) {
    if ((st = dev_alloc(ctx, &staging, lex_bytes)) != WD_OK) return st;
    cudaError_t e = cudaMemcpyAsync(staging, U, lex_bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    c.stream);
    if (e != cudaSuccess) {
      cudaFree(staging);
      return cuda_err(ctx, e, "gauge upload");
    }
    src = staging;
  }
  if (temporal_gauge) {
    const size_t gbytes = (size_t)2 * c.g.Vh * 9 * sizeof(double2);
    st = dev_alloc(ctx, &glex, gbytes);
    if (st == WD_OK) st = dev_alloc(ctx, &c.gfix, (size_t)2 * 9 * c.g.stride * sizeof(double2));
    if (st == WD_OK) {
      const long long ns = (long long)c.g.X * c.g.Y * c.g.Z;
      temporal_gauge_g_kernel<<<grid_for(c, (int)ns, 128), 128, 0, c.stream>>>(c.g, staging, glex);
      temporal_gauge_apply_kernel<<<grid_for(c, 2 * c.g.Vh, 128), 128, 0, c.stream>>>(c.g, staging, glex);
      temporal_gauge_pack_kernel<<<grid_for(c, 2 * c.g.Vh, 256), 256, 0, c.stream>>>(c.g, glex, c.gfix);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_err(ctx, e, "temporal gauge");
    }
  }
  c.recon = recon;
  c.low_recon = (flags & WD_GAUGE_RECON8) ? 8 : 12;
  const int nc = recon / 2;
  if (st == WD_OK) st = dev_alloc(ctx, &c.gauge[WD_F64], (size_t)8 * nc * c.g.stride * sizeof(double2));
  if (st == WD_OK) {
    gauge_pack_f64_kernel<<<grid_for(c, 2 * c.g.Vh, 256), 256, 0, c.stream>>>(c.g, src, (double2*)c.gauge[WD_F64],
                                                                               nc);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) st = cuda_err(ctx, e, "gauge pack");
  }
  if (staging) cudaFree(staging);
  if (glex) cudaFree(glex);
  if (st == WD_OK) {
    c.gauge_loaded = true;
    c.g.tfix = temporal_gauge;
  } else {
    dev_free((void*&)c.gfix);
  }
  return st;
}

static wd_status field_io(wd_ctx* ctx, bool import, void* field, double* lex, int is_device, int parity, int prec) {
  if (!ctx || !field || !lex || (parity != 0 && parity != 1) || !valid_prec(prec))
    return set_err(ctx, WD_ERR_INVALID_ARG, "field import/export: bad args");
  Ctx& c = ctx->c;
  WD_CK(ctx, cudaSetDevice(c.device));
  const PrecOps* o = prec_ops(prec);
  const size_t lex_bytes = (size_t)2 * c.g.Vh * 24 * sizeof(double);
  double* dlex = lex;
  wd_status st;
  if (!is_device) {
    if ((st = ensure_staging(ctx)) != WD_OK) return st;
    dlex = c.lex_staging;
    // export fills only the sites of one parity: upload the host array first
    // so that the other parity's sites come back unchanged
    WD_CK(ctx, cudaMemcpyAsync(dlex, lex, lex_bytes, cudaMemcpyHostToDevice, c.stream));
  }
  if (import) o->import_lex(c, field, dlex, parity, c.stream);
  else o->export_lex(c, dlex, field, parity, c.stream);
  WD_CK_LAUNCH(ctx, "field import/export");
  if (!is_device) {
    if (!import) WD_CK(ctx, cudaMemcpyAsync(lex, dlex, lex_bytes, cudaMemcpyDeviceToHost, c.stream));
    WD_CK(ctx, cudaStreamSynchronize(c.stream));
  }
  return WD_OK;
}

wd_status wd_field_import(wd_ctx* ctx, void* field, const double* lex, int is_device, wd_parity parity,
                          wd_prec prec) {
  return field_io(ctx, true, field, const_cast<double*>(lex), is_device, parity, prec);
}

wd_status wd_field_export(wd_ctx* ctx, double* lex, const void* field, int is_device, wd_parity parity,
                          wd_prec prec) {
  return field_io(ctx, false, const_cast<void*>(field), lex, is_device, parity, prec);
}

wd_status wd_dslash(wd_ctx* ctx, void* out, const void* in, wd_parity out_parity, int dagger, wd_prec prec) {
  if (!ctx || !out || !in || out == in || (out_parity != 0 && out_parity != 1) || !valid_prec(prec))
    return set_err(ctx, WD_ERR_INVALID_ARG, "wd_dslash: bad args");
  WD_CK(ctx, cudaSetDevice(ctx->c.device));
  wd_status st = ensure_gauge(ctx, prec);
  if (st != WD_OK) return st;
  prec_ops(prec)->dslash(ctx->c, out, in, out_parity, dagger ? 1 : 0, ctx->c.stream);
  WD_CK_LAUNCH(ctx, "wd_dslash");
  return WD_OK;
}

// ---- T-slab decomposition (Sec. 6)
static wd_status slab_check(wd_ctx* ctx, int prec, const char* what) {
  if (!ctx || !valid_prec(prec)) return set_err(ctx, WD_ERR_INVALID_ARG, std::string(what) + ": bad args");
  Ctx& c = ctx->c;
  if (c.g.T < 2 || (c.g.T & 1))
    return set_err(ctx, WD_ERR_INVALID_ARG, std::string(what) + ": the slab's T must be even and >= 2");
  if (c.gauge_loaded && (c.g.tfix || (prec != WD_F64 && c.low_recon != 12)))
    return set_err(ctx, WD_ERR_INVALID_ARG,
                   std::string(what) + ": slabs take general links with 12-real FP32 / 16-bit copies (no temporal "
                                       "gauge, no 8-number links)");
  return WD_OK;
}

size_t wd_slab_face_bytes(const wd_ctx* ctx, wd_prec prec) {
  if (!ctx || !valid_prec(prec)) return 0;
  return prec_ops(prec)->slab_face_bytes(ctx->c);
}

size_t wd_slab_link_face_bytes(const wd_ctx* ctx, wd_prec prec) {
  if (!ctx || !valid_prec(prec)) return 0;
  return prec_ops(prec)->slab_link_face_bytes(ctx->c);
}

wd_status wd_slab_pack_faces(wd_ctx* ctx, void* face_lo, void* face_hi, const void* in, int dagger, wd_prec prec) {
  wd_status st = slab_check(ctx, prec, "wd_slab_pack_faces");
  if (st != WD_OK) return st;
  if (!face_lo || !face_hi || !in || face_lo == face_hi)
    return set_err(ctx, WD_ERR_INVALID_ARG, "wd_slab_pack_faces: bad pointers");
  WD_CK(ctx, cudaSetDevice(ctx->c.device));
  prec_ops(prec)->slab_pack_faces(ctx->c, face_lo, face_hi, in, dagger ? 1 : 0, ctx->c.stream);
  WD_CK_LAUNCH(ctx, "wd_slab_pack_faces");
  return WD_OK;
}

wd_status wd_slab_pack_link_face(wd_ctx* ctx, void* link_face, wd_prec prec) {
  wd_status st = slab_check(ctx, prec, "wd_slab_pack_link_face");
  if (st != WD_OK) return st;
  if (!link_face) return set_err(ctx, WD_ERR_INVALID_ARG, "wd_slab_pack_link_face: null face");
  WD_CK(ctx, cudaSetDevice(ctx->c.device));
  if ((st = ensure_gauge(ctx, prec)) != WD_OK) return st;
  if ((st = slab_check(ctx, prec, "wd_slab_pack_link_face")) != WD_OK) return st;
  prec_ops(prec)->slab_pack_link_face(ctx->c, link_face, ctx->c.stream);
  WD_CK_LAUNCH(ctx, "wd_slab_pack_link_face");
  return WD_OK;
}

wd_status wd_dslash_slab(wd_ctx* ctx, void* out, const void* in, const void* halo_lo, const void* halo_hi,
                         const void* link_halo, int flip_lo, int flip_hi, wd_parity out_parity, int dagger,
                         wd_prec prec, int region) {
  wd_status st = slab_check(ctx, prec, "wd_dslash_slab");
  if (st != WD_OK) return st;
  if (!out || !in || out == in || (out_parity != 0 && out_parity != 1) || region < 0 || region > 2)
    return set_err(ctx, WD_ERR_INVALID_ARG, "wd_dslash_slab: bad args");
  if (region != 0 && (!halo_lo || !halo_hi || !link_halo))
    return set_err(ctx, WD_ERR_INVALID_ARG, "wd_dslash_slab: the boundary slices need both halos and the link halo");
  WD_CK(ctx, cudaSetDevice(ctx->c.device));
  if ((st = ensure_gauge(ctx, prec)) != WD_OK) return st;
  if ((st = slab_check(ctx, prec, "wd_dslash_slab")) != WD_OK) return st;
  prec_ops(prec)->slab_dslash(ctx->c, out, in, halo_lo, halo_hi, link_halo, flip_lo ? 1 : 0, flip_hi ? 1 : 0,
                              out_parity, dagger ? 1 : 0, region, ctx->c.stream);
  WD_CK_LAUNCH(ctx, "wd_dslash_slab");
  return WD_OK;
}

wd_status wd_dslash_xpay(wd_ctx* ctx, void* out, const void* in, const void* x, double a, wd_parity out_parity,
                         int dagger, wd_prec prec) {
  if (!ctx || !out || !in || !x || out == in || (out_parity != 0 && out_parity != 1) || !valid_prec(prec))
    return set_err(ctx, WD_ERR_INVALID_ARG, "wd_dslash_xpay: bad args");
  WD_CK(ctx, cudaSetDevice(ctx->c.device));
  wd_status st = ensure_gauge(ctx, prec);
  if (st != WD_OK) return st;
  prec_ops(prec)->dslash_xpay(ctx->c, out, in, x, a, nullptr, out_parity, dagger ? 1 : 0, ctx->c.stream);
  WD_CK_LAUNCH(ctx, "wd_dslash_xpay");
  return WD_OK;
}

wd_status wd_apply_M(wd_ctx* ctx, void* out, const void* in, double kappa, wd_operator which, int dagger,
                     wd_prec prec) {
  if (!ctx || !out || !in || out == in || !valid_prec(prec) || (which != WD_M_FULL && which != WD_M_SCHUR_EVEN))
    return set_err(ctx, WD_ERR_INVALID_ARG, "wd_apply_M: bad args");
  Ctx& c = ctx->c;
  WD_CK(ctx, cudaSetDevice(c.device));
  wd_status st = ensure_gauge(ctx, prec);
  if (st != WD_OK) return st;
  const PrecOps* o = prec_ops(prec);
  const int dg = dagger ? 1 : 0;
  if (which == WD_M_FULL) {
    const size_t fb = field_bytes(c, prec);
    const char* ie = (const char*)in;
    char* oe = (char*)out;
    o->dslash_xpay(c, oe, ie + fb, ie, -kappa, nullptr, 0, dg, c.stream);
    o->dslash_xpay(c, oe + fb, ie, ie + fb, -kappa, nullptr, 1, dg, c.stream);
  } else {
    if ((st = ensure_tmp_odd(ctx, prec)) != WD_OK) return st;
    o->dslash(c, c.tmp_odd[prec], in, 1, dg, c.stream);
    o->dslash_xpay(c, out, c.tmp_odd[prec], in, -kappa * kappa, nullptr, 0, dg, c.stream);
  }
  WD_CK_LAUNCH(ctx, "wd_apply_M");
  return WD_OK;
}

wd_status wd_norm2(wd_ctx* ctx, double* result, const void* field, wd_prec prec) {
  if (!ctx || !result || !field || !valid_prec(prec)) return set_err(ctx, WD_ERR_INVALID_ARG, "wd_norm2: bad args");
  Ctx& c = ctx->c;
  WD_CK(ctx, cudaSetDevice(c.device));
  prec_ops(prec)->norm2(c, c.scalars + 8, field, c.stream);
  WD_CK_LAUNCH(ctx, "wd_norm2");
  WD_CK(ctx, cudaMemcpyAsync(c.host_pinned + 8, c.scalars + 8, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  WD_CK(ctx, cudaStreamSynchronize(c.stream));
  *result = c.host_pinned[8];
  return WD_OK;
}

wd_status wd_solve_device(wd_ctx* ctx, void* x, const void* b, double kappa, const wd_solve_params* params,
                          wd_solve_info* info) {
  if (!ctx || !x || !b || x == b) return set_err(ctx, WD_ERR_INVALID_ARG, "wd_solve_device: bad args");
  WD_CK(ctx, cudaSetDevice(ctx->c.device));
  return solve_device(ctx, x, b, kappa, params, info);
}

wd_status wd_solve(wd_ctx* ctx, double* x, const double* b, double kappa, const wd_solve_params* params,
                   wd_solve_info* info) {
  if (!ctx || !x || !b) return set_err(ctx, WD_ERR_INVALID_ARG, "wd_solve: bad args");
  Ctx& c = ctx->c;
  WD_CK(ctx, cudaSetDevice(c.device));
  const auto t0 = std::chrono::steady_clock::now();
  const size_t f64 = field_bytes(c, WD_F64);
  wd_status st;
  for (int k = 0; k < 2; ++k)
    if (!c.sb_full[k] && (st = dev_alloc(ctx, &c.sb_full[k], 2 * f64)) != WD_OK) return st;
  if ((st = ensure_staging(ctx)) != WD_OK) return st;
  const size_t lex_bytes = (size_t)2 * c.g.Vh * 24 * sizeof(double);
  const PrecOps* o64 = ops_f64();
  char* bf = (char*)c.sb_full[0];
  char* xf = (char*)c.sb_full[1];
  if (params && params->initial_guess == 1) {  // the starting x, through the same staging buffer
    WD_CK(ctx, cudaMemcpyAsync(c.lex_staging, x, lex_bytes, cudaMemcpyHostToDevice, c.stream));
    o64->import_lex(c, xf, c.lex_staging, 0, c.stream);
    o64->import_lex(c, xf + f64, c.lex_staging, 1, c.stream);
  }
  WD_CK(ctx, cudaMemcpyAsync(c.lex_staging, b, lex_bytes, cudaMemcpyHostToDevice, c.stream));
  o64->import_lex(c, bf, c.lex_staging, 0, c.stream);
  o64->import_lex(c, bf + f64, c.lex_staging, 1, c.stream);
  WD_CK_LAUNCH(ctx, "wd_solve import");
  wd_status rs = solve_device(ctx, xf, bf, kappa, params, info);
  if (rs != WD_OK && rs != WD_ERR_NOT_CONVERGED && rs != WD_ERR_BREAKDOWN && rs != WD_ERR_NUMERIC) return rs;
  o64->export_lex(c, c.lex_staging, xf, 0, c.stream);
  o64->export_lex(c, c.lex_staging, xf + f64, 1, c.stream);
  WD_CK_LAUNCH(ctx, "wd_solve export");
  WD_CK(ctx, cudaMemcpyAsync(x, c.lex_staging, lex_bytes, cudaMemcpyDeviceToHost, c.stream));
  WD_CK(ctx, cudaStreamSynchronize(c.stream));
  if (info) info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return rs;
}

}  // extern "C"
