// Multi-right-hand-side dslash and the batched Krylov solver.
//
// Many sources and masses share one gauge field (Sec. 3: solutions for many
// source vectors b).  A block of the multi-RHS dslash covers 32 output sites
// and TR right-hand sides: it loads the 8 links of each of its 32 sites once
// into shared memory (decoded, third row rebuilt once) and every chunk of TR
// right-hand sides reuses them, so a launch reads each link from DRAM once
// however many right-hand sides it serves.  Each right-hand side has its own
// coefficient (kappa), its own fused epilogue and its own FP64 reductions.
//
// Reductions of a batch are two-stage: the producing kernel writes one FP64
// partial per (right-hand side, quantity, block); a finalise kernel with one
// block per right-hand side sums them in block order (deterministic) and runs
// that system's finaliser, and the last of its blocks decides for the whole
// batch (any reliable update pending; all converged).  Spreading the final
// FP64 sums over many SMs matters on GB300, whose FP64 pipe is 1/58 of FP32.
#pragma once

#include "wd_kernels.cuh"

namespace wd {

// Device state of a batch beyond the per-system SolverCtl array.
struct BatchCtl {
  unsigned counter[4];  // tickets of the finalise kernels (zero between uses)
  int any_update;       // some active system ends this iteration with an update
  int all_done;
  int in_graph;
  int loops;
  int max_loops;
  int step_loops;  // WHILE-body executions since the host last launched the loop
  int step_limit;  // pause (return to the host) after this many, for serving
  unsigned long long h_update, h_loop;
  int nupd;           // systems due for a reliable update this iteration
  int upd_list[256];  // their indices, ascending
};

struct BatchArgs {
  int nrhs;
  const SolverCtl* ctl;  // nullptr: every right-hand side active
  int mode;              // 0: active unless done; 1: active when an update is due
  double* partials;      // [(r * NRED + k) * nblocks + block]
  const BatchCtl* bc;    // mode 1: the compacted list of systems due for an update
};

__device__ __forceinline__ bool rhs_active(const BatchArgs& a, int r) {
  if (r >= a.nrhs) return false;
  if (!a.ctl) return true;
  const volatile SolverCtl* c = a.ctl + r;
  return !c->done && (a.mode == 0 || c->do_update);
}

// even-odd indices of the 8 neighbours of site h (forward, backward per mu)
__device__ __forceinline__ void neighbours(const Geom& g, int h, int x, int y, int z, int t, int (&nb)[8]) {
  const int xo = x & 1;
  nb[0] = (x == g.X - 1) ? h - (g.Xh - 1) : h + xo;
  nb[1] = (x == 0) ? h + (g.Xh - 1) : h - (xo ^ 1);
  nb[2] = (y == g.Y - 1) ? h - g.wy : h + g.Xh;
  nb[3] = (y == 0) ? h + g.wy : h - g.Xh;
  nb[4] = (z == g.Z - 1) ? h - g.wz : h + g.XhY;
  nb[5] = (z == 0) ? h + g.wz : h - g.XhY;
  nb[6] = (t == g.T - 1) ? h - g.wt : h + g.XhYZ;
  nb[7] = (t == 0) ? h + g.wt : h - g.XhYZ;
}

// one hop with the link taken from the shared-memory tile (column sx)
template <int MU, bool FWD, bool DAGGER, typename R, class In>
__device__ __forceinline__ void hop_tile(const In& in, const R* lk, int sx, int h_nbr, bool flip, R (&acc)[24]) {
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  constexpr int which = 2 * MU + (FWD ? 0 : 1);
  R psi[24];
  R w = 1;
  if constexpr (In::kScaled) w = in.load_raw(h_nbr, psi);
  else in.load(h_nbr, psi);
  R hs[12];
  project<MU, S>(psi, hs);
  R u[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) u[k] = lk[(which * 18 + k) * 32 + sx];
  R gs[12];
  su3_mul<!FWD>(u, hs, gs);
  if constexpr (In::kScaled) {
    reconstruct_scaled<MU, S>(gs, acc, flip ? -w : w);
  } else {
    if (flip) {
#pragma unroll
      for (int k = 0; k < 12; ++k) gs[k] = -gs[k];
    }
    reconstruct<MU, S>(gs, acc);
  }
}

// temporal hop from the tile: half-spinor load, diagonal projector
template <bool FWD, bool DAGGER, typename R, class In>
__device__ __forceinline__ void hop_tile_t(const In& in, const R* lk, int sx, int h_nbr, bool flip, bool unit,
                                           R (&acc)[24]) {
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  constexpr bool upper = (S == +1);
  constexpr int which = 6 + (FWD ? 0 : 1);
  R hs[12];
  R w = 1;
  if constexpr (In::kScaled) {
    float f[12];
    w = in.load_raw_half(h_nbr, upper, f);
#pragma unroll
    for (int k = 0; k < 12; ++k) hs[k] = f[k];
  } else {
    in.load_half(h_nbr, upper, hs);
  }
  if (unit) {  // temporal gauge: the link is 1
    accumulate_temporal<FWD, upper>(hs, acc, flip ? -(R)2 * w : (R)2 * w);
    return;
  }
  R u[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) u[k] = lk[(which * 18 + k) * 32 + sx];
  R gs[12];
  su3_mul<!FWD>(u, hs, gs);
  accumulate_temporal<FWD, upper>(gs, acc, flip ? -(R)2 * w : (R)2 * w);
}

template <bool DAGGER, typename R, class In>
__device__ __forceinline__ void dslash_site_tile(const In& in, const R* lk, int sx, const int (&nb)[8], bool top,
                                                 bool bot, bool unit_fwd, bool unit_bwd, R (&acc)[24]) {
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0;
  hop_tile<0, true, DAGGER>(in, lk, sx, nb[0], false, acc);
  hop_tile<0, false, DAGGER>(in, lk, sx, nb[1], false, acc);
  hop_tile<1, true, DAGGER>(in, lk, sx, nb[2], false, acc);
  hop_tile<1, false, DAGGER>(in, lk, sx, nb[3], false, acc);
  hop_tile<2, true, DAGGER>(in, lk, sx, nb[4], false, acc);
  hop_tile<2, false, DAGGER>(in, lk, sx, nb[5], false, acc);
  hop_tile_t<true, DAGGER>(in, lk, sx, nb[6], top, unit_fwd, acc);
  hop_tile_t<false, DAGGER>(in, lk, sx, nb[7], bot, unit_bwd, acc);
}

template <typename R>
constexpr size_t tile_link_bytes() {
  return (size_t)8 * 18 * 32 * sizeof(R);
}

// ---- two right-hand sides per thread in FP32x2 registers.  The systems of a
// pair share every link, so the SU(3) products, the reconstructions and the
// accumulators run as packed (sm_100 family) FMA2 operations on (system a,
// system b); the tile holds each link value as a broadcast pair (u, u), read
// with one 64-bit shared load.  Decoding and projection stay per system.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fms2(float2 a, float2 b, float2 c) {  // c - a b
  return __ffma2_rn(make_float2(-a.x, -a.y), b, c);
}

// g = U h (DAG false) or U^dag h, both spin rows; u: the link's 18 values as
// pairs at u[k * 32]
template <bool DAG>
__device__ __forceinline__ void su3_mul2(const float2* u, const float2 (&h)[12], float2 (&g)[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int e = DAG ? (j * 3 + i) : (i * 3 + j);
      const float2 ur = u[(2 * e) * 32], ui = u[(2 * e + 1) * 32];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const float2 hr = h[(s * 3 + j) * 2], hi = h[(s * 3 + j) * 2 + 1];
        float2& re = g[(s * 3 + i) * 2];
        float2& im = g[(s * 3 + i) * 2 + 1];
        if constexpr (DAG) {  // conj(U_ji) h_j
          re = fma2(ur, hr, re);
          re = fma2(ui, hi, re);
          im = fma2(ur, hi, im);
          im = fms2(ui, hr, im);
        } else {  // U_ij h_j
          re = fma2(ur, hr, re);
          re = fms2(ui, hi, re);
          im = fma2(ur, hi, im);
          im = fma2(ui, hr, im);
        }
      }
    }
  }
}

// reconstruct_scaled() on pairs: a += w P g for both systems
template <int MU, int S_>
__device__ __forceinline__ void reconstruct_scaled2(const float2 (&g)[12], float2 (&a)[24], float2 w) {
  constexpr int S = (MU == 1) ? -S_ : S_;
  const float2 ws = (S > 0) ? w : make_float2(-w.x, -w.y);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 g0r = g[c * 2], g0i = g[c * 2 + 1];
    const float2 g1r = g[(3 + c) * 2], g1i = g[(3 + c) * 2 + 1];
    a[(0 + c) * 2] = fma2(w, g0r, a[(0 + c) * 2]);
    a[(0 + c) * 2 + 1] = fma2(w, g0i, a[(0 + c) * 2 + 1]);
    a[(3 + c) * 2] = fma2(w, g1r, a[(3 + c) * 2]);
    a[(3 + c) * 2 + 1] = fma2(w, g1i, a[(3 + c) * 2 + 1]);
    if constexpr (MU == 0) {
      a[(6 + c) * 2] = fma2(ws, g1i, a[(6 + c) * 2]);
      a[(6 + c) * 2 + 1] = fms2(ws, g1r, a[(6 + c) * 2 + 1]);
      a[(9 + c) * 2] = fma2(ws, g0i, a[(9 + c) * 2]);
      a[(9 + c) * 2 + 1] = fms2(ws, g0r, a[(9 + c) * 2 + 1]);
    } else if constexpr (MU == 1) {
      a[(6 + c) * 2] = fma2(ws, g1r, a[(6 + c) * 2]);
      a[(6 + c) * 2 + 1] = fma2(ws, g1i, a[(6 + c) * 2 + 1]);
      a[(9 + c) * 2] = fms2(ws, g0r, a[(9 + c) * 2]);
      a[(9 + c) * 2 + 1] = fms2(ws, g0i, a[(9 + c) * 2 + 1]);
    } else {
      a[(6 + c) * 2] = fma2(ws, g0i, a[(6 + c) * 2]);
      a[(6 + c) * 2 + 1] = fms2(ws, g0r, a[(6 + c) * 2 + 1]);
      a[(9 + c) * 2] = fms2(ws, g1i, a[(9 + c) * 2]);
      a[(9 + c) * 2 + 1] = fma2(ws, g1r, a[(9 + c) * 2 + 1]);
    }
  }
}

// decode + project one system's neighbour (as hop_tile does), w its scale
template <int MU, int S, class In>
__device__ __forceinline__ float project_one(const In& in, int h_nbr, float (&hs)[12]) {
  float psi[24];
  float w = 1.f;
  if constexpr (In::kScaled) w = in.load_raw(h_nbr, psi);
  else in.load(h_nbr, psi);
  project<MU, S>(psi, hs);
  return w;
}

template <int MU, bool FWD, bool DAGGER, class In>
__device__ __forceinline__ void hop_tile2(const In& ina, const In& inb, const float2* lk2, int sx, int h_nbr,
                                          float2 (&acc)[24]) {
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  constexpr int which = 2 * MU + (FWD ? 0 : 1);
  float2 h2[12];
  float2 w;
  {
    float ha[12], hb[12];
    w.x = project_one<MU, S>(ina, h_nbr, ha);
    w.y = project_one<MU, S>(inb, h_nbr, hb);
#pragma unroll
    for (int k = 0; k < 12; ++k) h2[k] = make_float2(ha[k], hb[k]);
  }
  float2 g2[12];
  su3_mul2<!FWD>(lk2 + which * 18 * 32 + sx, h2, g2);
  reconstruct_scaled2<MU, S>(g2, acc, w);
}

template <bool FWD, bool DAGGER, class In>
__device__ __forceinline__ void hop_tile2_t(const In& ina, const In& inb, const float2* lk2, int sx, int h_nbr,
                                            bool flip, bool unit, float2 (&acc)[24]) {
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  constexpr bool upper = (S == +1);
  constexpr int which = 6 + (FWD ? 0 : 1);
  constexpr int o = upper ? 0 : 12;
  float2 h2[12];
  float2 w = make_float2(1.f, 1.f);
  {
    float ha[12], hb[12];
    if constexpr (In::kScaled) {
      w.x = ina.load_raw_half(h_nbr, upper, ha);
      w.y = inb.load_raw_half(h_nbr, upper, hb);
    } else {
      ina.load_half(h_nbr, upper, ha);
      inb.load_half(h_nbr, upper, hb);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) h2[k] = make_float2(ha[k], hb[k]);
  }
  const float2 w2 = flip ? make_float2(-2.f * w.x, -2.f * w.y) : make_float2(2.f * w.x, 2.f * w.y);
  if (unit) {  // temporal gauge: the link is 1
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[o + k] = fma2(w2, h2[k], acc[o + k]);
    return;
  }
  float2 g2[12];
  su3_mul2<!FWD>(lk2 + which * 18 * 32 + sx, h2, g2);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[o + k] = fma2(w2, g2[k], acc[o + k]);
}

template <bool DAGGER, class In>
__device__ __forceinline__ void dslash_site_tile2(const In& ina, const In& inb, const float2* lk2, int sx,
                                                  const int (&nb)[8], bool top, bool bot, bool unit_fwd,
                                                  bool unit_bwd, float2 (&acc)[24]) {
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = make_float2(0.f, 0.f);
  hop_tile2<0, true, DAGGER>(ina, inb, lk2, sx, nb[0], acc);
  hop_tile2<0, false, DAGGER>(ina, inb, lk2, sx, nb[1], acc);
  hop_tile2<1, true, DAGGER>(ina, inb, lk2, sx, nb[2], acc);
  hop_tile2<1, false, DAGGER>(ina, inb, lk2, sx, nb[3], acc);
  hop_tile2<2, true, DAGGER>(ina, inb, lk2, sx, nb[4], acc);
  hop_tile2<2, false, DAGGER>(ina, inb, lk2, sx, nb[5], acc);
  hop_tile2_t<true, DAGGER>(ina, inb, lk2, sx, nb[6], top, unit_fwd, acc);
  hop_tile2_t<false, DAGGER>(ina, inb, lk2, sx, nb[7], bot, unit_bwd, acc);
}

// Multi-RHS dslash: block (32 sites) x (TR right-hand sides), grid-stride over
// 32-site tiles; dynamic shared memory = links + nrhs * NRED doubles.
template <bool DAGGER, typename R, class In, class G, class Epi, int TR>
__global__ void __launch_bounds__(32 * TR) dslash_mrhs_kernel(Geom g, In in, G gauge, int parity, Epi epi,
                                                              BatchArgs ba) {
  pdl_wait();
  constexpr int NR = Epi::NRED > 0 ? Epi::NRED : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* lk = reinterpret_cast<R*>(smem_raw);
  double* sred = reinterpret_cast<double*>(smem_raw + tile_link_bytes<R>());
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if constexpr (Epi::NRED > 0)
    for (int i = tid; i < ba.nrhs * NR; i += 32 * TR) sred[i] = 0.0;
  const int ntiles = (g.Vh + 31) / 32;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();  // the previous tile's links are no longer read
    for (int id = tid; id < 256; id += 32 * TR) {
      const int which = id >> 5, sx = id & 31, hs = tile * 32 + sx;
      if (hs < g.Vh) {
        int x, y, z, t;
        site_coords(g, hs, parity, x, y, z, t);
        int nb[8];
        neighbours(g, hs, x, y, z, t, nb);
        const int mu = which >> 1;
        const bool fwd = (which & 1) == 0;
        // temporal gauge: unit temporal links off the last slice are not read
        if (g.tfix && mu == 3 && (fwd ? t != g.T - 1 : t != 0)) continue;
        R u[18];
        if (gauge.recon == 8) gauge.template load<true>(fwd ? parity : 1 - parity, mu, fwd ? hs : nb[which], u);
        else gauge.template load<false>(fwd ? parity : 1 - parity, mu, fwd ? hs : nb[which], u);
#pragma unroll
        for (int k = 0; k < 18; ++k) lk[(which * 18 + k) * 32 + sx] = u[k];
      }
    }
    __syncthreads();
    const int h = tile * 32 + threadIdx.x;
    const bool site_ok = h < g.Vh;
    int nb[8];
    bool top = false, bot = false, unit_fwd = false, unit_bwd = false;
    if (site_ok) {
      int x, y, z, t;
      site_coords(g, h, parity, x, y, z, t);
      neighbours(g, h, x, y, z, t, nb);
      top = g.tbc_anti && (t == g.T - 1);
      bot = g.tbc_anti && (t == 0);
      unit_fwd = g.tfix && (t != g.T - 1);
      unit_bwd = g.tfix && (t != 0);
    }
    const int nwork = (ba.mode == 1 && ba.bc) ? *(const volatile int*)&ba.bc->nupd : ba.nrhs;
    for (int r0 = 0; r0 < nwork; r0 += TR) {
      const int i = r0 + threadIdx.y;
      const int r = (ba.mode == 1 && ba.bc) ? (i < nwork ? ba.bc->upd_list[i] : ba.nrhs) : i;
      double red[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) red[k] = 0.0;
      if (site_ok && rhs_active(ba, r)) {
        R acc[24];
        dslash_site_tile<DAGGER>(in.at(r), lk, threadIdx.x, nb, top, bot, unit_fwd, unit_bwd, acc);
        epi.at(r)(h, acc, red);
      }
      if constexpr (Epi::NRED > 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) red[k] += __shfl_down_sync(0xffffffffu, red[k], o);
        if (threadIdx.x == 0 && r < ba.nrhs)
#pragma unroll
          for (int k = 0; k < NR; ++k) sred[r * NR + k] += red[k];
      }
    }
  }
  if constexpr (Epi::NRED > 0) {
    __syncthreads();
    for (int i = tid; i < ba.nrhs * NR; i += 32 * TR) ba.partials[(size_t)i * gridDim.x + blockIdx.x] = sred[i];
  }
}

// Multi-RHS dslash with two systems per thread (FP32 and 16-bit storage):
// block (32 sites) x (TP pairs of right-hand sides), grid-stride over 32-site
// tiles; dynamic shared memory = links as broadcast pairs + nrhs * NRED
// doubles.  An unpaired or inactive system of a pair rides along on its
// partner's data and writes nothing.
template <typename R>
constexpr size_t tile_link_bytes2() {
  return (size_t)8 * 18 * 32 * sizeof(float2);
}

template <bool DAGGER, class In, class G, class Epi, int TP>
__global__ void __launch_bounds__(32 * TP) dslash_mrhs2_kernel(Geom g, In in, G gauge, int parity, Epi epi,
                                                               BatchArgs ba) {
  pdl_wait();
  constexpr int NR = Epi::NRED > 0 ? Epi::NRED : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* lk2 = reinterpret_cast<float2*>(smem_raw);
  double* sred = reinterpret_cast<double*>(smem_raw + tile_link_bytes2<float>());
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if constexpr (Epi::NRED > 0)
    for (int i = tid; i < ba.nrhs * NR; i += 32 * TP) sred[i] = 0.0;
  const int ntiles = (g.Vh + 31) / 32;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();  // the previous tile's links are no longer read
    for (int id = tid; id < 256; id += 32 * TP) {
      const int which = id >> 5, sx = id & 31, hs = tile * 32 + sx;
      if (hs < g.Vh) {
        int x, y, z, t;
        site_coords(g, hs, parity, x, y, z, t);
        int nb[8];
        neighbours(g, hs, x, y, z, t, nb);
        const int mu = which >> 1;
        const bool fwd = (which & 1) == 0;
        if (g.tfix && mu == 3 && (fwd ? t != g.T - 1 : t != 0)) continue;
        float u[18];
        if (gauge.recon == 8) gauge.template load<true>(fwd ? parity : 1 - parity, mu, fwd ? hs : nb[which], u);
        else gauge.template load<false>(fwd ? parity : 1 - parity, mu, fwd ? hs : nb[which], u);
#pragma unroll
        for (int k = 0; k < 18; ++k) lk2[(which * 18 + k) * 32 + sx] = make_float2(u[k], u[k]);
      }
    }
    __syncthreads();
    const int h = tile * 32 + threadIdx.x;
    const bool site_ok = h < g.Vh;
    int nb[8];
    bool top = false, bot = false, unit_fwd = false, unit_bwd = false;
    if (site_ok) {
      int x, y, z, t;
      site_coords(g, h, parity, x, y, z, t);
      neighbours(g, h, x, y, z, t, nb);
      top = g.tbc_anti && (t == g.T - 1);
      bot = g.tbc_anti && (t == 0);
      unit_fwd = g.tfix && (t != g.T - 1);
      unit_bwd = g.tfix && (t != 0);
    }
    const bool listed = ba.mode == 1 && ba.bc;
    const int nwork = listed ? *(const volatile int*)&ba.bc->nupd : ba.nrhs;
    for (int r0 = 0; r0 < nwork; r0 += 2 * TP) {
      const int i = r0 + 2 * threadIdx.y;
      const int ra = listed ? (i < nwork ? ba.bc->upd_list[i] : ba.nrhs) : i;
      const int rb = listed ? (i + 1 < nwork ? ba.bc->upd_list[i + 1] : ba.nrhs) : i + 1;
      const bool act_a = site_ok && rhs_active(ba, ra);
      const bool act_b = site_ok && rhs_active(ba, rb);
      double red_a[NR], red_b[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) red_a[k] = red_b[k] = 0.0;
      if (act_a || act_b) {
        const In ia = in.at(act_a ? ra : rb), ib = in.at(act_b ? rb : ra);
        float2 acc2[24];
        dslash_site_tile2<DAGGER>(ia, ib, lk2, threadIdx.x, nb, top, bot, unit_fwd, unit_bwd, acc2);
        float acc[24];
        if (act_a) {
#pragma unroll
          for (int k = 0; k < 24; ++k) acc[k] = acc2[k].x;
          epi.at(ra)(h, acc, red_a);
        }
        if (act_b) {
#pragma unroll
          for (int k = 0; k < 24; ++k) acc[k] = acc2[k].y;
          epi.at(rb)(h, acc, red_b);
        }
      }
      if constexpr (Epi::NRED > 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            red_a[k] += __shfl_down_sync(0xffffffffu, red_a[k], o);
            red_b[k] += __shfl_down_sync(0xffffffffu, red_b[k], o);
          }
        if (threadIdx.x == 0) {
          if (ra < ba.nrhs)
#pragma unroll
            for (int k = 0; k < NR; ++k) sred[ra * NR + k] += red_a[k];
          if (rb < ba.nrhs)
#pragma unroll
            for (int k = 0; k < NR; ++k) sred[rb * NR + k] += red_b[k];
        }
      }
    }
  }
  if constexpr (Epi::NRED > 0) {
    __syncthreads();
    for (int i = tid; i < ba.nrhs * NR; i += 32 * TP) ba.partials[(size_t)i * gridDim.x + blockIdx.x] = sred[i];
  }
}

// Per-system dslash over a batch: the single-system site kernel with
// blockIdx.y naming the system (in mode 1, the y-th entry of the list of
// systems due for an update; blocks past the list's end return at once).
// Always used for FP64, where the FP64 pipe, not the link bytes, sets the
// time, so sharing a link tile between systems gains nothing, while a tile
// whose systems are mostly idle (one reliable update due among several)
// leaves the SM a few computing warps; used for the inner precision when the
// launch shape says so (tr = 0: few systems).
template <bool DAGGER, bool TFIX, bool R8, typename R, class In, class G, class Epi>
__global__ void __launch_bounds__(kDslashBlock, (DslashOccupancy<R, In, Epi::NRED, TFIX, R8>::kMinBlocks))
    dslash_rhs_kernel(Geom g, In in, G gauge, int parity, Epi epi, BatchArgs ba) {
  pdl_wait();
  constexpr int NR = Epi::NRED > 0 ? Epi::NRED : 1;
  const int i = blockIdx.y;
  int r = i;
  if (ba.mode == 1 && ba.bc) {
    const int nwork = *(const volatile int*)&ba.bc->nupd;
    r = i < nwork ? ba.bc->upd_list[i] : ba.nrhs;
  }
  if (!rhs_active(ba, r)) return;  // uniform over the block
  const In v = in.at(r);
  const Epi e = epi.at(r);
  double red[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) red[k] = 0.0;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
    R acc[24];
    if constexpr (UseAsync<In, R8>::value) dslash_site_async<DAGGER, TFIX>(g, v, gauge, h, parity, acc);
    else dslash_site<DAGGER, TFIX, R8, Epi::NRED == 0>(g, v, gauge, h, parity, acc);
    e(h, acc, red);
  }
  if constexpr (Epi::NRED > 0) {
    __shared__ double sm[32][NR];
    block_sum<NR>(red, sm);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < NR; ++k) ba.partials[((size_t)r * NR + k) * gridDim.x + blockIdx.x] = red[k];
  }
}

// Site kernel over a batch: blockIdx.y is the right-hand side.
template <class Op>
__global__ void __launch_bounds__(kBlasBlock) site_batch_kernel(int n, Op op, BatchArgs ba) {
  pdl_wait();
  constexpr int NR = Op::NRED > 0 ? Op::NRED : 1;
  const int r = blockIdx.y;
  double red[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) red[k] = 0.0;
  if (rhs_active(ba, r)) {
    const Op o = op.at(r);
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) o(h, red);
  }
  if constexpr (Op::NRED > 0) {
    __shared__ double sm[32][NR];
    block_sum<NR>(red, sm);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < NR; ++k) ba.partials[((size_t)r * NR + k) * gridDim.x + blockIdx.x] = red[k];
  }
}

// Second stage: block r sums system r's partials in block order and runs its
// finaliser; the last block decides for the batch.  `which` selects the
// ticket counter; set_update != 0 publishes "any update pending" to the IF
// node of the solver graph.
template <int NR, class Fin>
__global__ void __launch_bounds__(128) batch_finalize_kernel(BatchArgs ba, int nblk, Fin fin, BatchCtl* bc,
                                                             int which, int set_update) {
  pdl_wait();
  const int r = blockIdx.x;
  double s[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) s[k] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NR; ++k) s[k] += __ldcg(ba.partials + ((size_t)r * NR + k) * nblk + b);
  __shared__ double sm[32][NR];
  __shared__ bool last;
  block_sum<NR>(s, sm);
  if (threadIdx.x == 0) {
    if (rhs_active(ba, r)) fin.at(r)(s);
    __threadfence();
    const unsigned ticket = atomicInc(&bc->counter[which], gridDim.x - 1);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0 && set_update) {
    __threadfence();
    int any = 0;
    for (int q = 0; q < ba.nrhs; ++q) {
      const volatile SolverCtl* c = ba.ctl + q;
      if (!c->done && c->do_update) bc->upd_list[any++] = q;
    }
    bc->nupd = any;
    bc->any_update = any > 0;
    if (bc->in_graph) cudaGraphSetConditional((cudaGraphConditionalHandle)bc->h_update, any > 0 ? 1u : 0u);
  }
}

__global__ void batch_loop_control_kernel(BatchCtl* bc, const SolverCtl* ctl, int nrhs);

// WHILE(some system active and the step budget not used up) { iteration;
// IF(any update) { reliable updates }; loop control } as an instantiated graph.
cudaError_t build_batch_loop_graph(const Ctx& c, int prec, BatchBufs& b, const BatchLaunch& bl, cudaGraph_t* graph,
                                   cudaGraphExec_t* exec, unsigned long long* h_update, unsigned long long* h_loop);
__global__ void batch_init_kernel(SolverCtl* ctl, BatchCtl* bc, int nrhs, double tol, double delta, int max_iter,
                                  const double* kappas, const double* bnorm2, int in_graph,
                                  unsigned long long h_update, unsigned long long h_loop);

// ------------------------------------------------------------ launchers
struct BatchLaunch {
  int nrhs;
  int tr;       // right-hand sides per chunk (1, 2, 4 or 8), inner precision;
                // 0: one system per block row (dslash_rhs_kernel)
  int grid;     // multi-RHS dslash blocks (tr = 0: blocks per system), inner precision
  int blas_gx;  // site-kernel blocks per right-hand side
  int grid64 = 0;    // FP64 dslash (dslash_rhs_kernel): blocks per system; 0 = grid
  int pack = 0;      // 1: two systems per thread in FP32x2 registers (tr = 2, 4, 8
                     // systems per chunk: tr / 2 thread rows), FP32 / 16-bit storage
};

// blocks per system of the FP64 per-system dslash: the single-system grid
inline int rhs_grid64(const Geom& g, int num_sms) {
  const int b = (g.Vh + kDslashBlock - 1) / kDslashBlock;
  return b < num_sms * 16 ? b : num_sms * 16;
}

template <typename R>
inline int mrhs_grid(const BatchLaunch& bl) {
  return (sizeof(R) == 8 && bl.grid64 > 0) ? bl.grid64 : bl.grid;
}

template <typename R, class In, class G, class Epi>
void launch_dslash_mrhs(const Geom& g, const BatchLaunch& bl, const In& in, const G& gauge, int parity, int dagger,
                        const Epi& epi, const BatchArgs& ba, cudaStream_t s) {
  constexpr int NR = Epi::NRED > 0 ? Epi::NRED : 1;
  const size_t smem = tile_link_bytes<R>() + (size_t)bl.nrhs * NR * sizeof(double);
  const int grid = mrhs_grid<R>(bl);
  if (sizeof(R) == 8 || bl.tr == 0) {
    const dim3 gr(grid, bl.nrhs);
    auto go = [&](auto dag, auto tfix, auto rec8) {
      launch_pdl(dslash_rhs_kernel<decltype(dag)::value, decltype(tfix)::value, decltype(rec8)::value, R, In, G, Epi>,
                 gr, dim3(kDslashBlock), 0, s, g, in, gauge, parity, epi, ba);
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    if constexpr (sizeof(R) == 4) {
      if (gauge.recon == 8) {
        if (g.tfix) dagger ? go(T_{}, T_{}, T_{}) : go(F_{}, T_{}, T_{});
        else dagger ? go(T_{}, F_{}, T_{}) : go(F_{}, F_{}, T_{});
        return;
      }
    }
    if (g.tfix) dagger ? go(T_{}, T_{}, F_{}) : go(F_{}, T_{}, F_{});
    else dagger ? go(T_{}, F_{}, F_{}) : go(F_{}, F_{}, F_{});
    return;
  }
  const int tr = bl.tr;
  if constexpr (sizeof(R) == 4) {
    if (bl.pack) {
      const size_t smem2 = tile_link_bytes2<R>() + (size_t)bl.nrhs * NR * sizeof(double);
#define WD_MRHS2_CASE(TRV)                                                                                  \
  case TRV:                                                                                                 \
    if (dagger)                                                                                             \
      launch_pdl(dslash_mrhs2_kernel<true, In, G, Epi, TRV / 2>, dim3(grid), dim3(32, TRV / 2), smem2, s, g, \
                 in, gauge, parity, epi, ba);                                                               \
    else                                                                                                    \
      launch_pdl(dslash_mrhs2_kernel<false, In, G, Epi, TRV / 2>, dim3(grid), dim3(32, TRV / 2), smem2, s,   \
                 g, in, gauge, parity, epi, ba);                                                            \
    break;
      switch (tr) {
        WD_MRHS2_CASE(2)
        WD_MRHS2_CASE(4)
        WD_MRHS2_CASE(8)
      }
#undef WD_MRHS2_CASE
      return;
    }
  }
#define WD_MRHS_CASE(TRV)                                                                                   \
  case TRV:                                                                                                 \
    if (dagger)                                                                                             \
      launch_pdl(dslash_mrhs_kernel<true, R, In, G, Epi, TRV>, dim3(grid), dim3(32, TRV), smem, s, g, in,    \
                 gauge, parity, epi, ba);                                                                   \
    else                                                                                                    \
      launch_pdl(dslash_mrhs_kernel<false, R, In, G, Epi, TRV>, dim3(grid), dim3(32, TRV), smem, s, g, in,   \
                 gauge, parity, epi, ba);                                                                   \
    break;
  switch (tr) {
    WD_MRHS_CASE(1)
    WD_MRHS_CASE(2)
    WD_MRHS_CASE(4)
    WD_MRHS_CASE(8)
  }
#undef WD_MRHS_CASE
}

template <class Op>
void launch_sites_batch(const Geom& g, const BatchLaunch& bl, const Op& op, const BatchArgs& ba, cudaStream_t s) {
  launch_pdl(site_batch_kernel<Op>, dim3(bl.blas_gx, bl.nrhs), dim3(kBlasBlock), 0, s, g.Vh, op, ba);
}

template <int NR, class Fin>
void launch_finalize(const BatchLaunch& bl, const BatchArgs& ba, int nblk, const Fin& fin, BatchCtl* bc, int which,
                     int set_update, cudaStream_t s) {
  launch_pdl(batch_finalize_kernel<NR, Fin>, dim3(bl.nrhs), dim3(128), 0, s, ba, nblk, fin, bc, which, set_update);
}

// Fields of a batched solve: one allocation per field kind, system r's field
// at base + r * (field bytes); the solver control block has one SolverCtl per
// system.
struct BatchBufs {
  SolverCtl* ctl;
  BatchCtl* bc;
  double* partials;
  double* kappas;   // [nrhs]
  double* scal;     // [4 * nrhs] scratch scalars (|b_e|^2, |b_o|^2, residuals)
  void *b, *x;      // F64 full fields (even then odd), nrhs of them
  void *b_hat, *xe, *tmp64;             // F64 single-parity
  void *r_hat, *r_tilde, *p, *v, *t, *x_hat, *tmp;  // inner precision
};

template <int P>
struct ImplBatch {
  using T = Tr<P>;
  using S = typename T::S;
  using R = typename T::R;
  using T64 = Tr<WD_F64>;

  static size_t fb(const Geom& g) { return T::bytes(g.stride); }
  static size_t fb64(const Geom& g) { return T64::bytes(g.stride); }
  static S v(const void* p, const Geom& g) { return T::view(p, g, fb(g)); }
  static SpinorF64 v64(const void* p, const Geom& g, size_t rs) { return T64::view(p, g, rs); }

  // API: out_r = D in_r for r < nrhs (fields back to back)
  static void dslash(const Ctx& c, const BatchLaunch& bl, void* out, const void* in, int parity, int dagger,
                     cudaStream_t s) {
    EpiStore<S> e{v(out, c.g)};
    BatchArgs ba{bl.nrhs, nullptr, 0, nullptr};
    launch_dslash_mrhs<R>(c.g, bl, v(in, c.g), T::gauge(c), parity, dagger, e, ba, s);
  }

  // ---- batched BiCGstab (Sec. 5.1) with Alg. 2 reliable updates; one
  // SolverCtl per system, all systems step together, converged ones masked
  static void setup(const Ctx& c, const BatchLaunch& bl, BatchBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    BatchArgs ba{bl.nrhs, b.ctl, 0, b.partials};
    using Q = OpQuantDup<S, SpinorF64, FinBicgSetup>;
    Q q{v(b.r_hat, g), v(b.r_tilde, g), v64(b.b_hat, g, fb64(g)), c.red, FinBicgSetup{b.ctl}};
    launch_sites_batch(g, bl, q, ba, s);
    launch_finalize<3>(bl, ba, bl.blas_gx, FinBicgSetup{b.ctl}, b.bc, 0, 0, s);
    launch_sites_batch(g, bl, OpZero<S>{v(b.p, g)}, ba, s);
    launch_sites_batch(g, bl, OpZero<S>{v(b.v, g)}, ba, s);
    launch_sites_batch(g, bl, OpZero<S>{v(b.x_hat, g)}, ba, s);
  }

  static void iteration(const Ctx& c, const BatchLaunch& bl, BatchBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    BatchArgs ba{bl.nrhs, b.ctl, 0, b.partials};
    const Coef nk2{0.0, &b.ctl->neg_kappa2, (long)(sizeof(SolverCtl) / sizeof(double))};
    launch_sites_batch(g, bl, OpBicgP<S>{v(b.r_hat, g), v(b.p, g), v(b.v, g), b.ctl}, ba, s);
    EpiStore<S> e0{v(b.tmp, g)};
    launch_dslash_mrhs<R>(g, bl, v(b.p, g), T::gauge(c), 1, 0, e0, ba, s);
    EpiXpayDot<S, S, S, FinBicgAlpha> e1{v(b.v, g), v(b.p, g), v(b.r_tilde, g), nk2, c.red, FinBicgAlpha{b.ctl}};
    launch_dslash_mrhs<R>(g, bl, v(b.tmp, g), T::gauge(c), 0, 0, e1, ba, s);
    launch_finalize<2>(bl, ba, mrhs_grid<R>(bl), FinBicgAlpha{b.ctl}, b.bc, 0, 0, s);
    launch_sites_batch(g, bl, OpBicgS<S>{v(b.r_hat, g), v(b.v, g), b.ctl}, ba, s);
    launch_dslash_mrhs<R>(g, bl, v(b.r_hat, g), T::gauge(c), 1, 0, e0, ba, s);
    EpiXpayTS<S, S, FinBicgOmega> e2{v(b.t, g), v(b.r_hat, g), nk2, c.red, FinBicgOmega{b.ctl}};
    launch_dslash_mrhs<R>(g, bl, v(b.tmp, g), T::gauge(c), 0, 0, e2, ba, s);
    launch_finalize<3>(bl, ba, mrhs_grid<R>(bl), FinBicgOmega{b.ctl}, b.bc, 1, 0, s);
    OpBicgFinal<S> fo{v(b.x_hat, g), v(b.p, g), v(b.r_hat, g), v(b.t, g), v(b.r_tilde, g), b.ctl, c.red,
                      FinBicgIter{b.ctl}};
    launch_sites_batch(g, bl, fo, ba, s);
    launch_finalize<3>(bl, ba, bl.blas_gx, FinBicgIter{b.ctl}, b.bc, 2, 1, s);
  }

  // reliable update for the systems that asked for one (mode 1)
  static void update(const Ctx& c, const BatchLaunch& bl, BatchBufs& b, cudaStream_t s) {
    const Geom& g = c.g;
    BatchArgs ba{bl.nrhs, b.ctl, 1, b.partials, b.bc};
    const Coef nk2{0.0, &b.ctl->neg_kappa2, (long)(sizeof(SolverCtl) / sizeof(double))};
    launch_sites_batch(g, bl, OpAccumulate<S>{v64(b.xe, g, fb64(g)), v(b.x_hat, g)}, ba, s);
    EpiStore<SpinorF64> e0{v64(b.tmp64, g, fb64(g))};
    launch_dslash_mrhs<double>(g, bl, v64(b.xe, g, fb64(g)), T64::gauge(c), 1, 0, e0, ba, s);
    EpiRelupBicg<S, S, FinRelupBicg> e1{v64(b.b_hat, g, fb64(g)), v64(b.xe, g, fb64(g)), v(b.r_hat, g),
                                        v(b.r_tilde, g), nk2, c.red, FinRelupBicg{b.ctl}};
    launch_dslash_mrhs<double>(g, bl, v64(b.tmp64, g, fb64(g)), T64::gauge(c), 0, 0, e1, ba, s);
    launch_finalize<4>(bl, ba, mrhs_grid<double>(bl), FinRelupBicg{b.ctl}, b.bc, 3, 0, s);
  }
};

}  // namespace wd
