// Device building blocks of the Wilson-Dirac library (sm_103a).
//
// Storage formats, the 12-real link reconstruction (App. A.1), the spin
// projection of the DeGrand-Rossi projectors (App. B) onto half spinors, the
// dslash of one even-odd site (Sec. 3-4), and the deterministic FP64 grid
// reduction used for every global sum (Sec. 5.1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wd {

// ------------------------------------------------------------------ geometry
struct Geom {
  int X, Y, Z, T;
  int Xh;      // X / 2
  int Vh;      // sites of one parity
  int stride;  // elements between component arrays of a field (>= Vh)
  int tbc_anti;
};

__device__ __forceinline__ void site_coords(const Geom& g, int h, int parity, int& x, int& y, int& z, int& t) {
  int r = h;
  int xh = r % g.Xh;
  r /= g.Xh;
  y = r % g.Y;
  r /= g.Y;
  z = r % g.Z;
  t = r / g.Z;
  x = 2 * xh + ((y + z + t + parity) & 1);
}

// even-odd index of the site (x,y,z,t): lexicographic index / 2 (X even)
__device__ __forceinline__ int cb_index(const Geom& g, int x, int y, int z, int t) {
  return (x >> 1) + g.Xh * (y + g.Y * (z + g.Z * t));
}

// ----------------------------------------------------------- spinor fields
// A spinor holds 24 reals, index k = (spin * 3 + colour) * 2 + reim.
// Every format is structure-of-arrays over the sites of one parity: chunk c
// of site h lives at base[c * stride + h], so a warp reads 32 consecutive
// 16-byte words per chunk.

constexpr float kInv32767 = 3.0518509475997192e-05f;  // (float)(1.0 / 32767.0)

struct SpinorF64 {
  using real = double;
  double2* p;
  int stride;
  static constexpr int kBytesPerSite = 192;
  template <typename R>
  __device__ __forceinline__ void load(int h, R (&v)[24]) const {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 d = __ldg(p + (size_t)c * stride + h);
      v[2 * c] = (R)d.x;
      v[2 * c + 1] = (R)d.y;
    }
  }
  template <typename R>
  __device__ __forceinline__ void store(int h, const R (&v)[24]) const {
#pragma unroll
    for (int c = 0; c < 12; ++c) p[(size_t)c * stride + h] = make_double2((double)v[2 * c], (double)v[2 * c + 1]);
  }
  // store; the stored values equal v
  template <typename R>
  __device__ __forceinline__ void store_get(int h, R (&v)[24]) const {
    store(h, v);
  }
};

struct SpinorF32 {
  using real = float;
  float4* p;
  int stride;
  static constexpr int kBytesPerSite = 96;
  template <typename R>
  __device__ __forceinline__ void load(int h, R (&v)[24]) const {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 d = __ldg(p + (size_t)c * stride + h);
      v[4 * c] = (R)d.x;
      v[4 * c + 1] = (R)d.y;
      v[4 * c + 2] = (R)d.z;
      v[4 * c + 3] = (R)d.w;
    }
  }
  __device__ __forceinline__ void store_f(int h, const float (&v)[24]) const {
#pragma unroll
    for (int c = 0; c < 6; ++c) p[(size_t)c * stride + h] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  }
  template <typename R>
  __device__ __forceinline__ void store(int h, const R (&v)[24]) const {
    float f[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) f[k] = to_float(v[k]);
    store_f(h, f);
  }
  // store; v is replaced by the values as stored
  template <typename R>
  __device__ __forceinline__ void store_get(int h, R (&v)[24]) const {
    float f[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      f[k] = to_float(v[k]);
      v[k] = (R)f[k];
    }
    store_f(h, f);
  }
  static __device__ __forceinline__ float to_float(double d) { return __double2float_rn(d); }
  static __device__ __forceinline__ float to_float(float f) { return f; }
};

// 16-bit formats with one FP32 norm per site (Sec. 4.5).  Codes: 3 x 16 B.
enum class Fmt16 { Q16, H16, B16 };

template <Fmt16 F>
struct Spinor16 {
  using real = float;
  uint4* p;      // [3][stride]
  float* norm;   // [stride]
  int stride;
  static constexpr int kBytesPerSite = 52;

  static __device__ __forceinline__ float lo(uint32_t w) {
    if constexpr (F == Fmt16::Q16) return (float)(int16_t)(w & 0xffffu);
    else if constexpr (F == Fmt16::H16) return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
    else return __uint_as_float(w << 16);
  }
  static __device__ __forceinline__ float hi(uint32_t w) {
    if constexpr (F == Fmt16::Q16) return (float)(int16_t)(w >> 16);
    else if constexpr (F == Fmt16::H16) return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
    else return __uint_as_float(w & 0xffff0000u);
  }
  // raw 16-bit values as float (codes, or the normalised fp16/bf16 numbers)
  // plus the factor that turns them into field values
  __device__ __forceinline__ float load_raw(int h, float (&v)[24]) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 d = __ldg(p + (size_t)c * stride + h);
      v[8 * c + 0] = lo(d.x); v[8 * c + 1] = hi(d.x);
      v[8 * c + 2] = lo(d.y); v[8 * c + 3] = hi(d.y);
      v[8 * c + 4] = lo(d.z); v[8 * c + 5] = hi(d.z);
      v[8 * c + 6] = lo(d.w); v[8 * c + 7] = hi(d.w);
    }
    float n = __ldg(norm + h);
    if constexpr (F == Fmt16::Q16) return __fmul_rn(n, kInv32767);
    else return n;
  }
  template <typename R>
  __device__ __forceinline__ void load(int h, R (&v)[24]) const {
    float f[24];
    float s = load_raw(h, f);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = (R)__fmul_rn(f[k], s);
  }

  static __device__ __forceinline__ uint32_t enc(float w, float scale) {
    if constexpr (F == Fmt16::Q16) {
      float q = rintf(__fmul_rn(w, scale));
      q = fminf(fmaxf(q, -32767.f), 32767.f);
      return (uint32_t)(uint16_t)(int16_t)q;
    } else if constexpr (F == Fmt16::H16) {
      return (uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(w, scale)));
    } else {
      return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(__fmul_rn(w, scale)));
    }
  }
  static __device__ __forceinline__ float f32(double d) { return __double2float_rn(d); }
  static __device__ __forceinline__ float f32(float f) { return f; }

  // Encode 24 values (Sec. 4.5 format; FP32 arithmetic, see the header).
  // v is replaced by the decoded values as stored.
  template <typename R>
  __device__ __forceinline__ void store_get(int h, R (&v)[24]) const {
    float f[24];
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      f[k] = f32(v[k]);
      m = fmaxf(m, fabsf(f[k]));
    }
    float scale;
    if constexpr (F == Fmt16::Q16) scale = (m > 0.f) ? __fdiv_rn(32767.f, m) : 0.f;
    else scale = (m > 0.f) ? __fdiv_rn(1.f, m) : 0.f;
    uint32_t w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = enc(f[2 * k], scale) | (enc(f[2 * k + 1], scale) << 16);
#pragma unroll
    for (int c = 0; c < 3; ++c) p[(size_t)c * stride + h] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    norm[h] = m;
    float d = (F == Fmt16::Q16) ? __fmul_rn(m, kInv32767) : m;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      v[2 * k] = (R)__fmul_rn(lo(w[k]), d);
      v[2 * k + 1] = (R)__fmul_rn(hi(w[k]), d);
    }
  }
  template <typename R>
  __device__ __forceinline__ void store(int h, const R (&v)[24]) const {
    R t[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) t[k] = v[k];
    store_get(h, t);
  }
};

using SpinorQ16 = Spinor16<Fmt16::Q16>;
using SpinorH16 = Spinor16<Fmt16::H16>;
using SpinorB16 = Spinor16<Fmt16::B16>;

// ------------------------------------------------------------- gauge fields
// Link U_mu(x), x of parity p with even-odd index h.  Reals index
// k = (row * 3 + col) * 2 + reim.  12-real storage keeps rows a, b; the third
// row is rebuilt as c = (a x b)^* (App. A.1).  Layout [p][mu][chunk][stride].

template <typename R>
__device__ __forceinline__ void reconstruct_row3(R (&u)[18]) {
  // c_i = conj(a_j b_k - a_k b_j), (i, j, k) cyclic
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    R ajr = u[2 * j], aji = u[2 * j + 1], akr = u[2 * k], aki = u[2 * k + 1];
    R bjr = u[6 + 2 * j], bji = u[6 + 2 * j + 1], bkr = u[6 + 2 * k], bki = u[6 + 2 * k + 1];
    R re = (ajr * bkr - aji * bki) - (akr * bjr - aki * bji);
    R im = (ajr * bki + aji * bkr) - (akr * bji + aki * bjr);
    u[12 + 2 * i] = re;
    u[12 + 2 * i + 1] = -im;
  }
}

struct GaugeF64 {
  using real = double;
  const double2* p;
  int stride;
  int recon;  // 12 or 18
  __device__ __forceinline__ void load(int parity, int mu, int h, double (&u)[18]) const {
    const int nc = recon / 2;
    const double2* b = p + (size_t)(parity * 4 + mu) * nc * stride + h;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double2 d = __ldcs(b + (size_t)c * stride);
      u[2 * c] = d.x;
      u[2 * c + 1] = d.y;
    }
    if (recon == 18) {
#pragma unroll
      for (int c = 6; c < 9; ++c) {
        double2 d = __ldcs(b + (size_t)c * stride);
        u[2 * c] = d.x;
        u[2 * c + 1] = d.y;
      }
    } else {
      reconstruct_row3(u);
    }
  }
};

struct GaugeF32 {
  using real = float;
  const float4* p;
  int stride;
  __device__ __forceinline__ void load(int parity, int mu, int h, float (&u)[18]) const {
    const float4* b = p + (size_t)(parity * 4 + mu) * 3 * stride + h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 d = __ldcs(b + (size_t)c * stride);
      u[4 * c] = d.x;
      u[4 * c + 1] = d.y;
      u[4 * c + 2] = d.z;
      u[4 * c + 3] = d.w;
    }
    reconstruct_row3(u);
  }
};

template <Fmt16 F>
struct Gauge16 {
  using real = float;
  const uint4* p8;  // [p][mu][stride]: reals 0..7
  const uint2* p4;  // [p][mu][stride]: reals 8..11
  int stride;
  __device__ __forceinline__ void load(int parity, int mu, int h, float (&u)[18]) const {
    size_t o = (size_t)(parity * 4 + mu) * stride + h;
    uint4 a = __ldcs(p8 + o);
    uint2 b = __ldcs(p4 + o);
    uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
    const float s = (F == Fmt16::Q16) ? kInv32767 : 1.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      u[2 * k] = Spinor16<F>::lo(w[k]) * s;
      u[2 * k + 1] = Spinor16<F>::hi(w[k]) * s;
    }
    reconstruct_row3(u);
  }
};

using GaugeQ16 = Gauge16<Fmt16::Q16>;
using GaugeH16 = Gauge16<Fmt16::H16>;
using GaugeB16 = Gauge16<Fmt16::B16>;

// ----------------------------------------------- spin projection (App. B)
// Half spinor h[(s * 3 + c) * 2 + reim], s = 0, 1.  For the projector
// P = 1 + S gamma_mu in the DeGrand-Rossi basis the two upper rows of P psi
// determine the lower two; project() forms the upper rows, reconstruct()
// adds the full four-spinor P psi' given the transformed upper rows psi'.
//   mu = x: h0 = p0 + S i p3, h1 = p1 + S i p2;  lower = (-S i h1, -S i h0)
//   mu = y: h0 = p0 - S p3,   h1 = p1 + S p2;    lower = ( S h1,   -S h0)
//   mu = z: h0 = p0 + S i p2, h1 = p1 - S i p3;  lower = (-S i h0,  S i h1)
//   mu = t: h0 = p0 + S p2,   h1 = p1 + S p3;    lower = ( S h0,    S h1)
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const R (&p)[24], R (&h)[12]) {
  constexpr R s = (R)S;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R p0r = p[(0 + c) * 2], p0i = p[(0 + c) * 2 + 1];
    const R p1r = p[(3 + c) * 2], p1i = p[(3 + c) * 2 + 1];
    const R p2r = p[(6 + c) * 2], p2i = p[(6 + c) * 2 + 1];
    const R p3r = p[(9 + c) * 2], p3i = p[(9 + c) * 2 + 1];
    R h0r, h0i, h1r, h1i;
    if constexpr (MU == 0) {
      h0r = p0r - s * p3i; h0i = p0i + s * p3r;
      h1r = p1r - s * p2i; h1i = p1i + s * p2r;
    } else if constexpr (MU == 1) {
      h0r = p0r - s * p3r; h0i = p0i - s * p3i;
      h1r = p1r + s * p2r; h1i = p1i + s * p2i;
    } else if constexpr (MU == 2) {
      h0r = p0r - s * p2i; h0i = p0i + s * p2r;
      h1r = p1r + s * p3i; h1i = p1i - s * p3r;
    } else {
      h0r = p0r + s * p2r; h0i = p0i + s * p2i;
      h1r = p1r + s * p3r; h1i = p1i + s * p3i;
    }
    h[c * 2] = h0r; h[c * 2 + 1] = h0i;
    h[(3 + c) * 2] = h1r; h[(3 + c) * 2 + 1] = h1i;
  }
}

template <int MU, int S, typename R>
__device__ __forceinline__ void reconstruct(const R (&g)[12], R (&a)[24]) {
  constexpr R s = (R)S;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R g0r = g[c * 2], g0i = g[c * 2 + 1];
    const R g1r = g[(3 + c) * 2], g1i = g[(3 + c) * 2 + 1];
    a[(0 + c) * 2] += g0r; a[(0 + c) * 2 + 1] += g0i;
    a[(3 + c) * 2] += g1r; a[(3 + c) * 2 + 1] += g1i;
    if constexpr (MU == 0) {  // lower = (-S i g1, -S i g0); -S i z = (S z.im, -S z.re)
      a[(6 + c) * 2] += s * g1i; a[(6 + c) * 2 + 1] -= s * g1r;
      a[(9 + c) * 2] += s * g0i; a[(9 + c) * 2 + 1] -= s * g0r;
    } else if constexpr (MU == 1) {  // lower = (S g1, -S g0)
      a[(6 + c) * 2] += s * g1r; a[(6 + c) * 2 + 1] += s * g1i;
      a[(9 + c) * 2] -= s * g0r; a[(9 + c) * 2 + 1] -= s * g0i;
    } else if constexpr (MU == 2) {  // lower = (-S i g0, S i g1)
      a[(6 + c) * 2] += s * g0i; a[(6 + c) * 2 + 1] -= s * g0r;
      a[(9 + c) * 2] -= s * g1i; a[(9 + c) * 2 + 1] += s * g1r;
    } else {  // lower = (S g0, S g1)
      a[(6 + c) * 2] += s * g0r; a[(6 + c) * 2 + 1] += s * g0i;
      a[(9 + c) * 2] += s * g1r; a[(9 + c) * 2 + 1] += s * g1i;
    }
  }
}

// g = U h (DAG = false) or U^dag h (DAG = true), for both spin rows of h
template <bool DAG, typename R>
__device__ __forceinline__ void su3_mul(const R (&u)[18], const R (&h)[12], R (&g)[12]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R re = 0, im = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int e = DAG ? (j * 3 + i) : (i * 3 + j);
        const R ur = u[2 * e], ui = DAG ? -u[2 * e + 1] : u[2 * e + 1];
        const R hr = h[(s * 3 + j) * 2], hi = h[(s * 3 + j) * 2 + 1];
        re += ur * hr - ui * hi;
        im += ur * hi + ui * hr;
      }
      g[(s * 3 + i) * 2] = re;
      g[(s * 3 + i) * 2 + 1] = im;
    }
  }
}

// One hop of the stencil: acc += P^{S mu} U psi(neighbour), where
// S = -1 forward / +1 backward for D, exchanged for D^dag (Sec. 3, eq. for M).
template <int MU, bool FWD, bool DAGGER, typename R, class In, class G>
__device__ __forceinline__ void hop(const In& in, const G& gauge, int parity, int h_link, int h_nbr, bool flip,
                                    R (&acc)[24]) {
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  R psi[24];
  in.load(h_nbr, psi);
  R hs[12];
  project<MU, S>(psi, hs);
  R u[18];
  gauge.load(FWD ? parity : 1 - parity, MU, h_link, u);
  R gs[12];
  su3_mul<!FWD>(u, hs, gs);
  if (flip) {
#pragma unroll
    for (int k = 0; k < 12; ++k) gs[k] = -gs[k];
  }
  reconstruct<MU, S>(gs, acc);
}

// acc = (D in)(site h of parity `parity`), or (D^dag in)(h)
template <bool DAGGER, typename R, class In, class G>
__device__ __forceinline__ void dslash_site(const Geom& g, const In& in, const G& gauge, int h, int parity,
                                            R (&acc)[24]) {
  int x, y, z, t;
  site_coords(g, h, parity, x, y, z, t);
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0;
  {
    const int xp = (x + 1 == g.X) ? 0 : x + 1, xm = (x == 0) ? g.X - 1 : x - 1;
    hop<0, true, DAGGER>(in, gauge, parity, h, cb_index(g, xp, y, z, t), false, acc);
    const int n = cb_index(g, xm, y, z, t);
    hop<0, false, DAGGER>(in, gauge, parity, n, n, false, acc);
  }
  {
    const int yp = (y + 1 == g.Y) ? 0 : y + 1, ym = (y == 0) ? g.Y - 1 : y - 1;
    hop<1, true, DAGGER>(in, gauge, parity, h, cb_index(g, x, yp, z, t), false, acc);
    const int n = cb_index(g, x, ym, z, t);
    hop<1, false, DAGGER>(in, gauge, parity, n, n, false, acc);
  }
  {
    const int zp = (z + 1 == g.Z) ? 0 : z + 1, zm = (z == 0) ? g.Z - 1 : z - 1;
    hop<2, true, DAGGER>(in, gauge, parity, h, cb_index(g, x, y, zp, t), false, acc);
    const int n = cb_index(g, x, y, zm, t);
    hop<2, false, DAGGER>(in, gauge, parity, n, n, false, acc);
  }
  {
    const bool top = (t + 1 == g.T), bot = (t == 0);
    const int tp = top ? 0 : t + 1, tm = bot ? g.T - 1 : t - 1;
    hop<3, true, DAGGER>(in, gauge, parity, h, cb_index(g, x, y, z, tp), top && g.tbc_anti, acc);
    const int n = cb_index(g, x, y, z, tm);
    hop<3, false, DAGGER>(in, gauge, parity, n, n, bot && g.tbc_anti, acc);
  }
}

// ------------------------------------------------------- FP64 reductions
// Deterministic single-pass grid reduction (Sec. 5.1: global sums in FP64,
// tree reduction): fixed-order warp-shuffle tree inside each block, one
// partial per block, and the last block to finish (found with an atomic
// ticket that resets itself) sums the partials in block order and runs the
// finaliser.  The result depends only on the grid size, never on timing.
struct RedScratch {
  double* partials;    // >= gridDim.x * N doubles
  unsigned* counter;   // zero between reductions
};

template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double (*sm)[N]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) sm[warp][k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      v[k] = (lane < nw) ? sm[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
  }
  __syncthreads();
}

// All threads of the block call this once, after their grid-stride loop.
// fin(const double* totals) runs on one thread of the last block.
template <int N, class Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[N], const RedScratch& rs, const Fin& fin) {
  __shared__ double sm[32][N];
  __shared__ bool is_last;
  block_sum<N>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) rs.partials[(size_t)blockIdx.x * N + k] = v[k];
    __threadfence();
    unsigned ticket = atomicInc(rs.counter, gridDim.x - 1);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s[N];
#pragma unroll
  for (int k = 0; k < N; ++k) s[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] += __ldcg(rs.partials + (size_t)b * N + k);
  block_sum<N>(s, sm);
  if (threadIdx.x == 0) fin(s);
}

// ------------------------------------------------------------ small maths
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

}  // namespace wd
