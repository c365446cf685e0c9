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
// Division of n < 2^31 by a fixed d with one multiply-high and a shift
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): q = (umulhi(n, m) + n) >> s with
// s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  uint32_t m;
  int s;
};

inline FastDiv make_fastdiv(int d) {
  int s = 0;
  while ((1LL << s) < d) ++s;
  const unsigned long long m = ((1ULL << 32) * ((1ULL << s) - (unsigned long long)d)) / (unsigned long long)d + 1;
  return FastDiv{(uint32_t)m, s};
}

__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  return (int)((__umulhi((uint32_t)n, f.m) + (uint32_t)n) >> f.s);
}

struct Geom {
  int X, Y, Z, T;
  int Xh;      // X / 2
  int Vh;      // sites of one parity
  int stride;  // elements between component arrays of a field (>= Vh)
  int tbc_anti;
  int tfix;           // temporal gauge (Sec. 4.3): U_4 = 1 off the slice t = T-1
  int XhY, XhYZ;      // even-odd index steps in y, z (t step is XhYZ)
  int wy, wz, wt;     // index jumps of the periodic wrap in y, z, t
  FastDiv dXh, dY, dZ;
  int h_begin, h_end;  // output sites of a dslash launch: [h_begin, h_end) (0, Vh: all)
};

inline Geom make_geom(const int dims[4], int tbc_anti) {
  Geom g{};
  g.X = dims[0];
  g.Y = dims[1];
  g.Z = dims[2];
  g.T = dims[3];
  g.Xh = dims[0] / 2;
  const long long vh = (long long)dims[0] * dims[1] * dims[2] * dims[3] / 2;
  g.Vh = (int)vh;
  g.stride = (int)((vh + 31) / 32 * 32);
  g.tbc_anti = tbc_anti ? 1 : 0;
  g.tfix = 0;
  g.XhY = g.Xh * g.Y;
  g.XhYZ = g.XhY * g.Z;
  g.wy = (g.Y - 1) * g.Xh;
  g.wz = (g.Z - 1) * g.XhY;
  g.wt = (g.T - 1) * g.XhYZ;
  g.dXh = make_fastdiv(g.Xh);
  g.dY = make_fastdiv(g.Y);
  g.dZ = make_fastdiv(g.Z);
  g.h_begin = 0;
  g.h_end = g.Vh;
  return g;
}

__device__ __forceinline__ void site_coords(const Geom& g, int h, int parity, int& x, int& y, int& z, int& t) {
  int q = fdiv(h, g.dXh);
  const int xh = h - q * g.Xh;
  int r = q;
  q = fdiv(r, g.dY);
  y = r - q * g.Y;
  r = q;
  q = fdiv(r, g.dZ);
  z = r - q * g.Z;
  t = q;
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
  static constexpr bool kScaled = false;
  static constexpr bool kIntCodes = false;
  static constexpr bool kPairedHops = false;
  double2* p;
  int stride;
  size_t rs;  // bytes from one right-hand side's field to the next (batches)
  static constexpr int kBytesPerSite = 192;
  __device__ __forceinline__ SpinorF64 at(int r) const {
    SpinorF64 v = *this;
    v.p = (double2*)((char*)p + (size_t)r * rs);
    return v;
  }
  template <typename R>
  __device__ __forceinline__ void load(int h, R (&v)[24]) const {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 d = __ldg(p + (size_t)c * stride + h);
      v[2 * c] = (R)d.x;
      v[2 * c + 1] = (R)d.y;
    }
  }
  // spins 0,1 (upper) or 2,3 (lower): 12 reals
  template <typename R>
  __device__ __forceinline__ void load_half(int h, bool upper, R (&v)[12]) const {
    const int c0 = upper ? 0 : 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double2 d = __ldg(p + (size_t)(c0 + c) * stride + h);
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
  static constexpr bool kScaled = false;
  static constexpr bool kIntCodes = false;
  static constexpr bool kPairedHops = false;
  float4* p;
  int stride;
  size_t rs;
  static constexpr int kBytesPerSite = 96;
  __device__ __forceinline__ SpinorF32 at(int r) const {
    SpinorF32 v = *this;
    v.p = (float4*)((char*)p + (size_t)r * rs);
    return v;
  }
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
  template <typename R>
  __device__ __forceinline__ void load_half(int h, bool upper, R (&v)[12]) const {
    const int c0 = upper ? 0 : 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 d = __ldg(p + (size_t)(c0 + c) * stride + h);
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

// 16-bit formats with one FP32 norm per site (Sec. 4.6).  Codes: 3 x 16 B.
enum class Fmt16 { Q16, H16, B16 };

template <Fmt16 F>
struct Spinor16 {
  using real = float;
  static constexpr bool kScaled = true;  // load_raw + one scale per site
  uint4* p;      // [3][stride]
  float* norm;   // [stride]
  int stride;
  size_t rs;
  static constexpr int kBytesPerSite = 52;
  __device__ __forceinline__ Spinor16 at(int r) const {
    Spinor16 v = *this;
    v.p = (uint4*)((char*)p + (size_t)r * rs);
    v.norm = (float*)((char*)norm + (size_t)r * rs);
    return v;
  }

  // int16 code q -> float q exactly, by the conversion unit: the 16-bit
  // stencil is issue-bound on the integer and FP32 pipes and leaves that unit
  // idle, and one conversion per code costs fewer instructions than decoding
  // the code on the busy pipes
  static __device__ __forceinline__ float q16_to_float(uint32_t half_bits) {
    return __int2float_rn((int)(short)(half_bits & 0xffffu));
  }
  static __device__ __forceinline__ float lo(uint32_t w) {
    if constexpr (F == Fmt16::Q16) return q16_to_float(w & 0xffffu);
    else if constexpr (F == Fmt16::H16) return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
    else return __uint_as_float(w << 16);
  }
  static __device__ __forceinline__ float hi(uint32_t w) {
    if constexpr (F == Fmt16::Q16) return __int2float_rn(((int)w) >> 16);
    else if constexpr (F == Fmt16::H16) return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
    else return __uint_as_float(w & 0xffff0000u);
  }
  // both values of a 32-bit word
  static __device__ __forceinline__ float2 pair(uint32_t w) {
    if constexpr (F == Fmt16::H16) {
      __half2 h = *reinterpret_cast<__half2*>(&w);
      return __half22float2(h);
    } else {
      return make_float2(lo(w), hi(w));
    }
  }
  // integer codes (Q16): the launch shapes of their kernels differ
  static constexpr bool kIntCodes = (F == Fmt16::Q16);
  // spin-paired hops (wd_async.cuh) for Q16 and bf16, whose decodes run on the
  // conversion and integer pipes; fp16 decodes run on the FMA pipe, which the
  // paired arithmetic keeps full, and fp16 is faster with the scalar hops
  static constexpr bool kPairedHops = (F != Fmt16::H16);
  // the factor that turns raw values into field values, from the site norm
  static __device__ __forceinline__ float scale_of(float n) {
    if constexpr (F == Fmt16::Q16) return __fmul_rn(n, kInv32767);
    else return n;
  }
  // 24 raw values from the 12 stored words
  static __device__ __forceinline__ void words(const uint32_t (&w)[12], float (&v)[24]) {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const float2 f = pair(w[j]);
      v[2 * j] = f.x;
      v[2 * j + 1] = f.y;
    }
  }
  // 12 raw values of half a spinor from its 6 words
  static __device__ __forceinline__ void words_half(const uint32_t (&w)[6], float (&v)[12]) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float2 f = pair(w[j]);
      v[2 * j] = f.x;
      v[2 * j + 1] = f.y;
    }
  }
  // raw 16-bit values as float (codes, or the normalised fp16/bf16 numbers)
  // plus the factor that turns them into field values
  __device__ __forceinline__ float load_raw(int h, float (&v)[24]) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 d = __ldg(p + (size_t)c * stride + h);
      const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = pair(w[j]);
        v[8 * c + 2 * j] = f.x;
        v[8 * c + 2 * j + 1] = f.y;
      }
    }
    float n = __ldg(norm + h);
    if constexpr (F == Fmt16::Q16) return __fmul_rn(n, kInv32767);
    else return n;
  }
  // spins 0,1 (values 0..11: chunk 0 and the first half of chunk 1) or
  // spins 2,3 (values 12..23: the second half of chunk 1 and chunk 2)
  __device__ __forceinline__ float load_raw_half(int h, bool upper, float (&v)[12]) const {
    uint32_t w[6];
    if (upper) {
      const uint4 a = __ldg(p + h);
      const uint2 b = __ldg(reinterpret_cast<const uint2*>(p + (size_t)stride + h));
      w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y;
    } else {
      const uint2 a = __ldg(reinterpret_cast<const uint2*>(p + (size_t)stride + h) + 1);
      const uint4 b = __ldg(p + (size_t)2 * stride + h);
      w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y; w[4] = b.z; w[5] = b.w;
    }
    words_half(w, v);
    return scale_of(__ldg(norm + h));
  }
  template <typename R>
  __device__ __forceinline__ void load(int h, R (&v)[24]) const {
    float f[24];
    const float s = load_raw(h, f);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = (R)__fmul_rn(f[k], s);
  }

  static __device__ __forceinline__ float f32(double d) { return __double2float_rn(d); }
  static __device__ __forceinline__ float f32(float f) { return f; }

  // Encode 24 values (Sec. 4.6 format; FP32 arithmetic, see the header).
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
    if constexpr (F == Fmt16::Q16) {
      // q = rint(f * scale) without a conversion instruction: s = fl(f * scale)
      // + 1.5 * 2^23 rounds to the nearest integer, ties to even, because
      // |fl(f * scale)| <= 32767 (1 + 2^-24)^2 < 2^22 (so no clamp is needed
      // either: m is the largest |f|); the low 16 bits of s are then q in two's
      // complement, and s - 1.5 * 2^23 = q exactly
      constexpr float kMagic = 12582912.0f;
      float sv[24];
#pragma unroll
      for (int k = 0; k < 24; ++k) sv[k] = __fadd_rn(__fmul_rn(f[k], scale), kMagic);
      uint32_t w[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) w[k] = __byte_perm(__float_as_uint(sv[2 * k]), __float_as_uint(sv[2 * k + 1]), 0x5410);
#pragma unroll
      for (int c = 0; c < 3; ++c) p[(size_t)c * stride + h] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
      norm[h] = m;
      const float d = __fmul_rn(m, kInv32767);
#pragma unroll
      for (int k = 0; k < 24; ++k) v[k] = (R)__fmul_rn(__fsub_rn(sv[k], kMagic), d);
      return;
    }
    // fp16 / bf16: both values of a word rounded (to nearest, ties to even,
    // each) by one packing conversion
    uint32_t w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 t = make_float2(__fmul_rn(f[2 * k], scale), __fmul_rn(f[2 * k + 1], scale));
      if constexpr (F == Fmt16::H16) {
        const __half2 q = __floats2half2_rn(t.x, t.y);
        w[k] = *reinterpret_cast<const uint32_t*>(&q);
      } else {
        const __nv_bfloat162 q = __floats2bfloat162_rn(t.x, t.y);
        w[k] = *reinterpret_cast<const uint32_t*>(&q);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) p[(size_t)c * stride + h] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    norm[h] = m;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 q = pair(w[k]);
      v[2 * k] = (R)__fmul_rn(q.x, m);
      v[2 * k + 1] = (R)__fmul_rn(q.y, m);
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
// Link words are read once per dslash: streaming loads (evict first).
template <class T>
__device__ __forceinline__ T ld_link(const T* p) {
  return __ldcs(p);
}

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
    R re = ajr * bkr;
    re -= aji * bki;
    re -= akr * bjr;
    re += aki * bji;
    R im = ajr * bki;
    im += aji * bkr;
    im -= akr * bji;
    im -= aki * bjr;
    u[12 + 2 * i] = re;
    u[12 + 2 * i + 1] = -im;
  }
}

// App. A.2: the link from its 8 stored numbers p = {arg a1, arg c1, a2, a3,
// b1} (complex a2, a3, b1 as re, im): |a1|^2 = 1 - |a2|^2 - |a3|^2 and
// |c1|^2 = 1 - |a1|^2 - |b1|^2 = |a2|^2 + |a3|^2 - |b1|^2 (negative arguments
// from rounding set to 0); with N^2 = |a2|^2 + |a3|^2 the unit vectors
// b' = (0, -a3^*, a2^*)/N and c' = (a x b')^* = (N, -a1^* a2/N, -a1^* a3/N)
// span the plane orthogonal to row a, and rows b, c are their SU(2) rotation
// with p2 = b1/N, p1 = c1^*/N: b = p1 b' + p2 c', c = -p2^* b' + p1^* c'.
// FAST: the SFU sine/cosine (16-bit storage, whose quantisation dominates).
template <bool FAST>
__device__ __forceinline__ void su3_from8(const float (&p)[8], float (&u)[18]) {
  const float a2r = p[2], a2i = p[3], a3r = p[4], a3i = p[5], b1r = p[6], b1i = p[7];
  float n2 = a2r * a2r;
  n2 += a2i * a2i;
  n2 += a3r * a3r;
  n2 += a3i * a3i;
  const float rn = rsqrtf(n2);  // 1/N
  float b12 = b1r * b1r;
  b12 += b1i * b1i;
  const float a1m = sqrtf(fmaxf(0.f, 1.f - n2));
  const float c1m = sqrtf(fmaxf(0.f, n2 - b12));
  float sa, ca, sc, cc;
  if constexpr (FAST) {
    __sincosf(p[0], &sa, &ca);
    __sincosf(p[1], &sc, &cc);
  } else {
    sincosf(p[0], &sa, &ca);
    sincosf(p[1], &sc, &cc);
  }
  const float a1r = a1m * ca, a1i = a1m * sa;
  const float c1r = c1m * cc, c1i = c1m * sc;
  // p2 = b1 / N, p1 = conj(c1) / N
  const float p2r = b1r * rn, p2i = b1i * rn;
  const float p1r = c1r * rn, p1i = -c1i * rn;
  // b' = (0, -conj(a3), conj(a2)) / N
  const float bp1r = -a3r * rn, bp1i = a3i * rn;
  const float bp2r = a2r * rn, bp2i = -a2i * rn;
  // c' = (N, -conj(a1) a2 / N, -conj(a1) a3 / N)
  float t;
  t = a1r * a2r;
  t += a1i * a2i;
  const float cp1r = -t * rn;
  t = a1r * a2i;
  t -= a1i * a2r;
  const float cp1i = -t * rn;
  t = a1r * a3r;
  t += a1i * a3i;
  const float cp2r = -t * rn;
  t = a1r * a3i;
  t -= a1i * a3r;
  const float cp2i = -t * rn;
  u[0] = a1r; u[1] = a1i; u[2] = a2r; u[3] = a2i; u[4] = a3r; u[5] = a3i;
  // row b: (b1, p1 b'_1 + p2 c'_1, p1 b'_2 + p2 c'_2)
  u[6] = b1r; u[7] = b1i;
  // row c: (c1, -conj(p2) b'_1 + conj(p1) c'_1, ...)
  u[12] = c1r; u[13] = c1i;
  const float bpr[2] = {bp1r, bp2r}, bpi[2] = {bp1i, bp2i}, cpr[2] = {cp1r, cp2r}, cpi[2] = {cp1i, cp2i};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float re = p1r * bpr[j];
    re -= p1i * bpi[j];
    re += p2r * cpr[j];
    re -= p2i * cpi[j];
    float im = p1r * bpi[j];
    im += p1i * bpr[j];
    im += p2r * cpi[j];
    im += p2i * cpr[j];
    u[8 + 2 * j] = re;
    u[9 + 2 * j] = im;
    // -conj(p2) b' + conj(p1) c'
    re = -p2r * bpr[j];
    re -= p2i * bpi[j];
    re += p1r * cpr[j];
    re += p1i * cpi[j];
    im = -p2r * bpi[j];
    im += p2i * bpr[j];
    im += p1r * cpi[j];
    im -= p1i * cpr[j];
    u[14 + 2 * j] = re;
    u[15 + 2 * j] = im;
  }
}

struct GaugeF64 {
  using real = double;
  static constexpr bool kScaled = false;
  static constexpr double kScale = 1.0;
  const double2* p;
  int stride;
  int recon;  // 12 or 18
  template <bool R8, typename R>
  __device__ __forceinline__ void load_scaled(int parity, int mu, int h, double (&u)[18], R& w) const {
    load_scaled_slot<R8>(parity * 4 + mu, h, u, w);
  }
  template <bool R8>
  __device__ __forceinline__ void load(int parity, int mu, int h, double (&u)[18]) const {
    load_slot(parity * 4 + mu, h, u);
  }
  // slot = parity * 4 + mu in a gauge field; a link face (one boundary
  // slice of temporal links) has one slot per parity
  template <bool R8, typename R>
  __device__ __forceinline__ void load_scaled_slot(int slot, int h, double (&u)[18], R&) const {
    load_slot(slot, h, u);
  }
  __device__ __forceinline__ void load_slot(int slot, int h, double (&u)[18]) const {
    const int nc = recon / 2;
    const double2* b = p + (size_t)slot * nc * stride + h;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double2 d = ld_link(b + (size_t)c * stride);
      u[2 * c] = d.x;
      u[2 * c + 1] = d.y;
    }
    if (recon == 18) {
#pragma unroll
      for (int c = 6; c < 9; ++c) {
        double2 d = ld_link(b + (size_t)c * stride);
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
  static constexpr bool kScaled = false;
  static constexpr float kScale = 1.f;
  const float4* p;
  int stride;
  int recon;  // 12: rows a, b (3 float4 per link); 8: App. A.2 numbers (2 float4)
  // R8: the kernel variant for recon == 8 (a compile-time choice, so the
  // 12-real kernels carry none of the 8-number code)
  template <bool R8, typename R>
  __device__ __forceinline__ void load_scaled(int parity, int mu, int h, float (&u)[18], R&) const {
    load_slot<R8>(parity * 4 + mu, h, u);
  }
  template <bool R8>
  __device__ __forceinline__ void load(int parity, int mu, int h, float (&u)[18]) const {
    load_slot<R8>(parity * 4 + mu, h, u);
  }
  template <bool R8, typename R>
  __device__ __forceinline__ void load_scaled_slot(int slot, int h, float (&u)[18], R&) const {
    load_slot<R8>(slot, h, u);
  }
  template <bool R8>
  __device__ __forceinline__ void load_slot(int slot, int h, float (&u)[18]) const {
    if constexpr (R8) {
      const float4* b = p + (size_t)slot * 2 * stride + h;
      const float4 d0 = ld_link(b), d1 = ld_link(b + stride);
      const float q[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
      su3_from8<false>(q, u);
      return;
    }
    const float4* b = p + (size_t)slot * 3 * stride + h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 d = ld_link(b + (size_t)c * stride);
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
  // Q16 links are used as raw codes: load_raw returns 32767 U (row c rebuilt
  // from the raw rows and rescaled), and kScale = 1/32767 is folded into the
  // accumulation.  fp16 / bf16 links hold U itself.
  static constexpr bool kScaled = (F == Fmt16::Q16);
  static constexpr float kScale = kInv32767;
  const uint4* p8;  // [p][mu][stride]: reals 0..7 (recon 12) or the 8 numbers of App. A.2
  const uint2* p4;  // [p][mu][stride]: reals 8..11 (recon 12)
  int stride;
  int recon;  // 12 or 8
  // App. A.2 numbers decoded to the link.  The two angles are 16-bit fixed
  // point in every 16-bit format (code = rint(32767 angle / pi)); a2, a3, b1
  // use the format's own encoding.
  __device__ __forceinline__ void load8(int parity, int mu, int h, float (&u)[18]) const {
    const uint4 a = ld_link(p8 + (size_t)(parity * 4 + mu) * stride + h);
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
    constexpr float kPiQ = 3.14159265358979f * kInv32767;
    float q[8];
    q[0] = Spinor16<Fmt16::Q16>::lo(w[0]) * kPiQ;
    q[1] = Spinor16<Fmt16::Q16>::hi(w[0]) * kPiQ;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      const float2 f = Spinor16<F>::pair(w[k]);
      q[2 * k] = f.x;
      q[2 * k + 1] = f.y;
    }
    if constexpr (F == Fmt16::Q16) {
#pragma unroll
      for (int k = 2; k < 8; ++k) q[k] *= kInv32767;
    }
    su3_from8<true>(q, u);
  }
  // the link values times 1/w' folded into w: Q16 12-real links come back as
  // raw codes (w *= 1/32767), everything else as values.  R8: the kernel
  // variant for recon == 8 (compile-time).
  template <bool R8, typename R>
  __device__ __forceinline__ void load_scaled(int parity, int mu, int h, float (&u)[18], R& w) const {
    if constexpr (R8) {
      load8(parity, mu, h, u);
    } else {
      load_raw_slot(parity * 4 + mu, h, u);
      if constexpr (F == Fmt16::Q16) w *= (R)kInv32767;
    }
  }
  // a link face (12-real links only): slot = parity
  template <bool R8, typename R>
  __device__ __forceinline__ void load_scaled_slot(int slot, int h, float (&u)[18], R& w) const {
    static_assert(!R8, "link faces hold 12-real links");
    load_raw_slot(slot, h, u);
    if constexpr (F == Fmt16::Q16) w *= (R)kInv32767;
  }
  __device__ __forceinline__ void load_raw(int parity, int mu, int h, float (&u)[18]) const {
    load_raw_slot(parity * 4 + mu, h, u);
  }
  __device__ __forceinline__ void load_raw_slot(int slot, int h, float (&u)[18]) const {
    size_t o = (size_t)slot * stride + h;
    uint4 a = ld_link(p8 + o);
    uint2 b = ld_link(p4 + o);
    const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
    from_words(w, u);
  }
  // the link from its 6 stored words (rows a, b): row c rebuilt, Q16 as raw
  // codes (32767 U; the caller folds in 1/32767)
  static __device__ __forceinline__ void from_words(const uint32_t (&w)[6], float (&u)[18]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float2 f = Spinor16<F>::pair(w[k]);
      u[2 * k] = f.x;
      u[2 * k + 1] = f.y;
    }
    reconstruct_row3(u);
    if constexpr (F == Fmt16::Q16) {
#pragma unroll
      for (int k = 12; k < 18; ++k) u[k] *= kInv32767;
    }
  }
  template <bool R8>
  __device__ __forceinline__ void load(int parity, int mu, int h, float (&u)[18]) const {
    if constexpr (R8) {
      load8(parity, mu, h, u);
      return;
    }
    load_raw(parity, mu, h, u);
    if constexpr (F == Fmt16::Q16) {
#pragma unroll
      for (int k = 0; k < 18; ++k) u[k] *= kInv32767;
    }
  }
};

using GaugeQ16 = Gauge16<Fmt16::Q16>;
using GaugeH16 = Gauge16<Fmt16::H16>;
using GaugeB16 = Gauge16<Fmt16::B16>;

// ----------------------------------------------- spin projection (App. B)
// The kernels work in the "non-relativistic" (UKQCD) basis of App. B, in
// which gamma_4 = diag(1,1,-1,-1): a temporal hop needs only two spin
// components of the neighbour (P^{+4} = diag(2,2,0,0), P^{-4} = diag(0,0,2,2)),
// so it loads half a spinor.  Fields cross the host boundary in the
// DeGrand-Rossi basis; import/export apply the basis change (psi_UK = S
// psi_DR, see OpImport).  In this basis gamma_1 and gamma_3 are those of the
// DeGrand-Rossi set and gamma_2 has the opposite sign.
// Half spinor h[(s * 3 + c) * 2 + reim], s = 0, 1.  For the spatial
// projectors P = 1 + S gamma_mu the two upper rows of P psi determine the
// lower two; project() forms the upper rows, reconstruct() adds the full
// four-spinor given the transformed upper rows g (here S2 = -S for y):
//   mu = x: h0 = p0 + S i p3,  h1 = p1 + S i p2;   lower = (-S i g1, -S i g0)
//   mu = y: h0 = p0 - S2 p3,   h1 = p1 + S2 p2;    lower = ( S2 g1,  -S2 g0)
//   mu = z: h0 = p0 + S i p2,  h1 = p1 - S i p3;   lower = (-S i g0,  S i g1)
template <int MU, int S_, typename R>
__device__ __forceinline__ void project(const R (&p)[24], R (&h)[12]) {
  static_assert(MU < 3, "temporal hops are diagonal in this basis");
  constexpr int S = (MU == 1) ? -S_ : S_;
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
    } else {
      h0r = p0r - s * p2i; h0i = p0i + s * p2r;
      h1r = p1r + s * p3i; h1i = p1i - s * p3r;
    }
    h[c * 2] = h0r; h[c * 2 + 1] = h0i;
    h[(3 + c) * 2] = h1r; h[(3 + c) * 2 + 1] = h1i;
  }
}

template <int MU, int S_, typename R>
__device__ __forceinline__ void reconstruct(const R (&g)[12], R (&a)[24]) {
  static_assert(MU < 3, "temporal hops are diagonal in this basis");
  constexpr int S = (MU == 1) ? -S_ : S_;
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
    } else {  // mu = z: lower = (-S i g0, S i g1)
      a[(6 + c) * 2] += s * g0i; a[(6 + c) * 2 + 1] -= s * g0r;
      a[(9 + c) * 2] -= s * g1i; a[(9 + c) * 2 + 1] += s * g1r;
    }
  }
}

// reconstruct() with every term scaled by w (the decode scale of a 16-bit
// neighbour and link, times a boundary sign): a += w P psi' in one FFMA each
template <int MU, int S_, typename R>
__device__ __forceinline__ void reconstruct_scaled(const R (&g)[12], R (&a)[24], R w) {
  static_assert(MU < 3, "temporal hops are diagonal in this basis");
  constexpr int S = (MU == 1) ? -S_ : S_;
  const R ws = w * (R)S;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R g0r = g[c * 2], g0i = g[c * 2 + 1];
    const R g1r = g[(3 + c) * 2], g1i = g[(3 + c) * 2 + 1];
    a[(0 + c) * 2] += w * g0r; a[(0 + c) * 2 + 1] += w * g0i;
    a[(3 + c) * 2] += w * g1r; a[(3 + c) * 2 + 1] += w * g1i;
    if constexpr (MU == 0) {
      a[(6 + c) * 2] += ws * g1i; a[(6 + c) * 2 + 1] -= ws * g1r;
      a[(9 + c) * 2] += ws * g0i; a[(9 + c) * 2 + 1] -= ws * g0r;
    } else if constexpr (MU == 1) {
      a[(6 + c) * 2] += ws * g1r; a[(6 + c) * 2 + 1] += ws * g1i;
      a[(9 + c) * 2] -= ws * g0r; a[(9 + c) * 2 + 1] -= ws * g0i;
    } else {
      a[(6 + c) * 2] += ws * g0i; a[(6 + c) * 2 + 1] -= ws * g0r;
      a[(9 + c) * 2] -= ws * g1i; a[(9 + c) * 2 + 1] += ws * g1r;
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
      // one FMA per real product: each accumulation is its own statement
      // (an expression "re += a*b - c*d" costs a multiply, an FMA and an add)
      R re = 0, im = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int e = DAG ? (j * 3 + i) : (i * 3 + j);
        const R ur = u[2 * e], ui = u[2 * e + 1];
        const R hr = h[(s * 3 + j) * 2], hi = h[(s * 3 + j) * 2 + 1];
        if constexpr (DAG) {  // conj(U_ji) h_j
          re += ur * hr;
          re += ui * hi;
          im += ur * hi;
          im -= ui * hr;
        } else {  // U_ij h_j
          re += ur * hr;
          re -= ui * hi;
          im += ur * hi;
          im += ui * hr;
        }
      }
      g[(s * 3 + i) * 2] = re;
      g[(s * 3 + i) * 2 + 1] = im;
    }
  }
}

// One hop of the stencil: acc += P^{S mu} U psi(neighbour), where
// S = -1 forward / +1 backward for D, exchanged for D^dag (Sec. 3, eq. for M).
// Temporal hop: P^{S 4} = 2 x (projector on spins 0,1 for S = +1, on 2,3 for
// S = -1); acc on those spins += 2 w (U or U^dag) psi_half
template <bool FWD, bool UPPER, typename R>
__device__ __forceinline__ void accumulate_temporal(const R (&g)[12], R (&a)[24], R w2) {
  constexpr int o = UPPER ? 0 : 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) a[o + k] += w2 * g[k];
}

// TFIX and off_slice: the link is the unit matrix (temporal gauge away from
// the last time slice): no link load and no SU(3) multiply.
template <bool FWD, bool DAGGER, bool TFIX, bool R8, typename R, class In, class G>
__device__ __forceinline__ void hop_t(const In& in, const G& gauge, int parity, int h_link, int h_nbr, bool flip,
                                      bool off_slice, R (&acc)[24]) {
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  constexpr bool upper = (S == +1);
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
  if constexpr (TFIX) {
    if (off_slice) {
      accumulate_temporal<FWD, upper>(hs, acc, flip ? -(R)2 * w : (R)2 * w);
      return;
    }
  }
  R u[18];
  gauge.template load_scaled<R8>(FWD ? parity : 1 - parity, 3, h_link, u, w);
  R gs[12];
  su3_mul<!FWD>(u, hs, gs);
  accumulate_temporal<FWD, upper>(gs, acc, flip ? -(R)2 * w : (R)2 * w);
}

template <int MU, bool FWD, bool DAGGER, bool R8, typename R, class In, class G>
__device__ __forceinline__ void hop(const In& in, const G& gauge, int parity, int h_link, int h_nbr, bool flip,
                                    R (&acc)[24]) {
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  constexpr bool kScaled = In::kScaled || G::kScaled;
  R psi[24];
  R w = 1;
  R hs[12];
  if constexpr (In::kScaled) w = in.load_raw(h_nbr, psi);
  else in.load(h_nbr, psi);
  project<MU, S>(psi, hs);
  R u[18];
  gauge.template load_scaled<R8>(FWD ? parity : 1 - parity, MU, h_link, u, w);
  R gs[12];
  su3_mul<!FWD>(u, hs, gs);
  if constexpr (kScaled) {
    reconstruct_scaled<MU, S>(gs, acc, flip ? -w : w);
  } else {
    if (flip) {
#pragma unroll
      for (int k = 0; k < 12; ++k) gs[k] = -gs[k];
    }
    reconstruct<MU, S>(gs, acc);
  }
}

// Lower spin rows of reconstruct(): a_lower (+)= S' L_mu(g), assigned when
// ASSIGN (the first direction of a site).
template <int MU, int S_, bool ASSIGN, typename R>
__device__ __forceinline__ void reconstruct_lower(const R (&g)[12], R (&a)[24]) {
  constexpr int S = (MU == 1) ? -S_ : S_;
  constexpr R s = (R)S;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R g0r = g[c * 2], g0i = g[c * 2 + 1];
    const R g1r = g[(3 + c) * 2], g1i = g[(3 + c) * 2 + 1];
    R l0r, l0i, l1r, l1i;  // rows 2 and 3
    if constexpr (MU == 0) {
      l0r = s * g1i; l0i = -s * g1r; l1r = s * g0i; l1i = -s * g0r;
    } else if constexpr (MU == 1) {
      l0r = s * g1r; l0i = s * g1i; l1r = -s * g0r; l1i = -s * g0i;
    } else {
      l0r = s * g0i; l0i = -s * g0r; l1r = -s * g1i; l1i = s * g1r;
    }
    if constexpr (ASSIGN) {
      a[(6 + c) * 2] = l0r; a[(6 + c) * 2 + 1] = l0i;
      a[(9 + c) * 2] = l1r; a[(9 + c) * 2 + 1] = l1i;
    } else {
      a[(6 + c) * 2] += l0r; a[(6 + c) * 2 + 1] += l0i;
      a[(9 + c) * 2] += l1r; a[(9 + c) * 2 + 1] += l1i;
    }
  }
}

__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The forward and backward hops of one spatial direction together, for
// unscaled fields (FP64, FP32).  With X = U_mu(x) P_f psi(x + mu) and
// B = U_mu^dag(x - mu) P_b psi(x - mu) (P_b the projector of opposite sign),
// the pair adds X + B to the upper spin rows and S' L_mu(X - B) to the lower
// ones.  One FMA chain forms Y = X + B starting from X, and X - B = 2X - Y:
// 12 adds fewer than two separate hops; the first direction of a site
// (FIRST) assigns its 24 values instead of adding them to zeros.
template <int MU, bool DAGGER, bool R8, bool FIRST, typename R, class In, class G>
__device__ __forceinline__ void hop_pair(const In& in, const G& gauge, int parity, int h, int np, int nm,
                                         R (&acc)[24]) {
  constexpr int SF = DAGGER ? +1 : -1;  // hop()'s S of the forward hop; the backward one has -SF
  R psi[24];
  R w = 1;
  in.load(np, psi);
  R hf[12];
  project<MU, SF>(psi, hf);
  R u[18];
  gauge.template load_scaled<R8>(parity, MU, h, u, w);
  R xd[12];  // X, then X - B
  su3_mul<false>(u, hf, xd);
  in.load(nm, psi);
  R hb[12];
  project<MU, -SF>(psi, hb);
  gauge.template load_scaled<R8>(1 - parity, MU, nm, u, w);
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int k = (sp * 3 + i) * 2;
      R re = xd[k], im = xd[k + 1];
#pragma unroll
      for (int j = 0; j < 3; ++j) {  // + conj(U_ji) hb_j, one FMA per real product
        const int e = j * 3 + i;
        const R ur = u[2 * e], ui = u[2 * e + 1];
        const R hr = hb[(sp * 3 + j) * 2], hi = hb[(sp * 3 + j) * 2 + 1];
        re += ur * hr;
        re += ui * hi;
        im += ur * hi;
        im -= ui * hr;
      }
      if constexpr (FIRST) {
        acc[k] = re;
        acc[k + 1] = im;
      } else {
        acc[k] += re;
        acc[k + 1] += im;
      }
      // one explicit FMA each: written as 2 x - y, the compiler turns 2 x
      // into x + x and the FMA into two adds (on GB300's FP64 pipe, 12 more
      // instructions per direction)
      xd[k] = fma_rn((R)2, xd[k], -re);
      xd[k + 1] = fma_rn((R)2, xd[k + 1], -im);
    }
  }
  reconstruct_lower<MU, SF, FIRST>(xd, acc);
}

// acc = (D in)(site h of parity `parity`), or (D^dag in)(h).  Neighbour
// indices by offsets from h: in the even-odd order a step in y, z, t moves
// the index by X/2, XY/2, XYZ/2; a step in x moves it by 0 or 1 depending on
// the parity of x.
// TFIX: the links are in the temporal gauge (g.tfix), so the temporal links
// are 1 off the last time slice (a compile-time variant: the kernels for
// general links carry no branch for it).
// PAIR: unscaled fields (FP64, FP32) take the spatial directions as hop pairs
// (hop_pair); the kernels ask for it only without fused reductions, where the
// pairs' longer live ranges cost no spills (with reductions, the FP64
// reliable-update kernel spilled 96 bytes and the solve lost 0.9 ms).
template <bool DAGGER, bool TFIX, bool R8, bool PAIR = false, typename R, class In, class G>
__device__ __forceinline__ void dslash_site(const Geom& g, const In& in, const G& gauge, int h, int parity,
                                            R (&acc)[24]) {
  int x, y, z, t;
  site_coords(g, h, parity, x, y, z, t);
  constexpr bool kPair = PAIR && !(In::kScaled || G::kScaled);
  if constexpr (!kPair) {
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
  }
  {
    const int xo = x & 1;
    const int np = (x == g.X - 1) ? h - (g.Xh - 1) : h + xo;
    const int nm = (x == 0) ? h + (g.Xh - 1) : h - (xo ^ 1);
    if constexpr (kPair) {
      hop_pair<0, DAGGER, R8, true>(in, gauge, parity, h, np, nm, acc);
    } else {
      hop<0, true, DAGGER, R8>(in, gauge, parity, h, np, false, acc);
      hop<0, false, DAGGER, R8>(in, gauge, parity, nm, nm, false, acc);
    }
  }
  {
    const int np = (y == g.Y - 1) ? h - g.wy : h + g.Xh;
    const int nm = (y == 0) ? h + g.wy : h - g.Xh;
    if constexpr (kPair) {
      hop_pair<1, DAGGER, R8, false>(in, gauge, parity, h, np, nm, acc);
    } else {
      hop<1, true, DAGGER, R8>(in, gauge, parity, h, np, false, acc);
      hop<1, false, DAGGER, R8>(in, gauge, parity, nm, nm, false, acc);
    }
  }
  {
    const int np = (z == g.Z - 1) ? h - g.wz : h + g.XhY;
    const int nm = (z == 0) ? h + g.wz : h - g.XhY;
    if constexpr (kPair) {
      hop_pair<2, DAGGER, R8, false>(in, gauge, parity, h, np, nm, acc);
    } else {
      hop<2, true, DAGGER, R8>(in, gauge, parity, h, np, false, acc);
      hop<2, false, DAGGER, R8>(in, gauge, parity, nm, nm, false, acc);
    }
  }
  {
    const bool top = (t == g.T - 1), bot = (t == 0);
    const int np = top ? h - g.wt : h + g.XhYZ;
    const int nm = bot ? h + g.wt : h - g.XhYZ;
    hop_t<true, DAGGER, TFIX, R8>(in, gauge, parity, h, np, top && g.tbc_anti, !top, acc);
    hop_t<false, DAGGER, TFIX, R8>(in, gauge, parity, nm, nm, bot && g.tbc_anti, !bot, acc);
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
