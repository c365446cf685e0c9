// T-slab domain decomposition, device side: the paper names multi-GPU
// operation as its next step (Sec. 6).  A rank owns the time slices
// t0 .. t0 + T - 1 of the lattice (its context's T is the slab thickness,
// even, so local and global parities agree) and the whole spatial volume.
// Per dslash it needs from each time neighbour one boundary slice of the
// input spinor, projected by the temporal hop's projector: in the internal
// (UKQCD) basis of App. B gamma_4 = diag(1, 1, -1, -1), so the projection is
// one half spinor (spins 0,1 or 2,3), 12 reals per site -- the same half the
// temporal hop of the stencil loads.  The backward hop of the first slice
// also needs U_4 on the lower neighbour's last slice ("link face", sent once
// per gauge field).
//
// Faces are single-slice arrays indexed by the site's even-odd index within
// its slice, (x/2) + X/2 (y + Y z), of `fs` = round32(X Y Z / 2) entries:
//   spinor face  F64: 6 x double2 [6][fs];  F32: 3 x float4 [3][fs];
//                16-bit: uint4 [fs] + uint2 [fs] (the 12 values as 6 words)
//                + float norm [fs] (the site's norm, unchanged)
//   link face    both parities of the slice, one slot per parity:
//                F64 [2][recon/2][fs] double2; F32 [2][3][fs] float4;
//                16-bit uint4 [2][fs] + uint2 [2][fs]
// Packing copies stored words (no decode, no re-encode), so a face carries
// exactly the values the sender's field holds.
#pragma once

#include "wd_device.cuh"

namespace wd {

inline int face_stride(const Geom& g) { return (g.XhYZ + 31) / 32 * 32; }

// Half-spinor faces as hop_t inputs: load_half / load_raw_half return the 12
// stored values (the face already holds the half the receiving hop needs).
struct FaceF64 {
  using real = double;
  static constexpr bool kScaled = false;
  const double2* p;
  int stride;
  template <typename R>
  __device__ __forceinline__ void load_half(int h, bool, R (&v)[12]) const {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double2 d = __ldg(p + (size_t)c * stride + h);
      v[2 * c] = (R)d.x;
      v[2 * c + 1] = (R)d.y;
    }
  }
};

struct FaceF32 {
  using real = float;
  static constexpr bool kScaled = false;
  const float4* p;
  int stride;
  template <typename R>
  __device__ __forceinline__ void load_half(int h, bool, R (&v)[12]) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 d = __ldg(p + (size_t)c * stride + h);
      v[4 * c] = (R)d.x;
      v[4 * c + 1] = (R)d.y;
      v[4 * c + 2] = (R)d.z;
      v[4 * c + 3] = (R)d.w;
    }
  }
};

template <Fmt16 F>
struct Face16 {
  using real = float;
  static constexpr bool kScaled = true;
  const uint4* a;
  const uint2* b;
  const float* norm;
  int stride;
  __device__ __forceinline__ float load_raw_half(int h, bool, float (&v)[12]) const {
    const uint4 x = __ldg(a + h);
    const uint2 y = __ldg(b + h);
    const uint32_t w[6] = {x.x, x.y, x.z, x.w, y.x, y.y};
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float2 f = Spinor16<F>::pair(w[j]);
      v[2 * j] = f.x;
      v[2 * j + 1] = f.y;
    }
    const float n = __ldg(norm + h);
    if constexpr (F == Fmt16::Q16) return __fmul_rn(n, kInv32767);
    else return n;
  }
};

// A link face seen through the gauge interface of hop_t: the slot is the
// link's parity (mu is always the temporal direction).
template <class G>
struct LinkFace {
  using real = typename G::real;
  static constexpr bool kScaled = G::kScaled;
  G g;
  template <bool R8, typename R>
  __device__ __forceinline__ void load_scaled(int parity, int, int h, R (&u)[18], R& w) const {
    g.template load_scaled_slot<R8>(parity, h, u, w);
  }
};

// (D in)(h) on a slab: spatial hops as on the whole lattice, temporal hops at
// the slab's first and last slice read the received halos.  lo: the lower
// neighbour's projected last slice and its link face; hi: the upper
// neighbour's projected first slice.  flip_lo / flip_hi: the halo crosses
// t = T_global - 1 <-> 0 with an antiperiodic time direction (factor -1).
template <bool DAGGER, typename R, class In, class G, class Fc, class LF>
__device__ __forceinline__ void dslash_site_slab(const Geom& g, const In& in, const G& gauge, const Fc& face_lo,
                                                 const Fc& face_hi, const LF& link_lo, bool flip_lo, bool flip_hi,
                                                 int h, int parity, R (&acc)[24]) {
  int x, y, z, t;
  site_coords(g, h, parity, x, y, z, t);
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0;
  {
    const int xo = x & 1;
    const int np = (x == g.X - 1) ? h - (g.Xh - 1) : h + xo;
    const int nm = (x == 0) ? h + (g.Xh - 1) : h - (xo ^ 1);
    hop<0, true, DAGGER, false>(in, gauge, parity, h, np, false, acc);
    hop<0, false, DAGGER, false>(in, gauge, parity, nm, nm, false, acc);
  }
  {
    const int np = (y == g.Y - 1) ? h - g.wy : h + g.Xh;
    const int nm = (y == 0) ? h + g.wy : h - g.Xh;
    hop<1, true, DAGGER, false>(in, gauge, parity, h, np, false, acc);
    hop<1, false, DAGGER, false>(in, gauge, parity, nm, nm, false, acc);
  }
  {
    const int np = (z == g.Z - 1) ? h - g.wz : h + g.XhY;
    const int nm = (z == 0) ? h + g.wz : h - g.XhY;
    hop<2, true, DAGGER, false>(in, gauge, parity, h, np, false, acc);
    hop<2, false, DAGGER, false>(in, gauge, parity, nm, nm, false, acc);
  }
  const int ts = g.XhYZ;  // sites of one parity per time slice
  if (t == g.T - 1)
    hop_t<true, DAGGER, false, false>(face_hi, gauge, parity, h, h - ts * (g.T - 1), flip_hi, false, acc);
  else
    hop_t<true, DAGGER, false, false>(in, gauge, parity, h, h + ts, false, false, acc);
  if (t == 0)
    hop_t<false, DAGGER, false, false>(face_lo, link_lo, parity, h, h, flip_lo, false, acc);
  else
    hop_t<false, DAGGER, false, false>(in, gauge, parity, h - ts, h - ts, false, false, acc);
}

// Output sites of a region: 0 = interior slices 1 .. T-2 (no halo needed, runs
// while the faces are exchanged), 1 = the two boundary slices, 2 = all.
struct SlabRegion {
  int kind, ts, T, Vh;
  __host__ __device__ __forceinline__ int count() const {
    return kind == 0 ? ts * (T - 2) : kind == 1 ? (T > 1 ? 2 * ts : ts) : Vh;
  }
  __device__ __forceinline__ int site(int i) const {
    if (kind == 0) return i + ts;
    if (kind == 1) return i < ts ? i : i + ts * (T - 2);
    return i;
  }
};

// Resident blocks per SM the register allocation is held to: the same choice
// as for the whole-lattice dslash kernels (FP64 3; FP32 and 16-bit 5, where
// the halo branches of the boundary slices fit without spills).
template <typename R, class In>
struct SlabOccupancy {
  static constexpr int kMinBlocks = (sizeof(R) == 8) ? 3 : 5;
};

template <bool DAGGER, typename R, class In, class G, class Fc, class LF, class Epi>
__global__ void __launch_bounds__(128, (SlabOccupancy<R, In>::kMinBlocks)) dslash_slab_kernel(Geom g, In in, G gauge, Fc face_lo, Fc face_hi,
                                                          LF link_lo, int flip_lo, int flip_hi, int parity,
                                                          SlabRegion reg, Epi epi) {
  static_assert(Epi::NRED == 0, "slab dslash epilogues carry no reduction");
  const int n = reg.count();
  double red[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int h = reg.site(i);
    R acc[24];
    dslash_site_slab<DAGGER>(g, in, gauge, face_lo, face_hi, link_lo, flip_lo != 0, flip_hi != 0, h, parity, acc);
    epi(h, acc, red);
  }
}

// ---- packing.  Spinor faces of one single-parity field: lo <- slice 0,
// hi <- slice T-1, each the half that the neighbour's hop projects onto:
// the lower neighbour's forward hop takes the lower half for D (upper for
// D^dag), the upper neighbour's backward hop the upper half for D (lower for
// D^dag).
__device__ __forceinline__ bool face_lo_upper(int dagger) { return dagger != 0; }
__device__ __forceinline__ bool face_hi_upper(int dagger) { return dagger == 0; }

static __global__ void pack_faces_f64_kernel(Geom g, const double2* in, int stride, double2* lo, double2* hi, int fs,
                                      int dagger) {
  const int ts = g.XhYZ;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ts; i += gridDim.x * blockDim.x) {
    const bool top = i >= ts;
    const int hf = top ? i - ts : i;
    const int h = top ? hf + ts * (g.T - 1) : hf;
    const bool upper = top ? face_hi_upper(dagger) : face_lo_upper(dagger);
    double2* out = top ? hi : lo;
    const int c0 = upper ? 0 : 6;
    for (int c = 0; c < 6; ++c) out[(size_t)c * fs + hf] = in[(size_t)(c0 + c) * stride + h];
  }
}

static __global__ void pack_faces_f32_kernel(Geom g, const float4* in, int stride, float4* lo, float4* hi, int fs,
                                      int dagger) {
  const int ts = g.XhYZ;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ts; i += gridDim.x * blockDim.x) {
    const bool top = i >= ts;
    const int hf = top ? i - ts : i;
    const int h = top ? hf + ts * (g.T - 1) : hf;
    const bool upper = top ? face_hi_upper(dagger) : face_lo_upper(dagger);
    float4* out = top ? hi : lo;
    const int c0 = upper ? 0 : 3;
    for (int c = 0; c < 3; ++c) out[(size_t)c * fs + hf] = in[(size_t)(c0 + c) * stride + h];
  }
}

// 16-bit: the upper half is chunk 0 and the first two words of chunk 1, the
// lower half the last two words of chunk 1 and chunk 2; the norm goes along
static __global__ void pack_faces_16_kernel(Geom g, const uint4* in, const float* norm, int stride, uint4* lo_a,
                                     uint2* lo_b, float* lo_n, uint4* hi_a, uint2* hi_b, float* hi_n, int fs,
                                     int dagger) {
  const int ts = g.XhYZ;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ts; i += gridDim.x * blockDim.x) {
    const bool top = i >= ts;
    const int hf = top ? i - ts : i;
    const int h = top ? hf + ts * (g.T - 1) : hf;
    const bool upper = top ? face_hi_upper(dagger) : face_lo_upper(dagger);
    const uint4 c0 = in[h], c1 = in[(size_t)stride + h], c2 = in[(size_t)2 * stride + h];
    uint4 a;
    uint2 b;
    if (upper) {
      a = c0;
      b = make_uint2(c1.x, c1.y);
    } else {
      a = make_uint4(c1.z, c1.w, c2.x, c2.y);
      b = make_uint2(c2.z, c2.w);
    }
    (top ? hi_a : lo_a)[hf] = a;
    (top ? hi_b : lo_b)[hf] = b;
    (top ? hi_n : lo_n)[hf] = norm[h];
  }
}

// Link face: U_4 of the last slice, both parities, in the gauge copy's own
// words.  `words` 16-byte (or 8-byte) words per link in the gauge layout
// [parity * 4 + mu][words][stride] are copied to [parity][words][fs].
template <class W>
__global__ void pack_link_face_kernel(Geom g, const W* gauge, int words, int stride, W* out, int fs) {
  const int ts = g.XhYZ;
  const int n = 2 * ts * words;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int hf = i % ts;
    const int rest = i / ts;
    const int w = rest % words, q = rest / words;
    const int h = hf + ts * (g.T - 1);
    out[((size_t)q * words + w) * fs + hf] = gauge[((size_t)(q * 4 + 3) * words + w) * stride + h];
  }
}

}  // namespace wd
