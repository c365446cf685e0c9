// The dslash of one site for 16-bit storage (Sec. 4.6) with its neighbour
// data staged through shared memory by asynchronous copies (cp.async).
//
// Each thread owns three stages of shared-memory slots (structure of arrays
// by thread, so a warp's accesses are conflict-free).  A stage holds one
// neighbour's stored words (a spinor: 3 x 16 B of codes and the 4 B norm; a
// temporal half spinor: 24 B and the norm) and the link of the hop (16 B +
// 8 B).  While hop k is computed the copies for hops k+1 and k+2 are in
// flight, so the loads of eight hops overlap with the arithmetic without
// holding any register; the arithmetic is that of hop() and hop_t() (the
// same decoders, projections, SU(3) products and reconstructions, in the
// same order).  Copies are ordered per thread: no thread reads another's
// slots, so no barrier is needed.  16-byte spinor words bypass L1 (.cg: the
// slots take most of the SM's shared memory and L1 is small); link words go
// with an L2 evict-first policy.
#pragma once

#include "wd_device.cuh"

namespace wd {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16_cg(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// link words are read once per dslash: copies with an L2 evict-first policy,
// so that they do not displace the neighbour spinors that other sites reuse
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp16_cg_ef(void* dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp8_ca_ef(void* dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp8_ca(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4_ca(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kAsyncBlock = 128;  // threads per block of the kernels that use these slots
constexpr bool kSpinPairs = true;  // packed FP32 pairs over spin rows (async_hop_pairs)
constexpr int kAsyncStages = 3;

struct AsyncSlots {
  uint4 sp[kAsyncStages][3][kAsyncBlock];  // spinor words (temporal: 24 B in chunks 0, 1)
  float sn[kAsyncStages][kAsyncBlock];     // site norm
  uint4 l4[kAsyncStages][kAsyncBlock];     // link words 0..3
  uint2 l2[kAsyncStages][kAsyncBlock];     // link words 4, 5
};

// hops in the order of dslash_site: x+, x-, y+, y-, z+, z-, t+, t-
template <int K>
struct HopK {
  static constexpr int MU = K / 2;
  static constexpr bool FWD = (K % 2) == 0;
  static constexpr int ST = K % kAsyncStages;
};

template <int K, bool DAGGER, bool TFIX, class In, class G>
__device__ __forceinline__ void async_issue(AsyncSlots& sm, const In& in, const G& gauge, int parity, int h,
                                            const int (&nb)[8], bool top, bool bot) {
  using H = HopK<K>;
  const int tid = threadIdx.x;
  const int n = nb[K];
  const size_t st = (size_t)in.stride;
  if constexpr (H::MU < 3) {
#pragma unroll
    for (int c = 0; c < 3; ++c) cp16_cg(&sm.sp[H::ST][c][tid], in.p + c * st + n);
  } else {
    constexpr int S = (H::FWD != DAGGER) ? -1 : +1;
    if constexpr (S == +1) {  // spins 0, 1: chunk 0 and the first half of chunk 1
      cp16_cg(&sm.sp[H::ST][0][tid], in.p + n);
      cp8_ca(&sm.sp[H::ST][1][tid], reinterpret_cast<const uint2*>(in.p + st + n));
    } else {  // spins 2, 3: the second half of chunk 1 and chunk 2
      cp8_ca(&sm.sp[H::ST][0][tid], reinterpret_cast<const uint2*>(in.p + st + n) + 1);
      cp16_cg(&sm.sp[H::ST][1][tid], in.p + 2 * st + n);
    }
  }
  cp4_ca(&sm.sn[H::ST][tid], in.norm + n);
  // the temporal links of the temporal gauge are 1 off the last slice
  const bool unit = TFIX && H::MU == 3 && (H::FWD ? !top : !bot);
  if (!unit) {
    const int slot = (H::FWD ? parity : 1 - parity) * 4 + H::MU;
    const size_t o = (size_t)slot * gauge.stride + (H::FWD ? h : n);
    const uint64_t pol = l2_evict_first();
    cp16_cg_ef(&sm.l4[H::ST][tid], gauge.p8 + o, pol);
    cp8_ca_ef(&sm.l2[H::ST][tid], gauge.p4 + o, pol);
  }
}

template <int K, bool DAGGER, bool TFIX, class In, class G>
__device__ __forceinline__ void async_hop(const AsyncSlots& sm, const Geom& g, bool top, bool bot, float (&acc)[24]) {
  using H = HopK<K>;
  constexpr int MU = H::MU;
  constexpr bool FWD = H::FWD;
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  const int tid = threadIdx.x;
  float w = In::scale_of(sm.sn[H::ST][tid]);
  const bool unit = TFIX && MU == 3 && (FWD ? !top : !bot);
  float u[18];
  if (!unit) {
    const uint4 a = sm.l4[H::ST][tid];
    const uint2 b = sm.l2[H::ST][tid];
    const uint32_t lw[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
    G::from_words(lw, u);
    if constexpr (G::kScaled) w *= G::kScale;  // Q16 links come back as raw codes
  }
  if constexpr (MU < 3) {
    uint32_t sw[12];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 d = sm.sp[H::ST][c][tid];
      sw[4 * c] = d.x; sw[4 * c + 1] = d.y; sw[4 * c + 2] = d.z; sw[4 * c + 3] = d.w;
    }
    float psi[24], hs[12];
    In::words(sw, psi);
    project<MU, S>(psi, hs);
    float gs[12];
    su3_mul<!FWD>(u, hs, gs);
    reconstruct_scaled<MU, S>(gs, acc, w);
  } else {
    constexpr bool upper = (S == +1);
    uint32_t hw[6];
    if constexpr (upper) {
      const uint4 a = sm.sp[H::ST][0][tid];
      const uint2 b = *reinterpret_cast<const uint2*>(&sm.sp[H::ST][1][tid]);
      hw[0] = a.x; hw[1] = a.y; hw[2] = a.z; hw[3] = a.w; hw[4] = b.x; hw[5] = b.y;
    } else {
      const uint2 a = *reinterpret_cast<const uint2*>(&sm.sp[H::ST][0][tid]);
      const uint4 b = sm.sp[H::ST][1][tid];
      hw[0] = a.x; hw[1] = a.y; hw[2] = b.x; hw[3] = b.y; hw[4] = b.z; hw[5] = b.w;
    }
    float hs[12];
    In::words_half(hw, hs);
    const bool flip = g.tbc_anti && (FWD ? top : bot);
    if (unit) {
      accumulate_temporal<FWD, upper>(hs, acc, flip ? -2.f * w : 2.f * w);
    } else {
      float gs[12];
      su3_mul<!FWD>(u, hs, gs);
      accumulate_temporal<FWD, upper>(gs, acc, flip ? -2.f * w : 2.f * w);
    }
  }
}

// ---------------------------------------------------------------------------
// The same hops on spin pairs, with the packed FP32 operations of the sm_100
// family (FFMA2, FMUL2: two lanes per instruction).  Every link element
// multiplies two spin rows of the projected half spinor, so a packed operation
// takes one element in both lanes and the pair (row 0, row 1).  The
// accumulator holds pairs over spins (0, 1) and (3, 2); with that order every
// reconstruction adds pair to pair except the lower rows of the z hop.  Each
// value is computed by the operations of the scalar path, in its order and
// with the same roundings (projections by +-1 multipliers are exact), so the
// results are those of dslash_site.
// acc2[c * 2 + ri] = (spin 0, spin 1), acc2[6 + c * 2 + ri] = (spin 3, spin 2)
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// g = U h (DAG false) or U^dag h (DAG true) on spin pairs: hr[j], hi[j] are
// the real and imaginary parts of colour j of the two rows
template <bool DAG>
__device__ __forceinline__ void su3_mul_pairs(const float (&u)[18], const float2 (&hr)[3], const float2 (&hi)[3],
                                              float2 (&gr)[3], float2 (&gi)[3]) {
  float2 nh[3];  // -hi for U h, -hr for U^dag h
#pragma unroll
  for (int j = 0; j < 3; ++j) nh[j] = __fmul2_rn(DAG ? hr[j] : hi[j], dup2(-1.f));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int e = DAG ? (j * 3 + i) : (i * 3 + j);
      const float2 ur = dup2(u[2 * e]), ui = dup2(u[2 * e + 1]);
      if (j == 0) {  // + 0, as the scalar path's first term (a zero sum is +0)
        gr[i] = __ffma2_rn(ur, hr[0], dup2(0.f));
        gi[i] = __ffma2_rn(ur, hi[0], dup2(0.f));
      } else {
        gr[i] = __ffma2_rn(ur, hr[j], gr[i]);
        gi[i] = __ffma2_rn(ur, hi[j], gi[i]);
      }
      if constexpr (DAG) {  // conj(U_ji) h_j
        gr[i] = __ffma2_rn(ui, hi[j], gr[i]);
        gi[i] = __ffma2_rn(ui, nh[j], gi[i]);
      } else {  // U_ij h_j
        gr[i] = __ffma2_rn(ui, nh[j], gr[i]);
        gi[i] = __ffma2_rn(ui, hr[j], gi[i]);
      }
    }
  }
}

// reconstruct_scaled() on spin pairs
template <int MU, int S_>
__device__ __forceinline__ void reconstruct_pairs(const float2 (&gr)[3], const float2 (&gi)[3], float2 (&a)[12],
                                                  float w) {
  constexpr int S = (MU == 1) ? -S_ : S_;
  const float ws = w * (float)S;
  const float2 wp = dup2(w);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a[2 * c] = __ffma2_rn(wp, gr[c], a[2 * c]);
    a[2 * c + 1] = __ffma2_rn(wp, gi[c], a[2 * c + 1]);
    float2& lr = a[6 + 2 * c];
    float2& li = a[6 + 2 * c + 1];
    if constexpr (MU == 0) {  // spin 3 += -S i g0, spin 2 += -S i g1
      lr = __ffma2_rn(dup2(ws), gi[c], lr);
      li = __ffma2_rn(dup2(-ws), gr[c], li);
    } else if constexpr (MU == 1) {  // spin 3 += -S g0, spin 2 += S g1
      lr = __ffma2_rn(make_float2(-ws, ws), gr[c], lr);
      li = __ffma2_rn(make_float2(-ws, ws), gi[c], li);
    } else {  // spin 3 += S i g1, spin 2 += -S i g0: crosses the pair
      lr.x = fmaf(-ws, gi[c].y, lr.x);
      lr.y = fmaf(ws, gi[c].x, lr.y);
      li.x = fmaf(ws, gr[c].y, li.x);
      li.y = fmaf(-ws, gr[c].x, li.y);
    }
  }
}

template <int K, bool DAGGER, bool TFIX, class In, class G>
__device__ __forceinline__ void async_hop_pairs(const AsyncSlots& sm, const Geom& g, bool top, bool bot,
                                                float2 (&acc)[12]) {
  using H = HopK<K>;
  constexpr int MU = H::MU;
  constexpr bool FWD = H::FWD;
  constexpr int S = (FWD != DAGGER) ? -1 : +1;
  const int tid = threadIdx.x;
  float w = In::scale_of(sm.sn[H::ST][tid]);
  const bool unit = TFIX && MU == 3 && (FWD ? !top : !bot);
  float u[18];
  if (!unit) {
    const uint4 a = sm.l4[H::ST][tid];
    const uint2 b = sm.l2[H::ST][tid];
    const uint32_t lw[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
    G::from_words(lw, u);
    if constexpr (G::kScaled) w *= G::kScale;  // Q16 links come back as raw codes
  }
  float2 hr[3], hi[3];
  if constexpr (MU < 3) {
    uint32_t sw[12];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 d = sm.sp[H::ST][c][tid];
      sw[4 * c] = d.x; sw[4 * c + 1] = d.y; sw[4 * c + 2] = d.z; sw[4 * c + 3] = d.w;
    }
    // project() on pairs: p = (spin 0, spin 1) and q = (spin 3, spin 2), or
    // (spin 2, spin 3) for z; word s * 3 + c holds (re, im) of spin s, colour c
    // (each word decoded whole, as the scalar path does: fp16 pairs convert
    // in one instruction)
    constexpr int qa = (MU == 2) ? 2 : 3, qb = (MU == 2) ? 3 : 2;
    constexpr float s = (float)((MU == 1) ? -S : S);
    float2 pw[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) pw[j] = In::pair(sw[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 pr = make_float2(pw[c].x, pw[3 + c].x);
      const float2 pi = make_float2(pw[c].y, pw[3 + c].y);
      const float2 qr = make_float2(pw[qa * 3 + c].x, pw[qb * 3 + c].x);
      const float2 qi = make_float2(pw[qa * 3 + c].y, pw[qb * 3 + c].y);
      if constexpr (MU == 0) {  // h0 = p0 + s i p3, h1 = p1 + s i p2
        hr[c] = __ffma2_rn(dup2(-s), qi, pr);
        hi[c] = __ffma2_rn(dup2(s), qr, pi);
      } else if constexpr (MU == 1) {  // h0 = p0 - s p3, h1 = p1 + s p2
        hr[c] = __ffma2_rn(make_float2(-s, s), qr, pr);
        hi[c] = __ffma2_rn(make_float2(-s, s), qi, pi);
      } else {  // h0 = p0 + s i p2, h1 = p1 - s i p3
        hr[c] = __ffma2_rn(make_float2(-s, s), qi, pr);
        hi[c] = __ffma2_rn(make_float2(s, -s), qr, pi);
      }
    }
    float2 gr[3], gi[3];
    su3_mul_pairs<!FWD>(u, hr, hi, gr, gi);
    reconstruct_pairs<MU, S>(gr, gi, acc, w);
  } else {
    constexpr bool upper = (S == +1);
    uint32_t hw[6];
    if constexpr (upper) {
      const uint4 a = sm.sp[H::ST][0][tid];
      const uint2 b = *reinterpret_cast<const uint2*>(&sm.sp[H::ST][1][tid]);
      hw[0] = a.x; hw[1] = a.y; hw[2] = a.z; hw[3] = a.w; hw[4] = b.x; hw[5] = b.y;
    } else {
      const uint2 a = *reinterpret_cast<const uint2*>(&sm.sp[H::ST][0][tid]);
      const uint4 b = sm.sp[H::ST][1][tid];
      hw[0] = a.x; hw[1] = a.y; hw[2] = b.x; hw[3] = b.y; hw[4] = b.z; hw[5] = b.w;
    }
    // rows of the half spinor: (spin 0, spin 1) upper; (spin 3, spin 2) lower,
    // the order of the accumulator pairs
    constexpr int ra = upper ? 0 : 3, rb = upper ? 3 : 0;
    float2 pw[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) pw[j] = In::pair(hw[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hr[c] = make_float2(pw[ra + c].x, pw[rb + c].x);
      hi[c] = make_float2(pw[ra + c].y, pw[rb + c].y);
    }
    const bool flip = g.tbc_anti && (FWD ? top : bot);
    const float2 t2 = dup2(flip ? -2.f * w : 2.f * w);
    constexpr int o = upper ? 0 : 6;
    if (unit) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[o + 2 * c] = __ffma2_rn(t2, hr[c], acc[o + 2 * c]);
        acc[o + 2 * c + 1] = __ffma2_rn(t2, hi[c], acc[o + 2 * c + 1]);
      }
    } else {
      float2 gr[3], gi[3];
      su3_mul_pairs<!FWD>(u, hr, hi, gr, gi);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[o + 2 * c] = __ffma2_rn(t2, gr[c], acc[o + 2 * c]);
        acc[o + 2 * c + 1] = __ffma2_rn(t2, gi[c], acc[o + 2 * c + 1]);
      }
    }
  }
}

template <int K, bool DAGGER, bool TFIX, class In, class G>
__device__ __forceinline__ void async_step_pairs(AsyncSlots& sm, const Geom& g, const In& in, const G& gauge,
                                                 int parity, int h, const int (&nb)[8], bool top, bool bot,
                                                 float2 (&acc)[12]) {
  if constexpr (K + 2 < 8) async_issue<K + 2, DAGGER, TFIX>(sm, in, gauge, parity, h, nb, top, bot);
  cp_commit();
  cp_wait<2>();  // the copies of hop K have landed
  async_hop_pairs<K, DAGGER, TFIX, In, G>(sm, g, top, bot, acc);
}

template <int K, bool DAGGER, bool TFIX, class In, class G>
__device__ __forceinline__ void async_step(AsyncSlots& sm, const Geom& g, const In& in, const G& gauge, int parity,
                                           int h, const int (&nb)[8], bool top, bool bot, float (&acc)[24]) {
  if constexpr (K + 2 < 8) async_issue<K + 2, DAGGER, TFIX>(sm, in, gauge, parity, h, nb, top, bot);
  cp_commit();
  cp_wait<2>();  // the copies of hop K have landed
  async_hop<K, DAGGER, TFIX, In, G>(sm, g, top, bot, acc);
}

// acc = (D in)(h) (or D^dag), 16-bit spinors and 12-real 16-bit links; the
// caller's block has kAsyncBlock threads.
template <bool DAGGER, bool TFIX, class In, class G>
__device__ __forceinline__ void dslash_site_async(const Geom& g, const In& in, const G& gauge, int h, int parity,
                                                  float (&acc)[24]) {
  __shared__ AsyncSlots sm;
  int x, y, z, t;
  site_coords(g, h, parity, x, y, z, t);
  int nb[8];
  {
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
  const bool top = (t == g.T - 1), bot = (t == 0);
  async_issue<0, DAGGER, TFIX>(sm, in, gauge, parity, h, nb, top, bot);
  cp_commit();
  async_issue<1, DAGGER, TFIX>(sm, in, gauge, parity, h, nb, top, bot);
  cp_commit();
  if constexpr (kSpinPairs && In::kPairedHops) {
    float2 a2[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) a2[k] = make_float2(0.f, 0.f);
    async_step_pairs<0, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
    async_step_pairs<1, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
    async_step_pairs<2, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
    async_step_pairs<3, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
    async_step_pairs<4, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
    async_step_pairs<5, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
    async_step_pairs<6, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
    async_step_pairs<7, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, a2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int ri = 0; ri < 2; ++ri) {
        acc[(0 + c) * 2 + ri] = a2[2 * c + ri].x;
        acc[(3 + c) * 2 + ri] = a2[2 * c + ri].y;
        acc[(9 + c) * 2 + ri] = a2[6 + 2 * c + ri].x;
        acc[(6 + c) * 2 + ri] = a2[6 + 2 * c + ri].y;
      }
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0.f;
  async_step<0, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
  async_step<1, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
  async_step<2, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
  async_step<3, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
  async_step<4, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
  async_step<5, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
  async_step<6, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
  async_step<7, DAGGER, TFIX>(sm, g, in, gauge, parity, h, nb, top, bot, acc);
}

}  // namespace wd
