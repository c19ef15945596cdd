// Device code of the atlas deposit, shared by k_deposit (deposit.cu) and the
// fused continuation + re-trace + deposit kernel (trace.cu): every stored
// photon's incident energy goes to the texel of its position in a top-down
// XZ atlas, accumulated in unsigned 64-bit fixed point (E * 2^scale_log2,
// exact power-of-two scaling then round to nearest even) so that the sum does not
// depend on the order of the atomics.  The texel decision is made in FP32
// with explicitly rounded operations (no fused multiply-add).
#pragma once
#include "pv_scene.h"

namespace pvk {

// Texel of coordinate p over [lo, hi) with res texels, given the mapping's
// scale = res / (hi - lo) (correctly rounded FP32 division, computed once per
// atlas by AtlasMap): explicitly rounded FP32, no fused multiply-add.
__device__ __forceinline__ int atlas_texel(float p, float lo, float scale, uint32_t res) {
  const float u = __fmul_rn(__fsub_rn(p, lo), scale);
  const float f = floorf(u);
  if (!(f >= 0.0f)) return 0;
  if (f >= (float)res) return (int)res - 1;
  return (int)f;
}

// An atlas with its two texel scales, worked out once per thread.
struct AtlasMap {
  pv_atlas at;
  float sx, sz;
};

__device__ __forceinline__ AtlasMap atlas_map(const pv_atlas& at) {
  AtlasMap m;
  m.at = at;
  m.sx = __fdiv_rn((float)at.width, __fsub_rn(at.x1, at.x0));
  m.sz = __fdiv_rn((float)at.height, __fsub_rn(at.z1, at.z0));
  return m;
}

// E * 2^s rounded to the nearest integer, ties to even, saturated to the
// unsigned 64-bit range: the value of float E is m * 2^(e - 150) with its
// 24-bit significand m, so the fixed-point value is m shifted by e - 150 + s,
// rounded on the bits shifted out.  Integer operations only: a float to
// 64-bit integer conversion instruction runs on the FP64 pipe, which is
// narrow on this GPU.  E <= 0 and NaN give 0, +inf gives 2^64 - 1.
__device__ __forceinline__ unsigned long long fixed_point(float E, int s) {
  const uint32_t b = __float_as_uint(E);
  if ((int32_t)b <= 0) return 0ull;                           // +0, negative numbers, negative NaNs
  const uint32_t ex = b >> 23;
  if (ex == 255u) return (b & 0x7FFFFFu) ? 0ull : ~0ull;      // NaN, +inf
  const uint32_t m = ex ? (b & 0x7FFFFFu) | 0x800000u : b;    // subnormals: exponent 1, no hidden bit
  const int sh = (int)(ex ? ex : 1u) - 150 + s;               // value = m * 2^sh
  if (sh >= 0) return sh > 40 ? ~0ull : (unsigned long long)m << sh;   // m < 2^24: fits for sh <= 40
  const int r = -sh;
  if (r > 24) return 0ull;                                    // value < 2^24 / 2^25 = 1 / 2
  const uint32_t q = m >> r;
  const uint32_t rem = m & ((1u << r) - 1u), half = 1u << (r - 1);
  return q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
}

// One photon (position x, energy e) into the atlas.
__device__ __forceinline__ void deposit_point(const AtlasMap& am, float3 x, float3 e) {
  const pv_atlas& at = am.at;
  const int tx = atlas_texel(x.x, at.x0, am.sx, at.width);
  const int tz = atlas_texel(x.z, at.z0, am.sz, at.height);
  unsigned long long* t = reinterpret_cast<unsigned long long*>(at.data) + 3 * ((size_t)tz * at.width + tx);
  atomicAdd(t, fixed_point(e.x, at.scale_log2));
  atomicAdd(t + 1, fixed_point(e.y, at.scale_log2));
  atomicAdd(t + 2, fixed_point(e.z, at.scale_log2));
}

// The first L photons of path p into the atlas, added (kSub false) or taken
// back out (kSub true: the same fixed-point values, negated modulo 2^64, so
// that a deposit followed by its removal leaves every texel's sum as it was).
template <bool kSub = false>
__device__ __forceinline__ void deposit_rows(const AtlasMap& am, uint32_t n, uint32_t L, const float4* pa,
                                             const float4* pb, uint32_t p) {
  const pv_atlas& at = am.at;
  for (uint32_t k = 0; k < L; ++k) {
    // streaming loads: the path buffers must not evict the atlas from L2
    const float4 x = __ldcs(pa + (size_t)k * n + p);
    const float4 e = __ldcs(pb + (size_t)k * n + p);
    const int tx = atlas_texel(x.x, at.x0, am.sx, at.width);
    const int tz = atlas_texel(x.z, at.z0, am.sz, at.height);
    unsigned long long* t = reinterpret_cast<unsigned long long*>(at.data) + 3 * ((size_t)tz * at.width + tx);
    const unsigned long long v[3] = {fixed_point(e.x, at.scale_log2), fixed_point(e.y, at.scale_log2),
                                     fixed_point(e.z, at.scale_log2)};
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(t + c, kSub ? 0ull - v[c] : v[c]);
  }
}

// The photons of path p (its info word's count, at most B) into the atlas.
__device__ __forceinline__ void deposit_path(const AtlasMap& am, uint32_t n, uint32_t B, const uint32_t* info,
                                             const float4* pa, const float4* pb, uint32_t p) {
  deposit_rows<false>(am, n, min(info_nseg(__ldcs(info + p)), B), pa, pb, p);
}

// The photons of the paths p of the warp's lanes (0xFFFFFFFF: none) into the
// atlas, dealt out over the lanes row by row: the warp's photon list is row 0
// of every lane's path (in lane order), then row 1 of the paths that have
// one, and so on, and photon q goes to lane q mod 32.  Every lane has a photon
// in all but the last round, whatever the paths' lengths, and lanes next to
// each other read the same row of paths next to each other (coalesced when
// the warp's paths are consecutive).  Called by all lanes of the warp.
__device__ __forceinline__ void deposit_warp(const AtlasMap& am, uint32_t n, uint32_t B, const uint32_t* info,
                                             const float4* pa, const float4* pb, uint32_t p) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t cnt = p != 0xFFFFFFFFu ? min(info_nseg(__ldcs(info + p)), B) : 0u;
  const uint32_t rows = __reduce_max_sync(0xffffffffu, cnt);
  // kk: the first row not yet dealt out in full, cum: the photons of the rows before it, m: its paths' lanes
  uint32_t kk = 0, cum = 0;
  unsigned m = __ballot_sync(0xffffffffu, cnt > 0u);
  for (uint32_t base = 0; kk < rows; base += 32) {
    const uint32_t R = base + lane;            // this lane's photon rank
    uint32_t k_own = rows, j_own = 0;
    unsigned m_own = 0u;
    // the rows this round covers (the same steps on every lane)
    while (kk < rows && cum < base + 32) {
      const uint32_t ck = __popc(m);
      if (R >= cum && R < cum + ck) {
        k_own = kk;
        j_own = R - cum;
        m_own = m;
      }
      if (cum + ck > base + 32) break;         // the row goes on in the next round
      cum += ck;
      ++kk;
      m = __ballot_sync(0xffffffffu, cnt > kk);
    }
    const uint32_t owner = k_own < rows ? __fns(m_own, 0u, (int)j_own + 1) : 0u;
    const uint32_t po = __shfl_sync(0xffffffffu, p, owner);
    if (k_own >= rows) continue;
    // streaming loads: the path buffers must not evict the atlas from L2
    const float4 x = __ldcs(pa + (size_t)k_own * n + po);
    const float4 e = __ldcs(pb + (size_t)k_own * n + po);
    deposit_point(am, make_float3(x.x, x.y, x.z), make_float3(e.x, e.y, e.z));
  }
}

}  // namespace pvk
