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
// atlas, dealt out over the lanes: photon q of the warp's list (paths in lane
// order, each path's photons in order) goes to lane q mod 32, so every lane
// has a photon in all but the last round, whatever the paths' lengths.
// Called by all lanes of the warp.
__device__ __forceinline__ void deposit_warp(const AtlasMap& am, uint32_t n, uint32_t B, const uint32_t* info,
                                             const float4* pa, const float4* pb, uint32_t p) {
  const int lane = threadIdx.x & 31;
  const uint32_t cnt = p != 0xFFFFFFFFu ? min(info_nseg(__ldcs(info + p)), B) : 0u;
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  const pv_atlas& at = am.at;
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t q = base + lane;
    uint32_t lo = 0, hi = 31;                  // owner: first lane whose inclusive count exceeds q
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const uint32_t mid = (lo + hi) >> 1;
      if (q < __shfl_sync(0xffffffffu, incl, mid)) hi = mid;
      else lo = mid + 1;
    }
    const uint32_t o_incl = __shfl_sync(0xffffffffu, incl, lo), o_cnt = __shfl_sync(0xffffffffu, cnt, lo);
    const uint32_t po = __shfl_sync(0xffffffffu, p, lo);
    if (q >= total) continue;
    const uint32_t k = q - (o_incl - o_cnt);
    // streaming loads: the path buffers must not evict the atlas from L2
    const float4 x = __ldcs(pa + (size_t)k * n + po);
    const float4 e = __ldcs(pb + (size_t)k * n + po);
    const int tx = atlas_texel(x.x, at.x0, am.sx, at.width);
    const int tz = atlas_texel(x.z, at.z0, am.sz, at.height);
    unsigned long long* t = reinterpret_cast<unsigned long long*>(at.data) + 3 * ((size_t)tz * at.width + tx);
    atomicAdd(t, fixed_point(e.x, at.scale_log2));
    atomicAdd(t + 1, fixed_point(e.y, at.scale_log2));
    atomicAdd(t + 2, fixed_point(e.z, at.scale_log2));
  }
}

}  // namespace pvk
