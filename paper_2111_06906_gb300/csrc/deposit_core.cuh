// Device code of the atlas deposit, shared by k_deposit (deposit.cu) and the
// fused continuation + re-trace + deposit kernel (trace.cu): every stored
// photon's incident energy goes to the texel of its position in a top-down
// XZ atlas, accumulated in unsigned 64-bit fixed point (E * 2^scale_log2,
// exact power-of-two scaling then round to nearest) so that the sum does not
// depend on the order of the atomics.  The texel decision is made in FP32
// with explicitly rounded operations (no fused multiply-add).
#pragma once
#include "pv_scene.h"

namespace pvk {

__device__ __forceinline__ int atlas_texel(float p, float lo, float hi, uint32_t res) {
  const float scale = __fdiv_rn((float)res, __fsub_rn(hi, lo));
  const float u = __fmul_rn(__fsub_rn(p, lo), scale);
  const float f = floorf(u);
  if (!(f >= 0.0f)) return 0;
  if (f >= (float)res) return (int)res - 1;
  return (int)f;
}

// The first L photons of path p into the atlas, added (kSub false) or taken
// back out (kSub true: the same fixed-point values, negated modulo 2^64, so
// that a deposit followed by its removal leaves every texel's sum as it was).
template <bool kSub = false>
__device__ __forceinline__ void deposit_rows(const pv_atlas& at, uint32_t n, uint32_t L, const float4* pa,
                                             const float4* pb, uint32_t p) {
  for (uint32_t k = 0; k < L; ++k) {
    // streaming loads: the path buffers must not evict the atlas from L2
    const float4 x = __ldcs(pa + (size_t)k * n + p);
    const float4 e = __ldcs(pb + (size_t)k * n + p);
    const int tx = atlas_texel(x.x, at.x0, at.x1, at.width);
    const int tz = atlas_texel(x.z, at.z0, at.z1, at.height);
    unsigned long long* t = reinterpret_cast<unsigned long long*>(at.data) + 3 * ((size_t)tz * at.width + tx);
    const unsigned long long v[3] = {__float2ull_rn(ldexpf(e.x, at.scale_log2)),
                                     __float2ull_rn(ldexpf(e.y, at.scale_log2)),
                                     __float2ull_rn(ldexpf(e.z, at.scale_log2))};
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(t + c, kSub ? 0ull - v[c] : v[c]);
  }
}

// The photons of path p (its info word's count, at most B) into the atlas.
__device__ __forceinline__ void deposit_path(const pv_atlas& at, uint32_t n, uint32_t B, const uint32_t* info,
                                             const float4* pa, const float4* pb, uint32_t p) {
  deposit_rows<false>(at, n, min(info_nseg(__ldcs(info + p)), B), pa, pb, p);
}

}  // namespace pvk
