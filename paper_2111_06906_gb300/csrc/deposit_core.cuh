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

// The photons of path p (its info word's count, at most B) into the atlas.
__device__ __forceinline__ void deposit_path(const pv_atlas& at, uint32_t n, uint32_t B, const uint32_t* info,
                                             const float4* pa, const float4* pb, uint32_t p) {
  const uint32_t L = min(info_nseg(__ldcs(info + p)), B);
  for (uint32_t k = 0; k < L; ++k) {
    // streaming loads: the path buffers must not evict the atlas from L2
    const float4 x = __ldcs(pa + (size_t)k * n + p);
    const float4 e = __ldcs(pb + (size_t)k * n + p);
    const int tx = atlas_texel(x.x, at.x0, at.x1, at.width);
    const int tz = atlas_texel(x.z, at.z0, at.z1, at.height);
    unsigned long long* t = reinterpret_cast<unsigned long long*>(at.data) + 3 * ((size_t)tz * at.width + tx);
    atomicAdd(t + 0, __float2ull_rn(ldexpf(e.x, at.scale_log2)));
    atomicAdd(t + 1, __float2ull_rn(ldexpf(e.y, at.scale_log2)));
    atomicAdd(t + 2, __float2ull_rn(ldexpf(e.z, at.scale_log2)));
  }
}

}  // namespace pvk
