// Deposit of every stored photon's incident energy into a top-down XZ atlas
// (the stand-in for the renderer's splat / gather step of Fig. 2).  Energies
// are accumulated in unsigned 64-bit fixed point (E * 2^scale_log2, exact
// power-of-two scaling then round to nearest) so that the sum is independent
// of the order of the atomics.  The texel decision is made in FP32 with
// explicitly rounded operations (no fused multiply-add).
#include "pv_scene.h"

using namespace pvk;

namespace {

__device__ __forceinline__ int texel(float p, float lo, float hi, uint32_t res) {
  const float scale = __fdiv_rn((float)res, __fsub_rn(hi, lo));
  const float u = __fmul_rn(__fsub_rn(p, lo), scale);
  const float f = floorf(u);
  if (!(f >= 0.0f)) return 0;
  if (f >= (float)res) return (int)res - 1;
  return (int)f;
}

__global__ void __launch_bounds__(256) k_deposit(uint32_t n, uint32_t B, const uint32_t* info, const float4* pa,
                                                 const float4* pb, pv_atlas at) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t L = min(info_nseg(__ldcs(info + p)), B);
    for (uint32_t k = 0; k < L; ++k) {
      // streaming loads: the path buffers must not evict the atlas from L2
      const float4 x = __ldcs(pa + (size_t)k * n + p);
      const float4 e = __ldcs(pb + (size_t)k * n + p);
      const int tx = texel(x.x, at.x0, at.x1, at.width);
      const int tz = texel(x.z, at.z0, at.z1, at.height);
      unsigned long long* t = reinterpret_cast<unsigned long long*>(at.data) + 3 * ((size_t)tz * at.width + tx);
      atomicAdd(t + 0, __float2ull_rn(ldexpf(e.x, at.scale_log2)));
      atomicAdd(t + 1, __float2ull_rn(ldexpf(e.y, at.scale_log2)));
      atomicAdd(t + 2, __float2ull_rn(ldexpf(e.z, at.scale_log2)));
    }
  }
}

}  // namespace

extern "C" int pv_deposit(pv_scene* s, const pv_paths* paths, const pv_atlas* atlas, void* stream) {
  const int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!atlas || !atlas->data || atlas->width == 0 || atlas->height == 0) return PV_ERR_ARG;
  if (!(atlas->x1 > atlas->x0) || !(atlas->z1 > atlas->z0) || atlas->scale_log2 < 0 || atlas->scale_log2 > 62)
    return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (cudaMemsetAsync(atlas->data, 0, (size_t)atlas->width * atlas->height * 3 * sizeof(uint64_t), st) != cudaSuccess)
    return PV_ERR_CUDA;
  const uint32_t n = paths->n;
  if (n) {
    const uint32_t blocks = (uint32_t)s->num_sms * 8u;
    k_deposit<<<blocks, 256, 0, st>>>(n, s->B, paths->info, reinterpret_cast<const float4*>(paths->pa),
                                      reinterpret_cast<const float4*>(paths->pb), *atlas);
  }
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
