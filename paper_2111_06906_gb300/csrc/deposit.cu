// Deposit of every stored photon's incident energy into a top-down XZ atlas
// (the stand-in for the renderer's splat / gather step of Fig. 2); the
// per-photon arithmetic is in deposit_core.cuh.
#include "deposit_core.cuh"

using namespace pvk;

namespace {

__global__ void __launch_bounds__(256) k_deposit(uint32_t n, uint32_t B, const uint32_t* info, const float4* pa,
                                                 const float4* pb, pv_atlas at) {
  const AtlasMap am = atlas_map(at);
  // whole warps loop, so that the photons of each round's 32 paths are dealt out over the lanes
  for (uint32_t b = blockIdx.x * blockDim.x; b < n; b += gridDim.x * blockDim.x) {
    const uint32_t p = b + threadIdx.x;
    deposit_warp(am, n, B, info, pa, pb, p < n ? p : 0xFFFFFFFFu);
  }
}

}  // namespace

namespace pvh {

int check_atlas(const pv_atlas* a) {
  if (!a || !a->data || a->width == 0 || a->height == 0) return PV_ERR_ARG;
  if (!(a->x1 > a->x0) || !(a->z1 > a->z0) || a->scale_log2 < 0 || a->scale_log2 > 62) return PV_ERR_ARG;
  return PV_OK;
}

void launch_deposit(pv_scene* s, const pv_paths* p, const pv_atlas* a, cudaStream_t st) {
  const uint32_t n = p->n;
  if (!n) return;
  const uint32_t blocks = (uint32_t)s->num_sms * 8u;
  k_deposit<<<blocks, 256, 0, st>>>(n, s->B, p->info, reinterpret_cast<const float4*>(p->pa),
                                    reinterpret_cast<const float4*>(p->pb), *a);
}

}  // namespace pvh

extern "C" int pv_deposit(pv_scene* s, const pv_paths* paths, const pv_atlas* atlas, void* stream) {
  int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if ((rc = pvh::check_atlas(atlas)) != PV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (cudaMemsetAsync(atlas->data, 0, (size_t)atlas->width * atlas->height * 3 * sizeof(uint64_t), st) != cudaSuccess)
    return PV_ERR_CUDA;
  pvh::launch_deposit(s, paths, atlas, st);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
