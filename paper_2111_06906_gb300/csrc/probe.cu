// FP32 issue-rate probe: the denominator of the traversal kernels' ALU
// roofline, measured on the device that runs them instead of derived from a
// data sheet.  Every thread runs kChains independent fused multiply-add
// chains, so the FMA pipe, not the dependency latency, bounds the kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pv.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;     // 128 FMAs per loop iteration: the loop's own two instructions cost 1.5 %
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(uint32_t iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
  const float m = 0.99999988f, c = 1.1920929e-07f;
#pragma unroll 1
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == -1.0f) sink[blockIdx.x] = s;     // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" int pv_fma_probe(uint32_t blocks, uint32_t iters, float* d_sink, uint64_t* fmas, void* stream) {
  if (!blocks || !iters || !d_sink || !fmas) return PV_ERR_ARG;
  *fmas = (uint64_t)blocks * kProbeThreads * iters * kUnroll * kChains;
  k_fma_probe<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, d_sink);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
