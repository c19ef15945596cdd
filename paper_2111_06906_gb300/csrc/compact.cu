// Compaction entry points (the kernel body is in compact_core.cuh).
#include <mutex>

#include "compact_core.cuh"

using namespace pvk;

namespace {

// ``failed``: null, or a word cleared before the launch that a tile giving
// up on its look-back sets (the count then reads kCompactFailed).
__global__ void __launch_bounds__(pvh::kCompactThreads) k_compact(const uint32_t* info, uint32_t n, uint32_t* list,
                                                                    uint32_t* count, unsigned long long* tiles,
                                                                    uint32_t* ticket, uint32_t n_tiles, int* status,
                                                                    uint32_t* stat_listed, uint32_t* failed) {
  __shared__ CompactSmem sm;
  if (threadIdx.x == 0) sm.tile = atomicAdd(ticket, 1u);
  __syncthreads();
  compact_tile(info, n, list, count, tiles, sm.tile, n_tiles, status, stat_listed, sm, failed);
}

}  // namespace

namespace pvh {

void launch_compact(pv_scene* s, const uint32_t* info, uint32_t n, uint32_t* list, uint32_t* count,
                    uint32_t* stats_listed, cudaStream_t st) {
  if (n == 0) {
    cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
    return;
  }
  const uint32_t n_tiles = (n + kTile - 1) / kTile;
  cudaMemsetAsync(s->ws_tiles, 0, (size_t)n_tiles * sizeof(uint64_t), st);
  cudaMemsetAsync(s->ws_ctr + CTR_TILE, 0, sizeof(uint32_t), st);
  k_compact<<<n_tiles, kCompactThreads, 0, st>>>(info, n, list, count, reinterpret_cast<unsigned long long*>(s->ws_tiles),
                                                 s->ws_ctr + CTR_TILE, n_tiles, s->status, stats_listed, nullptr);
}

}  // namespace pvh

extern "C" int pv_compact_replace(pv_scene* s, const pv_paths* paths, uint32_t* d_list, uint32_t* d_count, void* stream) {
  const int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!d_list || !d_count) return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  pvh::launch_compact(s, paths->info, paths->n, d_list, d_count, nullptr, st);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Allocation-free compaction.  Some callers must not allocate device memory
// once they are running: a renderer that reserves its whole memory budget at
// start-up, or one whose allocations belong to another framework's pool, and
// any frame loop that cannot afford the device-wide synchronisation a
// cudaMalloc may cause.  Such callers may also hold no pv_scene.  For them
// the look-back tile states live in this fixed array, which every GPU that
// loads the library keeps until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kStaticTiles = (PV_STATIC_COMPACT_MAX_PATHS + pvh::kTile - 1) / pvh::kTile;

// tile states [0, kStaticTiles), then the last word: the tile ticket (low 32
// bits) and the give-up flag (high 32 bits)
static __device__ __align__(256) unsigned long long g_compact_scratch[kStaticTiles + 1];

std::mutex g_scratch_mutex;
void* g_scratch_ptr[64] = {};

// Device address of the scratch array for the current device, looked up once
// per device (host code must not use the array's name as a device pointer).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PV_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_compact_scratch) != cudaSuccess || !p) return PV_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PV_OK;
}

}  // namespace

extern "C" int pv_compact_replace_static(const uint32_t* d_info, uint32_t n, uint32_t* d_list, uint32_t* d_count,
                                         void* stream) {
  if (!d_count || (n && (!d_info || !d_list))) return PV_ERR_ARG;
  if (n > PV_STATIC_COMPACT_MAX_PATHS) return PV_ERR_LIMIT;
  void* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != PV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) return cudaMemsetAsync(d_count, 0, sizeof(uint32_t), st) == cudaSuccess ? PV_OK : PV_ERR_CUDA;
  const uint32_t n_tiles = (n + pvh::kTile - 1) / pvh::kTile;
  unsigned long long* tiles = static_cast<unsigned long long*>(base);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(tiles + kStaticTiles);
  uint32_t* failed = ticket + 1;
  // the previous call's tile states, ticket and flag are still in the array: clear them
  if (cudaMemsetAsync(tiles, 0, (size_t)n_tiles * sizeof(unsigned long long), st) != cudaSuccess ||
      cudaMemsetAsync(ticket, 0, 2 * sizeof(uint32_t), st) != cudaSuccess)
    return PV_ERR_CUDA;
  k_compact<<<n_tiles, pvh::kCompactThreads, 0, st>>>(d_info, n, d_list, d_count, tiles, ticket, n_tiles, nullptr,
                                                      nullptr, failed);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
