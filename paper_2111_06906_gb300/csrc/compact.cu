// Compaction of the paths marked for replacement into an ascending id list:
// the "pruned paths array" pattern of Sec. 5.2 (process only the marked
// paths, packed into as few blocks as possible).  One pass over the info
// words: per-thread bit masks, warp and block scans, and a decoupled
// look-back across tiles (Merrill & Garland, "Single-pass parallel prefix
// scan with decoupled look-back", 2016).  Tiles take their index from an
// atomic ticket, so every tile a look-back waits on has already started.
#include <mutex>

#include "pv_scene.h"

using namespace pvk;

namespace {

constexpr unsigned long long kFlagAggregate = 1ull << 32;
constexpr unsigned long long kFlagPrefix = 2ull << 32;
constexpr unsigned long long kFlagMask = 3ull << 32;
constexpr uint32_t kSpinCap = 1u << 24;

__global__ void __launch_bounds__(pvh::kCompactThreads) k_compact(const uint32_t* info, uint32_t n, uint32_t* list,
                                                                    uint32_t* count, unsigned long long* tiles,
                                                                    uint32_t* ticket, uint32_t n_tiles, int* status,
                                                                    uint32_t* stat_listed) {
  constexpr int kWarps = pvh::kCompactThreads / 32;
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t base = tile * pvh::kTile + threadIdx.x * pvh::kCompactItems;
  uint32_t flags = 0;
  if (base + pvh::kCompactItems <= n && (reinterpret_cast<uintptr_t>(info) & 15u) == 0) {
    const uint4* q = reinterpret_cast<const uint4*>(info + base);
#pragma unroll
    for (int j = 0; j < pvh::kCompactItems / 4; ++j) {
      const uint4 v = __ldg(q + j);
      flags |= ((v.x >> 30) & 1u) << (4 * j) | ((v.y >> 30) & 1u) << (4 * j + 1) | ((v.z >> 30) & 1u) << (4 * j + 2) |
               ((v.w >> 30) & 1u) << (4 * j + 3);
    }
  } else {
    for (int j = 0; j < pvh::kCompactItems; ++j) {
      const uint32_t i = base + j;
      if (i < n && (__ldg(info + i) & PV_INFO_REPLACE)) flags |= 1u << j;
    }
  }
  const uint32_t cnt = __popc(flags);
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < kWarps ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < kWarps) s_warp[lane] = v;
  }
  __syncthreads();
  const uint32_t tile_total = s_warp[kWarps - 1];
  const uint32_t in_tile = (warp ? s_warp[warp - 1] : 0u) + incl - cnt;
  if (threadIdx.x == 0) {
    uint32_t prefix = 0;
    if (tile == 0) {
      atomicExch(tiles, kFlagPrefix | tile_total);
    } else {
      atomicExch(tiles + tile, kFlagAggregate | tile_total);
      int j = (int)tile - 1;
      uint32_t spins = 0;
      while (j >= 0) {
        const unsigned long long st = *reinterpret_cast<volatile unsigned long long*>(tiles + j);
        const unsigned long long f = st & kFlagMask;
        if (f == 0ull) {
          if (++spins > kSpinCap) {                // predecessor never published: give up, flag it
            record_error(status, PV_ERR_ITER_CAP);
            break;
          }
          continue;
        }
        prefix += (uint32_t)st;
        if (f == kFlagPrefix) break;
        --j;
      }
      atomicExch(tiles + tile, kFlagPrefix | (unsigned long long)(prefix + tile_total));
    }
    s_prefix = prefix;
  }
  __syncthreads();
  uint32_t pos = s_prefix + in_tile;
  for (int j = 0; j < pvh::kCompactItems; ++j)
    if ((flags >> j) & 1u) list[pos++] = base + j;
  if (tile == n_tiles - 1 && threadIdx.x == 0) {
    *count = s_prefix + tile_total;
    if (stat_listed) atomicAdd(stat_listed, s_prefix + tile_total);
  }
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
                                                 s->ws_ctr + CTR_TILE, n_tiles, s->status, stats_listed);
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

// tile states [0, kStaticTiles), then the tile ticket (low 32 bits of the last word)
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
  // the previous call's tile states and ticket are still in the array: clear them
  if (cudaMemsetAsync(tiles, 0, (size_t)n_tiles * sizeof(unsigned long long), st) != cudaSuccess ||
      cudaMemsetAsync(ticket, 0, sizeof(uint32_t), st) != cudaSuccess)
    return PV_ERR_CUDA;
  k_compact<<<n_tiles, pvh::kCompactThreads, 0, st>>>(d_info, n, d_list, d_count, tiles, ticket, n_tiles, nullptr,
                                                      nullptr);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
