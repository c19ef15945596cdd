// Compaction of the paths marked for replacement into an ascending id list:
// the "pruned paths array" pattern of Sec. 5.2 (process only the marked
// paths, packed into as few blocks as possible).  One pass over the info
// words: per-thread bit masks, warp and block scans, and a decoupled
// look-back across tiles (Merrill & Garland, "Single-pass parallel prefix
// scan with decoupled look-back", 2016).  Shared by compact.cu (one array)
// and batch.cu (one array per scene, tiles of all scenes in one launch).
#pragma once
#include "pv_scene.h"

namespace pvk {

constexpr unsigned long long kFlagAggregate = 1ull << 32;
constexpr unsigned long long kFlagPrefix = 2ull << 32;
constexpr unsigned long long kFlagMask = 3ull << 32;
constexpr uint32_t kSpinCap = 1u << 24;

struct CompactSmem {
  uint32_t tile, prefix;
  uint32_t warp[pvh::kCompactThreads / 32];
};

// One tile of kTile paths (tile index local to this array of info words),
// called by every thread of a kCompactThreads block.  Tiles of one array must
// take their indices in increasing order of start (an atomic ticket), so
// every tile a look-back waits on has already started.
//
// A look-back that waits longer than kSpinCap for a predecessor gives up and
// publishes a partial prefix.  It records PV_ERR_ITER_CAP in ``status``, and
// when ``failed`` is given it sets that word before publishing.  The last tile
// reads ``failed`` after its own look-back (every tile above a stuck one can
// only complete through a tile that gave up, whose flag it then sees) and
// writes kCompactFailed as the count instead of a wrong one.
constexpr uint32_t kCompactFailed = 0xFFFFFFFFu;

__device__ __forceinline__ void compact_tile(const uint32_t* info, uint32_t n, uint32_t* list, uint32_t* count,
                                             unsigned long long* tiles, uint32_t tile, uint32_t n_tiles, int* status,
                                             uint32_t* stat_listed, CompactSmem& sm, uint32_t* failed = nullptr) {
  constexpr int kWarps = pvh::kCompactThreads / 32;
  uint32_t& s_prefix = sm.prefix;
  uint32_t* const s_warp = sm.warp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
            if (failed) {
              atomicExch(failed, 1u);
              __threadfence();                     // the flag is visible before the partial prefix
            }
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
    bool gave_up = false;
    if (failed) {
      __threadfence();
      gave_up = atomicAdd(failed, 0u) != 0u;
    }
    *count = gave_up ? kCompactFailed : s_prefix + tile_total;
    if (stat_listed && !gave_up) atomicAdd(stat_listed, s_prefix + tile_total);
  }
}

}  // namespace pvk
