// Batched verification and re-trace of many scenes (include/pv_batch.h).
//
// One launch per step over all scenes: pose update (object transforms, leaf
// refit, wide-node refit, top level), verify (Sec. 3.1 + 3.2, tiles of every
// scene in one grid, thread- or warp-per-path), the Alg. 1 continuation and
// the re-trace (persistent kernels whose work lists are the concatenation of
// the scenes' lists, so small scenes share the GPU with large ones), and the
// compaction (tiles of every scene, one look-back chain per scene) when the
// caller asked for lists; without lists verify appends the paths it marks to
// each scene's work list directly and Alg. 1 runs inside the re-trace.  Per-scene
// state lives in device tables; the per-frame part (light poses, transforms,
// moved bits, frame number) is copied from pinned staging by the first node
// of a CUDA graph that is captured once and replayed every frame.
#include <algorithm>
#include <array>
#include <cstring>
#include <vector>

#include "compact_core.cuh"
#include "pv_batch.h"
#include "trace_core.cuh"
#include "update_core.cuh"
#include "verify_core.cuh"

using namespace pvk;

namespace {

constexpr uint32_t kBatchMax = PV_BATCH_MAX_SCENES;
constexpr int kRing = 3;                      // pinned staging slots of the per-frame data
constexpr uint32_t kGuard = 1u << 30;         // bound of the persistent loops

// Minimum resident blocks per SM of the batched flat-mapping verify (k_b_verify<.., 2>).
#ifndef PV_BATCH_FLAT_MIN_BLOCKS
#define PV_BATCH_FLAT_MIN_BLOCKS 5
#endif

// Minimum resident blocks per SM of the batched re-trace with lists (k_b_trace):
// 7 fits in 72 registers without spills (8 spills).
#ifndef PV_BATCH_TRACE_MIN_BLOCKS
#define PV_BATCH_TRACE_MIN_BLOCKS 7
#endif

// Static per-scene record (device table).
struct BScene {
  SceneView sv;                               // sv.moved is taken from the frame record
  VerifyArgs V;
  ContArgs C;
  TraceArgs T;                                // T.frame is taken from the frame record
  // pose update
  const float* d_local;
  const uint32_t* d_tri_prim;
  Tri* dtris;
  DynObj* objs;
  MovedGroups* groups;
  float* xf_old;
  float* xf_new;
  const Node* bnodes;                         // all binary nodes (the wide refit sources index them)
  Node* dnodes;                               // the dynamic tree's binary nodes (local indices)
  const uint32_t* node_parent;
  const uint32_t* leaf_parent;
  uint32_t* fit_flags;
  uint32_t n_dyn_tris, n_dyn;
  uint32_t refit_blocks;                      // k_b_refit_wide blocks of this scene (0: k_b_frame_top does its top)
  uint32_t* refit_done;                       // of them, finished this frame (reset by the last)
  const uint8_t* tri_slot;
  const uint32_t* t_link;
  const uint32_t* w_link;
  const uint8_t* w_nch;
  uint32_t* w_arrive;
  int* obox;
  const int* wsrc_dyn;
  const uint32_t* wcount_dyn;
  WNode* wnodes_dyn;
  WNode* wnodes;
  const Tri* tris;
  int top_off, s_wroot;
  int* root;
  // compaction
  unsigned long long* tiles;
  uint32_t n_tiles;
  uint32_t* list;
  uint32_t* count;
  uint32_t* stat_listed;
  uint32_t* ctr;                              // the scene's 16 work counters
};

// Per-frame per-scene record (copied from pinned staging each frame).
struct BFrame {
  FrameLights L;
  float xf[kMaxDyn][12];
  uint64_t moved;
  uint32_t frame;
  uint32_t pad;
};

struct BCounters {
  uint32_t cont, trace, compact, pad;
};

__device__ __forceinline__ void copy_words(void* dst, const void* src, uint32_t bytes, uint32_t t, uint32_t nt) {
  const uint32_t* a = static_cast<const uint32_t*>(src);
  uint32_t* b = static_cast<uint32_t*>(dst);
  for (uint32_t i = t; i < bytes / 4; i += nt) b[i] = a[i];
}

// Scene of work item g given the exclusive prefix pre[0..n] of the per-scene counts.
__device__ __forceinline__ uint32_t scene_of(const uint32_t* pre, uint32_t n, uint32_t g) {
  uint32_t lo = 0, hi = n;                    // pre[lo] <= g < pre[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Per-frame zeroing of every scene's counters and tile states.
__global__ void k_b_prologue(const BScene* S, const BFrame* F, BCounters* bc) {
  const uint32_t s = blockIdx.x;
  const BScene& B = S[s];
  if (s == 0 && threadIdx.x == 0) {
    bc->cont = 0;
    bc->trace = 0;
    bc->compact = 0;
  }
  if (threadIdx.x < 16) B.ctr[threadIdx.x] = 0u;
  for (uint32_t i = threadIdx.x; i < B.n_tiles; i += blockDim.x) B.tiles[i] = 0ull;
}

// ---------------------------------------------------------------- distribution maps (Sec. 3.1)
// The steps of dm.cu for one scene of the batch.  They read the frame's
// light poses, moved lights and frame number from the scene's frame record,
// so a captured frame stays right from one replay to the next; a light whose
// map did not move this frame is left alone, as dm.cu leaves it.

// DM_C of the moved lights with a map, cleared before verification counts it.
__global__ void k_b_dm_clear(const BFrame* F, uint32_t sc) {
  const FrameLights& L = F[sc].L;
  for (uint32_t l = 0; l < L.n; ++l) {
    if (!dm_moved(L, l)) continue;
    const DmLight& D = L.dm[l];
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < D.cells; c += gridDim.x * blockDim.x) D.dmc[c] = 0u;
  }
}

// Pass 1 of the prune (dm_prune_path, with the scene's seed and the frame's number); flag[p] = 1 when pruned.
__global__ void __launch_bounds__(256) k_b_dm_prune(const BScene* S, const BFrame* F, uint32_t sc, uint32_t* flag) {
  __shared__ uint32_t s_red[32];
  const BScene& B = S[sc];
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t pruned = 0;
  if (p < B.V.n) {
    pruned = dm_prune_path(F[sc].L, p, B.V.info, B.T.seed, F[sc].frame);
    flag[p] = pruned;
  }
  uint32_t* const ctr[1] = {B.V.stats ? &B.V.stats->n_pruned : nullptr};
  const uint32_t val[1] = {pruned};
  block_add_n<1>(ctr, val, s_red);
}

// Pass 2 (dm_commit_path): flag[p] becomes the free-path flag for the compaction.
__global__ void __launch_bounds__(256) k_b_dm_commit(const BScene* S, const BFrame* F, uint32_t sc, uint32_t* flag,
                                                     uint32_t* free_count) {
  const BScene& B = S[sc];
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B.V.n) return;
  flag[p] = dm_commit_path(F[sc].L, p, B.V.info, flag[p], free_count);
}

__global__ void k_b_dm_deficit(const BFrame* F, uint32_t sc, uint32_t l, uint32_t* def) {
  const FrameLights& L = F[sc].L;
  if (!dm_moved(L, l)) return;
  const DmLight& D = L.dm[l];
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= D.cells; c += gridDim.x * blockDim.x)
    def[c] = dm_deficit(D, c);
}

// Fill (dm_fill_path) for the free paths of light l, listed after those of the lights before it.
__global__ void __launch_bounds__(256) k_b_dm_fill(const BScene* S, const BFrame* F, uint32_t sc, uint32_t l,
                                                   const uint32_t* free_list, const uint32_t* free_count,
                                                   const uint32_t* pre) {
  __shared__ uint32_t s_red[32];
  const FrameLights& L = F[sc].L;
  if (!dm_moved(L, l)) return;                 // the same for every thread of the block
  const BScene& B = S[sc];
  const DmLight& D = L.dm[l];
  const uint32_t Fc = free_count[l];
  uint32_t off = 0;
  for (uint32_t k = 0; k < l; ++k) off += free_count[k];
  uint32_t filled = 0;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < Fc; j += gridDim.x * blockDim.x) {
    dm_fill_path(D, l, free_list[off + j], j, Fc, pre, B.V.info);
    ++filled;
  }
  uint32_t* const ctr[1] = {B.V.stats ? &B.V.stats->n_filled : nullptr};
  const uint32_t val[1] = {filled};
  block_add_n<1>(ctr, val, s_red);
}

// ---------------------------------------------------------------- pose update
// Per 256-triangle chunk of one scene (tab: scene, first triangle): the
// moved objects' triangles to the new pose and the direct wide refit.
// The last block of a scene to finish then does the scene's pose
// bookkeeping, top level and moved-object groups (k_b_frame_top's work).
__global__ void __launch_bounds__(256) k_b_refit_wide(const BScene* S, const BFrame* F, const uint32_t* tab) {
  __shared__ bool s_last;
  const uint32_t sc = tab[2 * blockIdx.x], i = tab[2 * blockIdx.x + 1] + threadIdx.x;
  const BScene& B = S[sc];
  const uint64_t moved = F[sc].moved;
  const uint32_t s = i < B.n_dyn_tris ? B.tri_slot[i] : 0u;
  const bool mv = i < B.n_dyn_tris && ((moved >> s) & 1ull);
  RefitArgs R;
  R.local = B.d_local;
  R.prim = B.d_tri_prim;
  R.tri_slot = B.tri_slot;
  R.dtris = B.dtris;
  R.n = B.n_dyn_tris;
  R.t_link = B.t_link;
  R.w_link = B.w_link;
  R.w_nch = B.w_nch;
  R.w_arrive = B.w_arrive;
  R.wdyn = B.wnodes_dyn;
  R.obox = B.obox;
  refit_tri(F[sc].xf[mv ? s : 0], mv, s, R, i);
  __threadfence();                             // this block's triangles, boxes and object-box atomics
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(B.refit_done, 1u) == B.refit_blocks - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();                             // the scene's other blocks' writes are visible from here
  if (threadIdx.x == 0) *B.refit_done = 0u;
  pose_bookkeeping(F[sc].xf, moved, B.n_dyn, B.objs, B.xf_old, B.xf_new, B.obox);
  if (!moved) return;
  build_top_and_groups(B.wnodes, B.tris, B.top_off, B.s_wroot, B.objs, (int)B.n_dyn, B.root, moved, B.groups);
}

// One block of 32 threads per scene: pose bookkeeping of every slot, then
// (when objects moved) the top level and the moved objects' groups.
__global__ void k_b_frame_top(const BScene* S, const BFrame* F) {
  const uint32_t s = blockIdx.x;
  const BScene& B = S[s];
  if (B.refit_blocks) return;                  // the scene's last refit block did it
  if (B.objs) pose_bookkeeping(F[s].xf, F[s].moved, B.n_dyn, B.objs, B.xf_old, B.xf_new, B.obox);
  if (!F[s].moved) return;
  build_top_and_groups(B.wnodes, B.tris, B.top_off, B.s_wroot, B.objs, (int)B.n_dyn, B.root, F[s].moved,
                       B.groups);
}

// ---------------------------------------------------------------- verify
// Resident blocks loop over the tile table (tab: scene, tile), in steps of
// the grid.  Entries of one scene are consecutive in the table, so a block
// stages a scene's view, lights, arguments and moved-object boxes in shared
// memory when its next entry belongs to another scene, and adds that scene's
// counters when it leaves it.
// Box-only variants are held to 5 resident blocks of 256 threads (51 registers), as the single-scene kernel.
template <bool kPointVis, bool kExact, int kMap>
__global__ void __launch_bounds__(256, (kPointVis || kExact) ? 2 : (kMap == 2 ? PV_BATCH_FLAT_MIN_BLOCKS : 5)) k_b_verify(const BScene* S, const BFrame* F,
                                                                                  const uint32_t* tab, uint32_t n_entries) {
  __shared__ VerifySmem sm;
  __shared__ SceneView s_sv;
  __shared__ FrameLights s_L;
  __shared__ VerifyArgs s_V;
  uint32_t cur = 0xFFFFFFFFu;
  int root = 0;
  Work wk;
  VerifyCount vc;
  for (uint32_t e = blockIdx.x; e < n_entries; e += gridDim.x) {
    const uint32_t sc = tab[2 * e], tile = tab[2 * e + 1];
    if (sc != cur) {
      if (cur != 0xFFFFFFFFu) {
        verify_counts_flush(s_V, vc, wk, kPointVis || kExact, sm);
        vc = VerifyCount();
        wk = Work();
      }
      __syncthreads();                         // the previous scene's shared state is no longer read
      copy_words(&s_sv, &S[sc].sv, sizeof(SceneView), threadIdx.x, blockDim.x);
      copy_words(&s_L, &F[sc].L, sizeof(FrameLights), threadIdx.x, blockDim.x);
      copy_words(&s_V, &S[sc].V, sizeof(VerifyArgs), threadIdx.x, blockDim.x);
      __syncthreads();
      if (threadIdx.x == 0) s_sv.moved = F[sc].moved;
      __syncthreads();
      verify_smem_init(s_sv, sm);
      root = *s_sv.root;
      cur = sc;
    }
    verify_tile<kPointVis, kExact, kMap>(s_sv, s_L, s_V, root, tile * blockDim.x + threadIdx.x, sm, vc, wk);
  }
  if (cur != 0xFFFFFFFFu) verify_counts_flush(s_V, vc, wk, kPointVis || kExact, sm);
}

// Shared-memory layout of the persistent kernels: per scene its view, its
// arguments, root, and counters; then the prefix of the work counts.
template <class Args>
struct PersistLayout {
  uint32_t sv, args, root, cnt, cnt64, pre, bytes;
  __host__ __device__ PersistLayout(uint32_t n) {
    auto up = [](uint32_t x) { return (x + 15u) & ~15u; };
    sv = 0;
    args = up(sv + n * (uint32_t)sizeof(SceneView));
    root = up(args + n * (uint32_t)sizeof(Args));
    cnt = up(root + n * 4u);
    cnt64 = up(cnt + n * 4u * 4u);
    pre = up(cnt64 + n * 2u * 8u);
    bytes = up(pre + (n + 1u) * 4u);
  }
};

// ---------------------------------------------------------------- Alg. 1 continuation
template <int S>
__global__ void __launch_bounds__(128) k_b_continue(const BScene* B, const BFrame* F, uint32_t n_scenes, BCounters* bc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PersistLayout<ContArgs> lay(n_scenes);
  SceneView* s_sv = reinterpret_cast<SceneView*>(smem + lay.sv);
  ContArgs* s_C = reinterpret_cast<ContArgs*>(smem + lay.args);
  int* s_root = reinterpret_cast<int*>(smem + lay.root);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + lay.cnt);
  unsigned long long* s_cnt64 = reinterpret_cast<unsigned long long*>(smem + lay.cnt64);
  uint32_t* s_pre = reinterpret_cast<uint32_t*>(smem + lay.pre);
  for (uint32_t s = 0; s < n_scenes; ++s) {
    copy_words(s_sv + s, &B[s].sv, sizeof(SceneView), threadIdx.x, blockDim.x);
    copy_words(s_C + s, &B[s].C, sizeof(ContArgs), threadIdx.x, blockDim.x);
  }
  for (uint32_t i = threadIdx.x; i < 4 * n_scenes; i += blockDim.x) s_cnt[i] = 0u;
  for (uint32_t i = threadIdx.x; i < 2 * n_scenes; i += blockDim.x) s_cnt64[i] = 0ull;
  __syncthreads();
  if (threadIdx.x < n_scenes) {
    s_sv[threadIdx.x].moved = F[threadIdx.x].moved;
    s_root[threadIdx.x] = *B[threadIdx.x].sv.root;
  }
  if (threadIdx.x == 0) {
    s_pre[0] = 0;
    for (uint32_t s = 0; s < n_scenes; ++s) s_pre[s + 1] = s_pre[s] + min(*B[s].C.count, B[s].C.n);
  }
  __syncthreads();
  const uint32_t total = s_pre[n_scenes];
  const int lane = threadIdx.x & 31;
  for (uint32_t guard = 0; guard < kGuard; ++guard) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&bc->cont, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= total) break;
    const uint32_t i = base + lane;
    if (i < total) {
      const uint32_t sc = scene_of(s_pre, n_scenes, i);
      const ContArgs& A = s_C[sc];
      ContCounters cc;
      Work wk;
      continue_path<S>(s_sv[sc], s_root[sc], A, A.list[i - s_pre[sc]], cc, wk);
      if (cc.rays) atomicAdd(s_cnt + 4 * sc + 0, cc.rays);
      if (cc.tail) atomicAdd(s_cnt + 4 * sc + 1, cc.tail);
      if (cc.upd) atomicAdd(s_cnt + 4 * sc + 2, cc.upd);
      if (cc.trunc) atomicAdd(s_cnt + 4 * sc + 3, cc.trunc);
      if (wk.nodes) atomicAdd(s_cnt64 + 2 * sc + 0, (unsigned long long)wk.nodes);
      if (wk.tris) atomicAdd(s_cnt64 + 2 * sc + 1, (unsigned long long)wk.tris);
    }
    __syncwarp();
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < n_scenes; s += blockDim.x) {
    pv_frame_stats* st = s_C[s].stats;
    if (!st) continue;
    if (s_cnt[4 * s + 0]) atomicAdd(&st->cont_rays, s_cnt[4 * s + 0]);
    if (s_cnt[4 * s + 1]) atomicAdd(&st->n_tail, s_cnt[4 * s + 1]);
    if (s_cnt[4 * s + 2]) atomicAdd(&st->n_updated, s_cnt[4 * s + 2]);
    if (s_cnt[4 * s + 3]) atomicAdd(&st->n_truncated, s_cnt[4 * s + 3]);
    if (s_cnt64[2 * s + 0]) atomicAdd((unsigned long long*)&st->node_visits, s_cnt64[2 * s + 0]);
    if (s_cnt64[2 * s + 1]) atomicAdd((unsigned long long*)&st->tri_tests, s_cnt64[2 * s + 1]);
  }
}

// ---------------------------------------------------------------- compaction
// Tiles take a global ticket; tile t is (scene, local tile) = tab[t], so the
// tiles of one scene start in increasing order and its look-back completes.
__global__ void __launch_bounds__(pvh::kCompactThreads) k_b_compact(const BScene* B, const uint32_t* tab, BCounters* bc) {
  __shared__ CompactSmem sm;
  if (threadIdx.x == 0) sm.tile = atomicAdd(&bc->compact, 1u);
  __syncthreads();
  const uint32_t t = sm.tile;
  const uint32_t sc = tab[2 * t], local = tab[2 * t + 1];
  const BScene& b = B[sc];
  compact_tile(b.V.info, b.V.n, b.list, b.count, b.tiles, local, b.n_tiles, b.sv.status, b.stat_listed, sm);
}

// ---------------------------------------------------------------- re-trace
// The persistent re-trace of trace.cu over the concatenated lists of all
// scenes: each lane carries the scene of its current path.
template <int kSteps, int S>
__global__ void __launch_bounds__(pvh::kTraceThreads, PV_BATCH_TRACE_MIN_BLOCKS) k_b_trace(const BScene* B, const BFrame* F, uint32_t n_scenes,
                                                                  BCounters* bc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PersistLayout<TraceArgs> lay(n_scenes);
  SceneView* s_sv = reinterpret_cast<SceneView*>(smem + lay.sv);
  TraceArgs* s_T = reinterpret_cast<TraceArgs*>(smem + lay.args);
  int* s_root = reinterpret_cast<int*>(smem + lay.root);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + lay.cnt);
  unsigned long long* s_cnt64 = reinterpret_cast<unsigned long long*>(smem + lay.cnt64);
  uint32_t* s_pre = reinterpret_cast<uint32_t*>(smem + lay.pre);
  for (uint32_t s = 0; s < n_scenes; ++s) {
    copy_words(s_sv + s, &B[s].sv, sizeof(SceneView), threadIdx.x, blockDim.x);
    copy_words(s_T + s, &B[s].T, sizeof(TraceArgs), threadIdx.x, blockDim.x);
  }
  for (uint32_t i = threadIdx.x; i < 4 * n_scenes; i += blockDim.x) s_cnt[i] = 0u;
  for (uint32_t i = threadIdx.x; i < 2 * n_scenes; i += blockDim.x) s_cnt64[i] = 0ull;
  __syncthreads();
  if (threadIdx.x < n_scenes) {
    s_sv[threadIdx.x].moved = F[threadIdx.x].moved;
    s_T[threadIdx.x].frame = F[threadIdx.x].frame;
    s_root[threadIdx.x] = *B[threadIdx.x].sv.root;
  }
  if (threadIdx.x == 0) {
    s_pre[0] = 0;
    for (uint32_t s = 0; s < n_scenes; ++s) s_pre[s + 1] = s_pre[s] + min(*B[s].T.count, B[s].T.n);
  }
  __syncthreads();
  const uint32_t total = s_pre[n_scenes];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  Work wk;
  PathState st;
  Ray r;
  Trav t;
  TStack<S> stk;
  uint32_t sc = 0, c_rays = 0, c_photons = 0;
  bool has_ray = false, exhausted = false;
  auto flush = [&]() {                         // the finished path's counters to its scene
    if (c_rays) atomicAdd(s_cnt + 4 * sc + 0, c_rays);
    if (c_photons) atomicAdd(s_cnt + 4 * sc + 1, c_photons);
    if (wk.nodes) atomicAdd(s_cnt64 + 2 * sc + 0, (unsigned long long)wk.nodes);
    if (wk.tris) atomicAdd(s_cnt64 + 2 * sc + 1, (unsigned long long)wk.tris);
    c_rays = c_photons = 0;
    wk.nodes = wk.tris = 0;
  };
  for (uint32_t guard = 0; guard < kGuard; ++guard) {
    const bool need = !has_ray && !exhausted;
    const unsigned nm = __ballot_sync(0xffffffffu, need);
    if (nm) {
      const int leader = __ffs(nm) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&bc->trace, (uint32_t)__popc(nm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const uint32_t idx = base + __popc(nm & lt);
        if (idx < total) {
          sc = scene_of(s_pre, n_scenes, idx);
          if (init_path(s_sv[sc], F[sc].L, s_T[sc], idx - s_pre[sc], st, r)) {
            trav_begin(t, s_root[sc]);
            has_ray = true;
          } else {
            flush();
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted && !has_ray)) break;
    const SceneView& sv = s_sv[sc];
    const TraceArgs& A = s_T[sc];
    const bool done = step_warp<kSteps, S>(sv, r, t, stk, st.excl, wk, !has_ray);
    if (!has_ray || !done) continue;
    ++c_rays;
    if (trace_hit(sv, A, st, r, t, c_photons)) {
      trav_begin(t, s_root[sc]);
    } else {
      has_ray = false;
      flush();
    }
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < n_scenes; s += blockDim.x) {
    pv_frame_stats* stt = s_T[s].stats;
    if (!stt) continue;
    if (s_cnt[4 * s + 0]) atomicAdd(&stt->trace_rays, s_cnt[4 * s + 0]);
    if (s_cnt[4 * s + 1]) atomicAdd(&stt->photons_written, s_cnt[4 * s + 1]);
    if (s_cnt64[2 * s + 0]) atomicAdd((unsigned long long*)&stt->node_visits, s_cnt64[2 * s + 0]);
    if (s_cnt64[2 * s + 1]) atomicAdd((unsigned long long*)&stt->tri_tests, s_cnt64[2 * s + 1]);
  }
}

// ---------------------------------------------------------------- Alg. 1 fused with the re-trace
// Shared-memory layout of the fused kernel: per scene its view, both
// argument records, root and counters; then the prefixes of the
// continuation and re-trace counts.
struct FusedLayout {
  uint32_t sv, cargs, targs, root, cnt, cnt64, cpre, pre, bytes;
  __host__ __device__ FusedLayout(uint32_t n) {
    auto up = [](uint32_t x) { return (x + 15u) & ~15u; };
    sv = 0;
    cargs = up(sv + n * (uint32_t)sizeof(SceneView));
    targs = up(cargs + n * (uint32_t)sizeof(ContArgs));
    root = up(targs + n * (uint32_t)sizeof(TraceArgs));
    cnt = up(root + n * 4u);
    cnt64 = up(cnt + n * 6u * 4u);
    cpre = up(cnt64 + n * 2u * 8u);
    pre = up(cpre + (n + 1u) * 4u);
    bytes = up(pre + (n + 1u) * 4u);
  }
};

// minimum resident blocks per SM of the fused kernel (a compile-time tuning knob)
#ifndef PV_BATCH_CT_MIN_BLOCKS
#define PV_BATCH_CT_MIN_BLOCKS 7
#endif

// k_cont_trace of trace.cu over all scenes: the work items are every
// scene's continuation list, then every scene's re-trace list; each lane
// carries the scene of its current path.  Per-path arithmetic is that of
// k_b_continue followed by k_b_trace.
template <int kSteps, int S>
__global__ void __launch_bounds__(pvh::kTraceThreads, PV_BATCH_CT_MIN_BLOCKS) k_b_cont_trace(const BScene* B, const BFrame* F,
                                                                       uint32_t n_scenes, BCounters* bc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const FusedLayout lay(n_scenes);
  SceneView* s_sv = reinterpret_cast<SceneView*>(smem + lay.sv);
  ContArgs* s_C = reinterpret_cast<ContArgs*>(smem + lay.cargs);
  TraceArgs* s_T = reinterpret_cast<TraceArgs*>(smem + lay.targs);
  int* s_root = reinterpret_cast<int*>(smem + lay.root);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + lay.cnt);
  unsigned long long* s_cnt64 = reinterpret_cast<unsigned long long*>(smem + lay.cnt64);
  uint32_t* s_cpre = reinterpret_cast<uint32_t*>(smem + lay.cpre);
  uint32_t* s_pre = reinterpret_cast<uint32_t*>(smem + lay.pre);
  for (uint32_t s = 0; s < n_scenes; ++s) {
    copy_words(s_sv + s, &B[s].sv, sizeof(SceneView), threadIdx.x, blockDim.x);
    copy_words(s_C + s, &B[s].C, sizeof(ContArgs), threadIdx.x, blockDim.x);
    copy_words(s_T + s, &B[s].T, sizeof(TraceArgs), threadIdx.x, blockDim.x);
  }
  for (uint32_t i = threadIdx.x; i < 6 * n_scenes; i += blockDim.x) s_cnt[i] = 0u;
  for (uint32_t i = threadIdx.x; i < 2 * n_scenes; i += blockDim.x) s_cnt64[i] = 0ull;
  __syncthreads();
  if (threadIdx.x < n_scenes) {
    s_sv[threadIdx.x].moved = F[threadIdx.x].moved;
    s_T[threadIdx.x].frame = F[threadIdx.x].frame;
    s_root[threadIdx.x] = *B[threadIdx.x].sv.root;
  }
  if (threadIdx.x == 0) {
    s_cpre[0] = 0;
    s_pre[0] = 0;
    for (uint32_t s = 0; s < n_scenes; ++s) {
      s_cpre[s + 1] = s_cpre[s] + min(*B[s].C.count, B[s].C.n);
      s_pre[s + 1] = s_pre[s] + min(*B[s].T.count, B[s].T.n);
    }
  }
  __syncthreads();
  const uint32_t n_cont = s_cpre[n_scenes];
  const uint32_t total = n_cont + s_pre[n_scenes];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  Work wk;
  PathState st;
  Ray r;
  Trav t;
  TStack<S> stk;
  uint32_t sc = 0, c_rays = 0, c_photons = 0, cmask = 0, cmeta = 0;
  bool has_ray = false, exhausted = false, cont = false;
  auto flush = [&]() {                         // the finished path's counters to its scene
    uint32_t* c = s_cnt + 6 * sc;
    if (c_rays) atomicAdd(c + 0, c_rays);
    if (c_photons) atomicAdd(c + 1, c_photons);
    if (wk.nodes) atomicAdd(s_cnt64 + 2 * sc + 0, (unsigned long long)wk.nodes);
    if (wk.tris) atomicAdd(s_cnt64 + 2 * sc + 1, (unsigned long long)wk.tris);
    c_rays = c_photons = 0;
    wk.nodes = wk.tris = 0;
  };
  auto cont_flush = [&](const ContCounters& cc) {   // Alg. 1's counters of one step, to the lane's scene
    uint32_t* c = s_cnt + 6 * sc;
    if (cc.rays) atomicAdd(c + 2, cc.rays);
    if (cc.tail) atomicAdd(c + 3, cc.tail);
    if (cc.upd) atomicAdd(c + 4, cc.upd);
    if (cc.trunc) atomicAdd(c + 5, cc.trunc);
  };
  for (uint32_t guard = 0; guard < kGuard; ++guard) {
    const bool need = !has_ray && !exhausted;
    const unsigned nm = __ballot_sync(0xffffffffu, need);
    if (nm) {
      const int leader = __ffs(nm) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&bc->trace, (uint32_t)__popc(nm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const uint32_t idx = base + __popc(nm & lt);
        if (idx < n_cont) {
          sc = scene_of(s_cpre, n_scenes, idx);
          const ContArgs& C = s_C[sc];
          st.pid = C.list[idx - s_cpre[sc]];
          ContCounters cc;
          const bool go = cont_begin(s_sv[sc], C, st.pid, st.cell, st.k, cmask, cmeta, st.E, st.excl, r, cc);
          cont_flush(cc);
          if (go) {
            trav_begin(t, s_root[sc]);
            has_ray = true;
            cont = true;
          } else {
            flush();
          }
        } else if (idx < total) {
          const uint32_t j = idx - n_cont;
          sc = scene_of(s_pre, n_scenes, j);
          if (init_path(s_sv[sc], F[sc].L, s_T[sc], j - s_pre[sc], st, r)) {
            trav_begin(t, s_root[sc]);
            has_ray = true;
            cont = false;
          } else {
            flush();
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted && !has_ray)) break;
    const SceneView& sv = s_sv[sc];
    const bool done = step_warp<kSteps, S>(sv, r, t, stk, st.excl, wk, !has_ray);
    if (!has_ray || !done) continue;
    if (cont) {
      const ContArgs& C = s_C[sc];
      ContCounters cc;
      float3 a_cur;
      int o = cont_hit(sv, C, st.pid, st.cell, st.k, cmask, cmeta, st.E, st.excl, r, t.best, t.tbest, a_cur, cc);
      if (o == kContNext && !cont_next(sv, C, st.pid, st.cell, st.k, cmask, cmeta, st.E, st.excl, a_cur, r, cc))
        o = kContDone;
      cont_flush(cc);
      if (o == kContNext) {
        trav_begin(t, s_root[sc]);
      } else if (o == kContTail && init_pid(sv, F[sc].L, s_T[sc], st.pid, false, st, r)) {
        cont = false;                          // Eq. 2 failed: re-trace from the failing vertex
        trav_begin(t, s_root[sc]);
      } else {
        has_ray = false;
        flush();
      }
      continue;
    }
    ++c_rays;
    if (trace_hit(sv, s_T[sc], st, r, t, c_photons)) {
      trav_begin(t, s_root[sc]);
    } else {
      has_ray = false;
      flush();
    }
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < n_scenes; s += blockDim.x) {
    pv_frame_stats* stt = s_T[s].stats;
    if (!stt) continue;
    const uint32_t* c = s_cnt + 6 * s;
    if (c[0]) atomicAdd(&stt->trace_rays, c[0]);
    if (c[1]) atomicAdd(&stt->photons_written, c[1]);
    if (c[2]) atomicAdd(&stt->cont_rays, c[2]);
    if (c[3]) {                                // the tails join the re-trace list
      atomicAdd(&stt->n_tail, c[3]);
      atomicAdd(&stt->n_listed, c[3]);
    }
    if (c[4]) atomicAdd(&stt->n_updated, c[4]);
    if (c[5]) atomicAdd(&stt->n_truncated, c[5]);
    if (s_cnt64[2 * s + 0]) atomicAdd((unsigned long long*)&stt->node_visits, s_cnt64[2 * s + 0]);
    if (s_cnt64[2 * s + 1]) atomicAdd((unsigned long long*)&stt->tri_tests, s_cnt64[2 * s + 1]);
  }
}

// ---------------------------------------------------------------- kernel selection
using VerifyKernel = void (*)(const BScene*, const BFrame*, const uint32_t*, uint32_t);
using ContKernel = void (*)(const BScene*, const BFrame*, uint32_t, BCounters*);
using TraceKernel = void (*)(const BScene*, const BFrame*, uint32_t, BCounters*);

VerifyKernel verify_kernel(bool vis, bool exact, int mapping) {
  static const VerifyKernel table[2][2][3] = {
      {{k_b_verify<false, false, 0>, k_b_verify<false, false, 1>, k_b_verify<false, false, 2>},
       {k_b_verify<false, true, 0>, k_b_verify<false, true, 1>, k_b_verify<false, true, 2>}},
      {{k_b_verify<true, false, 0>, k_b_verify<true, false, 1>, k_b_verify<true, false, 2>},
       {k_b_verify<true, true, 0>, k_b_verify<true, true, 1>, k_b_verify<true, true, 2>}}};
  return table[vis ? 1 : 0][exact ? 1 : 0][mapping < 0 || mapping > 2 ? 0 : mapping];
}

ContKernel cont_kernel(int stack) { return stack == 32 ? k_b_continue<32> : k_b_continue<64>; }

TraceKernel cont_trace_kernel(int steps, int stack) {
  if (stack == 32)
    return steps == 16 ? k_b_cont_trace<16, 32> : steps == 32 ? k_b_cont_trace<32, 32> : k_b_cont_trace<64, 32>;
  return steps == 16 ? k_b_cont_trace<16, 64> : steps == 32 ? k_b_cont_trace<32, 64> : k_b_cont_trace<64, 64>;
}

TraceKernel trace_kernel(int steps, int stack) {
  if (stack == 32) return steps == 16 ? k_b_trace<16, 32> : steps == 32 ? k_b_trace<32, 32> : k_b_trace<64, 32>;
  return steps == 16 ? k_b_trace<16, 64> : steps == 32 ? k_b_trace<32, 64> : k_b_trace<64, 64>;
}

int thread_index(int threads) { return threads == 64 ? 0 : threads == 128 ? 1 : 2; }

}  // namespace

struct pv_batch {
  std::vector<pv_batch_scene> items;
  uint32_t n = 0;
  pv_verify_params params{};
  bool exact = false;
  int num_sms = 0;
  BScene* d_scenes = nullptr;
  BFrame* d_frames = nullptr;
  BCounters* d_ctr = nullptr;
  BFrame* h_stage = nullptr;                  // pinned [kRing][n]
  cudaEvent_t slot_ev[kRing] = {};
  bool slot_used[kRing] = {};
  uint32_t next_slot = 0;
  uint32_t* d_vtab[3] = {};                   // verify tiles of 64, 128, 256 paths
  int occ_verify[2][3][3] = {};               // resident verify blocks per SM: [vis][mapping][tile size]
  uint32_t n_vtiles[3] = {};
  uint32_t* d_ctab = nullptr;
  uint32_t n_ctiles = 0;
  uint32_t* d_ftab = nullptr;
  uint32_t n_fit = 0;
  bool top_alone = false;                     // some scene has no refit blocks: k_b_frame_top runs
  bool fused = false;                         // no lists asked for: Alg. 1 runs inside the re-trace kernel
  size_t smem_cont = 0, smem_trace = 0, smem_ct = 0;
  int occ_cont[2] = {1, 1};                   // resident blocks per SM: [stack 32, 64]
  int occ_trace[3][2] = {{1, 1}, {1, 1}, {1, 1}};   // [steps 16, 32, 64][stack 32, 64]
  int occ_ct[3][2] = {{1, 1}, {1, 1}, {1, 1}};      // fused kernel, same indices
  uint32_t stack_need = 0;                    // largest over the scenes
  pv_batch_config cfg{0, 256, 64, 0, 64};
  cudaGraph_t graph[2] = {};
  cudaGraphExec_t exec[2] = {};
  cudaGraphNode_t copy_node[2] = {};
  cudaEvent_t ev[6] = {};
  float step_ms[5] = {};
  bool have_times = false;
  // tuning
  bool tuning = false;
  uint32_t tune_per = 1, tune_frame = 0, tune_phase = 0;
  size_t tune_idx = 0;
  std::vector<pv_batch_config> cands;
  std::vector<std::array<double, 5>> cand_ms;
  cudaStream_t last_stream = nullptr;
  cudaStream_t own_stream = nullptr;          // used for a NULL stream (capture needs a real one)
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? PV_OK : PV_ERR_CUDA; }

bool config_valid(const pv_batch* b, const pv_batch_config& c) {
  if (c.verify_mapping < 0 || c.verify_mapping > 2) return false;
  if (c.verify_mapping == 2 && b->params.mode != PV_MODE_ERROR) return false;   // flat: error mode only
  if (c.verify_threads != 64 && c.verify_threads != 128 && c.verify_threads != 256) return false;
  if (c.trace_steps != 16 && c.trace_steps != 32 && c.trace_steps != 64) return false;
  if (c.trace_blocks < 0 || c.trace_blocks > 16) return false;
  if (c.stack != 32 && c.stack != 64) return false;
  if ((uint32_t)c.stack < b->stack_need) return false;
  return true;
}

int stack_index(int stack) { return stack == 32 ? 0 : 1; }
int steps_index(int steps) { return steps == 16 ? 0 : steps == 32 ? 1 : 2; }

// Persistent grid: resident blocks per SM (occupancy measured at creation,
// optionally fewer) times the SM count.
int persistent_blocks(const pv_batch* b, int occupancy, int want) {
  int per = occupancy > 0 ? occupancy : 1;
  if (want > 0 && want < per) per = want;
  return per * b->num_sms;
}

// Every step of one frame, on stream st (captured or eager).  ev: optional
// six events bracketing the steps.
int enqueue_frame(pv_batch* b, cudaStream_t st, bool vis, const pv_batch_config& c, const BFrame* staging,
                  cudaEvent_t* ev) {
  const uint32_t n = b->n;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], st);
  };
  if (cudaMemcpyAsync(b->d_frames, staging, n * sizeof(BFrame), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PV_ERR_CUDA;
  mark(0);
  k_b_prologue<<<n, 256, 0, st>>>(b->d_scenes, b->d_frames, b->d_ctr);
  for (uint32_t i = 0; i < n; ++i) {          // DM_C of moved mapped lights, counted afresh by verification
    pv_scene* s = b->items[i].scene;
    if (!s->has_dm) continue;
    const FrameLights L = pvh::frame_lights(s);
    uint32_t cells = 0;
    for (uint32_t l = 0; l < L.n; ++l) cells = std::max(cells, L.dm[l].dims ? L.dm[l].cells : 0u);
    k_b_dm_clear<<<std::min<uint32_t>((cells + 255) / 256, 8u * (uint32_t)b->num_sms), 256, 0, st>>>(b->d_frames, i);
  }
  if (b->n_fit) k_b_refit_wide<<<b->n_fit, 256, 0, st>>>(b->d_scenes, b->d_frames, b->d_ftab);
  if (b->top_alone) k_b_frame_top<<<n, 32, 0, st>>>(b->d_scenes, b->d_frames);
  mark(1);
  const int ti = thread_index(c.verify_threads);
  const VerifyKernel vk = verify_kernel(vis, b->exact, c.verify_mapping);
  int& per = b->occ_verify[vis ? 1 : 0][c.verify_mapping < 0 || c.verify_mapping > 2 ? 0 : c.verify_mapping][ti];
  if (!per) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, vk, c.verify_threads, 0);
    if (per < 1) per = 1;
  }
  const uint32_t grid = std::min<uint32_t>(b->n_vtiles[ti], pvh::verify_block_cap((uint32_t)per * (uint32_t)b->num_sms));
  vk<<<grid, c.verify_threads, 0, st>>>(b->d_scenes, b->d_frames, b->d_vtab[ti], b->n_vtiles[ti]);
  mark(2);
  if (b->fused) {                             // verify appended what it marked; then Alg. 1 + re-trace
    mark(3);
    mark(4);
    const TraceKernel ctk = cont_trace_kernel(c.trace_steps, c.stack);
    ctk<<<persistent_blocks(b, b->occ_ct[steps_index(c.trace_steps)][stack_index(c.stack)], c.trace_blocks),
          pvh::kTraceThreads, b->smem_ct, st>>>(b->d_scenes, b->d_frames, n, b->d_ctr);
    mark(5);
    return cuda_rc(cudaGetLastError());
  }
  if (b->params.mode == PV_MODE_ERROR) {
    const ContKernel ck = cont_kernel(c.stack);
    ck<<<persistent_blocks(b, b->occ_cont[stack_index(c.stack)], 0), 128, b->smem_cont, st>>>(
        b->d_scenes, b->d_frames, n, b->d_ctr);
  }
  // with distribution maps: prune and fill, which need Alg. 1's final answer for every path
  for (uint32_t i = 0; i < n; ++i) {
    pv_scene* s = b->items[i].scene;
    if (!s->has_dm) continue;
    const uint32_t np = b->items[i].paths.n, blocks = (np + 255) / 256;
    if (!np) continue;
    if (cudaMemsetAsync(s->dm_ctr, 0, 8 * sizeof(uint32_t), st) != cudaSuccess) return PV_ERR_CUDA;
    k_b_dm_prune<<<blocks, 256, 0, st>>>(b->d_scenes, b->d_frames, i, s->dm_flag);
    k_b_dm_commit<<<blocks, 256, 0, st>>>(b->d_scenes, b->d_frames, i, s->dm_flag, s->dm_ctr);
    pvh::launch_compact(s, s->dm_flag, np, s->dm_free, s->dm_ctr + 4, nullptr, st);
    // that compaction used the scene's tile states: cleared again for the re-trace list's compaction below
    if (cudaMemsetAsync(s->ws_tiles, 0, (size_t)((np + pvh::kTile - 1) / pvh::kTile) * sizeof(uint64_t), st) !=
        cudaSuccess)
      return PV_ERR_CUDA;
    const FrameLights L = pvh::frame_lights(s);
    for (uint32_t l = 0; l < L.n; ++l) {
      if (!L.dm[l].dims) continue;
      k_b_dm_deficit<<<(L.dm[l].cells + 256) / 256, 256, 0, st>>>(b->d_frames, i, l, s->dm_scan);
      pvh::exclusive_scan(s->dm_scan, L.dm[l].cells + 1, st);
      const uint32_t fb = std::min<uint32_t>((s->lights_new[l].n_paths + 255) / 256, 8u * (uint32_t)s->num_sms);
      k_b_dm_fill<<<std::max<uint32_t>(fb, 1u), 256, 0, st>>>(b->d_scenes, b->d_frames, i, l, s->dm_free, s->dm_ctr,
                                                             s->dm_scan);
    }
  }
  mark(3);
  k_b_compact<<<b->n_ctiles, pvh::kCompactThreads, 0, st>>>(b->d_scenes, b->d_ctab, b->d_ctr);
  mark(4);
  const TraceKernel tk = trace_kernel(c.trace_steps, c.stack);
  tk<<<persistent_blocks(b, b->occ_trace[steps_index(c.trace_steps)][stack_index(c.stack)], c.trace_blocks),
       pvh::kTraceThreads,
       b->smem_trace, st>>>(b->d_scenes, b->d_frames, n, b->d_ctr);
  mark(5);
  return cuda_rc(cudaGetLastError());
}

void drop_graphs(pv_batch* b) {
  for (int v = 0; v < 2; ++v) {
    if (b->exec[v]) cudaGraphExecDestroy(b->exec[v]);
    if (b->graph[v]) cudaGraphDestroy(b->graph[v]);
    b->exec[v] = nullptr;
    b->graph[v] = nullptr;
    b->copy_node[v] = nullptr;
  }
}

int capture(pv_batch* b, int vis, cudaStream_t st) {
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PV_ERR_CUDA;
  const int rc = enqueue_frame(b, st, vis != 0, b->cfg, b->h_stage, nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != PV_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return PV_ERR_CUDA;
  }
  size_t count = 0;
  if (cudaGraphGetNodes(g, nullptr, &count) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PV_ERR_CUDA;
  }
  std::vector<cudaGraphNode_t> nodes(count);
  cudaGraphGetNodes(g, nodes.data(), &count);
  cudaGraphNode_t copy = nullptr;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeMemcpy) copy = nd;
  }
  cudaGraphExec_t ex = nullptr;
  if (!copy || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PV_ERR_CUDA;
  }
  b->graph[vis] = g;
  b->exec[vis] = ex;
  b->copy_node[vis] = copy;
  return PV_OK;
}

// Candidate list of a tuning phase around the current configuration.
std::vector<pv_batch_config> phase_candidates(const pv_batch* b, uint32_t phase) {
  std::vector<pv_batch_config> out;
  const pv_batch_config base = b->cfg;
  if (phase == 0) {                           // re-trace and continuation: steps, blocks per SM, stack
    for (int stack : {32, 64})
      for (int steps : {16, 32, 64})
        for (int blocks : {0, 4}) {
          pv_batch_config c = base;
          c.stack = stack;
          c.trace_steps = steps;
          c.trace_blocks = blocks;
          if (config_valid(b, c)) out.push_back(c);
        }
  } else {                                    // verify: mapping and tile size
    for (int mapping : {0, 1, 2})
      for (int threads : {64, 128, 256}) {
        pv_batch_config c = base;
        c.verify_mapping = mapping;
        c.verify_threads = threads;
        if (config_valid(b, c)) out.push_back(c);
      }
  }
  return out;
}

// Close the current tuning phase: keep the candidate with the fastest whole frame.
void finish_phase(pv_batch* b) {
  size_t best = 0;
  double best_ms = 1e300;
  for (size_t i = 0; i < b->cands.size(); ++i) {
    const auto& m = b->cand_ms[i];
    // whole frame: the verify mapping sets the order of the re-trace list, so it moves the
    // re-trace's time as well as its own
    const double ms = m[0] + m[1] + m[2] + m[3] + m[4];
    if (ms < best_ms) {
      best_ms = ms;
      best = i;
    }
  }
  if (!b->cands.empty()) {
    b->cfg = b->cands[best];
    for (int k = 0; k < 5; ++k) b->step_ms[k] = (float)(b->cand_ms[best][k] / b->tune_per);
    b->have_times = true;
  }
  ++b->tune_phase;
  b->tune_idx = 0;
  b->tune_frame = 0;
  if (b->tune_phase >= 2) {
    b->tuning = false;
    b->cands.clear();
    b->cand_ms.clear();
    drop_graphs(b);
    return;
  }
  b->cands = phase_candidates(b, b->tune_phase);
  b->cand_ms.assign(b->cands.size(), std::array<double, 5>{0, 0, 0, 0, 0});
  if (b->cands.empty()) finish_phase(b);
}

void free_batch(pv_batch* b) {
  if (!b) return;
  drop_graphs(b);
  for (auto& e : b->slot_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  void* ptrs[] = {b->d_scenes, b->d_frames, b->d_ctr, b->d_vtab[0], b->d_vtab[1], b->d_vtab[2],
                  b->d_ctab, b->d_ftab};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

int upload_table(const std::vector<uint32_t>& v, uint32_t** out) {
  if (v.empty()) return PV_OK;
  if (cudaMalloc(out, v.size() * sizeof(uint32_t)) != cudaSuccess) return PV_ERR_OOM;
  return cuda_rc(cudaMemcpy(*out, v.data(), v.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
}

}  // namespace

extern "C" int pv_batch_create(const pv_batch_scene* scenes, uint32_t n, const pv_verify_params* params, void* stream,
                               pv_batch** out) {
  if (!out) return PV_ERR_ARG;
  *out = nullptr;
  if (!scenes || !params || n == 0) return PV_ERR_ARG;
  if (n > kBatchMax) return PV_ERR_LIMIT;
  if (params->mode < PV_MODE_NAIVE_AABB || params->mode > PV_MODE_ERROR || !(params->tau >= 0.0f)) return PV_ERR_ARG;
  const bool fused = !scenes[0].d_list;       // lists for every scene, or for none
  for (uint32_t i = 0; i < n; ++i) {
    const pv_batch_scene& it = scenes[i];
    if (pvh::check_paths(it.scene, &it.paths) != PV_OK) return PV_ERR_ARG;
    if (!it.d_list != fused || !it.d_count != fused) return PV_ERR_ARG;
    // a graph replays refits, not the data-dependent rebuild; with maps, prune and fill need every path's
    // Alg. 1 answer before the list is made, so those batches run with lists
    if ((it.scene->flags & PV_BUILD_DYN_REBUILD) || (it.scene->has_dm && fused)) return PV_ERR_STATE;
    for (uint32_t j = 0; j < i; ++j)
      if (scenes[j].scene == it.scene) return PV_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  pv_batch* b = new pv_batch;
  b->items.assign(scenes, scenes + n);
  b->n = n;
  b->fused = fused;
  b->params = *params;
  if (params->mode == PV_MODE_ERROR) {        // measured best on the 16-district batch before any tuning
    b->cfg.verify_mapping = 2;
    b->cfg.verify_threads = 128;
    b->cfg.trace_steps = 32;
  }
  b->exact = params->mode == PV_MODE_NAIVE_EXACT ||
             (params->mode == PV_MODE_ERROR && (params->flags & PV_FLAG_ERROR_EXACT));
  b->num_sms = scenes[0].scene->num_sms;
  int rc = PV_OK;
  auto fail = [&](int r) { if (r != PV_OK && rc == PV_OK) rc = r; };
  // static per-scene records and work tables
  std::vector<BScene> hs(n);
  std::vector<uint32_t> vt[3], ct, ft;
  const uint32_t vthreads[3] = {64, 128, 256};
  for (uint32_t i = 0; i < n && rc == PV_OK; ++i) {
    pv_scene* s = scenes[i].scene;
    const pv_paths& p = scenes[i].paths;
    uint32_t need = 0;
    fail(pvh::stack_need(s, &need));
    b->stack_need = std::max(b->stack_need, need);
    s->moved = 0;                              // the batch's first frame compares against the current poses
    BScene& B = hs[i];
    std::memset(&B, 0, sizeof B);
    B.sv = pvh::view(s);
    B.V.n = p.n;
    B.V.info = p.info;
    B.V.origin = p.origin;
    B.V.pa = reinterpret_cast<float4*>(p.pa);
    B.V.pb = reinterpret_cast<const float4*>(p.pb);
    B.V.mode = params->mode;
    B.V.tau = params->tau;
    B.V.flags = params->flags;
    B.V.mask_out = s->ws_mask;
    B.V.cont_list = s->ws_cont;
    B.V.cont_count = s->ws_ctr + pvh::CTR_ALL;
    B.V.stats = scenes[i].d_stats;
    B.C.n = p.n;
    B.C.info = p.info;
    B.C.origin = p.origin;
    B.C.pa = reinterpret_cast<float4*>(p.pa);
    B.C.pb = reinterpret_cast<const float4*>(p.pb);
    B.C.mask = s->ws_mask;
    B.C.list = s->ws_cont;
    B.C.count = s->ws_ctr + pvh::CTR_ALL;
    B.C.ticket = nullptr;
    B.C.tau = params->tau;
    B.C.stats = scenes[i].d_stats;
    B.T.n = p.n;
    B.T.info = p.info;
    B.T.origin = p.origin;
    B.T.pa = reinterpret_cast<float4*>(p.pa);
    B.T.pb = reinterpret_cast<float4*>(p.pb);
    uint32_t* const list = fused ? s->ws_list : scenes[i].d_list;
    uint32_t* const count = fused ? s->ws_ctr + pvh::CTR_LIST : scenes[i].d_count;
    B.T.list = list;
    B.T.count = count;
    B.T.ticket = nullptr;
    B.T.seed = scenes[i].seed;
    B.T.frame = 0;
    B.T.stats = scenes[i].d_stats;
    B.d_local = s->d_local;
    B.d_tri_prim = s->d_tri_prim;
    B.dtris = s->tris + s->d_tri_off;
    B.objs = s->objs;
    B.groups = s->groups;
    B.xf_old = s->xf_old;
    B.xf_new = s->xf_new;
    B.bnodes = s->nodes;
    B.dnodes = s->nodes + s->d_node_off;
    B.node_parent = s->d_node_parent;
    B.leaf_parent = s->d_leaf_parent;
    B.fit_flags = s->d_fit_flags;
    B.n_dyn_tris = s->n_dyn_tris;
    B.n_dyn = s->n_dyn;
    B.tri_slot = s->d_tri_slot;
    B.t_link = s->t_link;
    B.w_link = s->w_link;
    B.w_nch = s->w_nch;
    B.w_arrive = s->w_arrive;
    B.obox = s->obox;
    B.wsrc_dyn = s->wsrc + 4 * (size_t)s->w_dyn_off;
    B.wcount_dyn = s->wcount + 1;
    B.wnodes_dyn = s->wnodes + s->w_dyn_off;
    B.wnodes = s->wnodes;
    B.tris = s->tris;
    B.top_off = (int)s->w_top_off;
    B.s_wroot = s->s_wroot;
    B.root = s->root;
    B.n_tiles = (p.n + pvh::kTile - 1) / pvh::kTile;
    B.tiles = reinterpret_cast<unsigned long long*>(s->ws_tiles);
    B.list = list;
    B.count = count;
    B.stat_listed = scenes[i].d_stats ? &scenes[i].d_stats->n_listed : nullptr;
    if (fused) {                               // verify appends the paths it marks: no compaction pass
      B.V.list_out = list;
      B.V.list_count = count;
    }
    B.ctr = s->ws_ctr;
    for (int k = 0; k < 3; ++k)
      for (uint32_t t = 0; t < (p.n + vthreads[k] - 1) / vthreads[k]; ++t) {
        vt[k].push_back(i);
        vt[k].push_back(t);
      }
    for (uint32_t t = 0; t < B.n_tiles; ++t) {
      ct.push_back(i);
      ct.push_back(t);
    }
    B.refit_blocks = 0;
    for (uint32_t base = 0; base < s->n_dyn_tris; base += 256) {
      ft.push_back(i);
      ft.push_back(base);
      ++B.refit_blocks;
    }
    B.refit_done = s->w_arrive ? s->w_arrive + s->n_dyn_tris : nullptr;   // the word after the arrival counters
    if (!B.refit_blocks) b->top_alone = true;
  }
  for (int k = 0; k < 3; ++k) b->n_vtiles[k] = (uint32_t)vt[k].size() / 2;
  b->n_ctiles = (uint32_t)ct.size() / 2;
  b->n_fit = (uint32_t)ft.size() / 2;
  if (rc == PV_OK) {
    if (cudaMalloc(&b->d_scenes, n * sizeof(BScene)) != cudaSuccess ||
        cudaMalloc(&b->d_frames, n * sizeof(BFrame)) != cudaSuccess ||
        cudaMalloc(&b->d_ctr, sizeof(BCounters)) != cudaSuccess ||
        cudaMallocHost(&b->h_stage, kRing * n * sizeof(BFrame)) != cudaSuccess)
      rc = PV_ERR_OOM;
  }
  for (int k = 0; k < 3 && rc == PV_OK; ++k) fail(upload_table(vt[k], &b->d_vtab[k]));
  if (rc == PV_OK) fail(upload_table(ct, &b->d_ctab));
  if (rc == PV_OK) fail(upload_table(ft, &b->d_ftab));
  if (rc == PV_OK) fail(cuda_rc(cudaMemcpy(b->d_scenes, hs.data(), n * sizeof(BScene), cudaMemcpyHostToDevice)));
  for (int k = 0; k < kRing && rc == PV_OK; ++k)
    fail(cuda_rc(cudaEventCreateWithFlags(&b->slot_ev[k], cudaEventDisableTiming)));
  for (int k = 0; k < 6 && rc == PV_OK; ++k) fail(cuda_rc(cudaEventCreate(&b->ev[k])));
  if (rc == PV_OK) fail(cuda_rc(cudaStreamCreate(&b->own_stream)));   // blocking: ordered with the legacy stream
  if (rc == PV_OK) {
    b->smem_cont = PersistLayout<ContArgs>(n).bytes;
    b->smem_trace = PersistLayout<TraceArgs>(n).bytes;
    b->smem_ct = FusedLayout(n).bytes;
    for (int s : {32, 64}) {
      const void* ck = (const void*)cont_kernel(s);
      fail(cuda_rc(cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_cont)));
      fail(cuda_rc(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ_cont[stack_index(s)], ck, 128, b->smem_cont)));
      for (int steps : {16, 32, 64}) {
        const void* tk = (const void*)trace_kernel(steps, s);
        fail(cuda_rc(cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_trace)));
        fail(cuda_rc(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ_trace[steps_index(steps)][stack_index(s)],
                                                                   tk, pvh::kTraceThreads, b->smem_trace)));
        const void* ctk = (const void*)cont_trace_kernel(steps, s);
        fail(cuda_rc(cudaFuncSetAttribute(ctk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_ct)));
        fail(cuda_rc(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ_ct[steps_index(steps)][stack_index(s)],
                                                                   ctk, pvh::kTraceThreads, b->smem_ct)));
      }
    }
    if (b->stack_need <= 32) b->cfg.stack = 32;
  }
  if (rc != PV_OK) {
    free_batch(b);
    return rc;
  }
  b->last_stream = st;
  *out = b;
  return PV_OK;
}

extern "C" int pv_batch_frame(pv_batch* b, const float* const* xforms, const pv_light* const* lights, uint32_t frame,
                              void* stream) {
  if (!b) return PV_ERR_ARG;
  cudaStream_t st = stream ? (cudaStream_t)stream : b->own_stream;
  for (uint32_t i = 0; i < b->n; ++i) {
    const int rc = pvh::stage_poses(b->items[i].scene, xforms ? xforms[i] : nullptr, lights ? lights[i] : nullptr);
    if (rc != PV_OK) return rc;
  }
  const uint32_t slot = b->next_slot;
  b->next_slot = (slot + 1) % kRing;
  if (b->slot_used[slot] && cudaEventSynchronize(b->slot_ev[slot]) != cudaSuccess) return PV_ERR_CUDA;
  BFrame* stage = b->h_stage + (size_t)slot * b->n;
  bool vis = false;
  for (uint32_t i = 0; i < b->n; ++i) {
    pv_scene* s = b->items[i].scene;
    BFrame& f = stage[i];
    f.L = pvh::frame_lights(s);
    std::memset(f.xf, 0, sizeof f.xf);
    for (uint32_t sl = 0; sl < s->n_dyn; ++sl) std::memcpy(f.xf[sl], &s->h_xf_new[12 * sl], 12 * sizeof(float));
    f.moved = s->moved;
    f.frame = frame;
    f.pad = 0;
    for (uint32_t l = 0; l < s->n_lights; ++l)
      if (((f.L.moved_mask >> l) & 1u) && s->lights_new[l].type == PV_LIGHT_POINT) vis = true;
    s->last_stream = st;
  }
  int rc = PV_OK;
  if (b->tuning) {
    const pv_batch_config c = b->cands[b->tune_idx];
    rc = enqueue_frame(b, st, vis, c, stage, b->ev);
    if (rc == PV_OK && cudaEventSynchronize(b->ev[5]) != cudaSuccess) rc = PV_ERR_CUDA;
    if (rc == PV_OK) {
      auto& m = b->cand_ms[b->tune_idx];
      for (int k = 0; k < 5; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev[k], b->ev[k + 1]);
        m[k] += ms;
      }
      // Round robin: candidate i runs on frames i, i + n, i + 2n, ... of the phase, so a
      // workload that drifts from frame to frame weighs on every candidate alike.
      if (++b->tune_idx >= b->cands.size()) {
        b->tune_idx = 0;
        if (++b->tune_frame >= b->tune_per) finish_phase(b);
      }
    }
  } else if (!b->exec[vis ? 1 : 0] && (rc = capture(b, vis ? 1 : 0, st)) != PV_OK) {
    // capture failed: nothing enqueued for this frame
  } else {
    const int v = vis ? 1 : 0;
    rc = cuda_rc(cudaGraphExecMemcpyNodeSetParams1D(b->exec[v], b->copy_node[v], b->d_frames, stage,
                                                     b->n * sizeof(BFrame), cudaMemcpyHostToDevice));
    if (rc == PV_OK) rc = cuda_rc(cudaGraphLaunch(b->exec[v], st));
  }
  if (rc == PV_OK) rc = cuda_rc(cudaEventRecord(b->slot_ev[slot], st));
  b->slot_used[slot] = rc == PV_OK;
  b->last_stream = st;
  return rc;
}

extern "C" int pv_batch_autotune(pv_batch* b, uint32_t frames_per_candidate) {
  if (!b) return PV_ERR_ARG;
  b->tuning = true;
  b->tune_per = frames_per_candidate ? frames_per_candidate : 1;
  b->tune_phase = 0;
  b->tune_idx = 0;
  b->tune_frame = 0;
  b->cands = phase_candidates(b, 0);
  b->cand_ms.assign(b->cands.size(), std::array<double, 5>{0, 0, 0, 0, 0});
  if (b->cands.empty()) finish_phase(b);
  return PV_OK;
}

extern "C" int pv_batch_tuning(const pv_batch* b) { return b ? (b->tuning ? 1 : 0) : PV_ERR_ARG; }

extern "C" int pv_batch_set_config(pv_batch* b, const pv_batch_config* cfg) {
  if (!b || !cfg || !config_valid(b, *cfg)) return PV_ERR_ARG;
  b->cfg = *cfg;
  drop_graphs(b);
  return PV_OK;
}

extern "C" int pv_batch_get_config(const pv_batch* b, pv_batch_config* cfg) {
  if (!b || !cfg) return PV_ERR_ARG;
  *cfg = b->cfg;
  return PV_OK;
}

extern "C" int pv_batch_step_times(const pv_batch* b, float* ms5) {
  if (!b || !ms5) return PV_ERR_ARG;
  if (!b->have_times) return PV_ERR_STATE;
  std::memcpy(ms5, b->step_ms, sizeof b->step_ms);
  return PV_OK;
}

extern "C" void pv_batch_destroy(pv_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->last_stream);
  cudaStreamSynchronize(b->own_stream);
  // the scenes must not keep the batch's own stream (destroyed below) as their last stream
  for (const pv_batch_scene& it : b->items)
    if (it.scene->last_stream == b->own_stream) it.scene->last_stream = nullptr;
  free_batch(b);
}
