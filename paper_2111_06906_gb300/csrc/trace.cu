// Persistent re-trace of the listed paths (and the trace-all baseline).
//
// "Generate rays" and "trace rays" of Fig. 2 fused into one kernel.  Each
// lane owns one path and one ray at a time.  A warp advances its lanes'
// traversals step by step until every lane's ray has ended, or for at most a
// fixed number of steps; then each lane whose ray ended stores the photon and
// starts its next ray (the next bounce, or the next list entry, taken with
// one atomic per warp), so a long ray holds its warp's other lanes only that
// many steps.  Rays are generated where the paper generates them (Sec. 4):
// from the light (start 0), or by Russian roulette and a cosine-weighted
// bounce at the first photon to re-trace.
#include <cstdlib>
#include <cstring>

#include "deposit_core.cuh"
#include "trace_core.cuh"
#include "verify_core.cuh"

using namespace pvk;

namespace {

// Compile-time tuning: minimum resident blocks; traversal steps between
// refills.  A warp keeps stepping until every lane's ray has ended (at most
// PV_TRACE_MAX_STEPS steps), so that the ray-end code (photon store, bounce
// sampling, next list entry) runs with all lanes at once: measured on the
// city and villa workloads this beats refilling each lane after a fixed
// number of steps (8) by 8-13 % on the re-trace and 14-15 % on trace-all.
// PV_TRACE_DONE_LANES < 32 stops once that many lanes are done (after at
// least PV_TRACE_STEPS steps); PV_TRACE_DONE_LANES > 32 restores the fixed
// PV_TRACE_STEPS-step loop.
#ifndef PV_TRACE_STEPS
#define PV_TRACE_STEPS 16
#endif
// Resident blocks asked of the register allocator: k_trace fits 8 blocks
// (64 registers) without spills, and that beat 7 by 3-5 % on the city and
// villa trace-all frames; k_cont_trace keeps 7 (72 registers), since 8 spill
// (and moving its per-path state to shared memory to avoid that cost more
// than the eighth block gained).
#ifndef PV_TRACE_MIN_BLOCKS
#define PV_TRACE_MIN_BLOCKS 8
#endif
// k_trace with the deposit (the trace-all frame): 8 blocks spill 24 bytes and
// still beat 7 blocks without spills by 4-5 % (villa 4.18 against 4.38 ms).
#ifndef PV_TRACE_DEP_MIN_BLOCKS
#define PV_TRACE_DEP_MIN_BLOCKS 8
#endif
#ifndef PV_CONT_TRACE_MIN_BLOCKS
#define PV_CONT_TRACE_MIN_BLOCKS 7
#endif
// k_cont_trace with the deposit: 1 deals the photons of the paths the warp's
// lanes finished out over its lanes (deposit_warp), 0 lets each lane deposit
// its own path's photons.
#ifndef PV_DEP_WARP
#define PV_DEP_WARP 1
#endif
#ifndef PV_TRACE_MAX_STEPS
#define PV_TRACE_MAX_STEPS 64
#endif
#ifndef PV_TRACE_DONE_LANES
#define PV_TRACE_DONE_LANES 32
#endif
// Traversal stack entries kept in shared memory (the rest in local memory).
// Measured on the city and villa workloads, 8, 16 or 32 shared entries made
// the re-trace and trace-all kernels 5-7 % slower than a local-memory stack,
// so the default keeps none.
#ifndef PV_TRACE_STACK_SHARED
#define PV_TRACE_STACK_SHARED 0
#endif
constexpr int kStackShared = PV_TRACE_STACK_SHARED < kStack ? PV_TRACE_STACK_SHARED : kStack;
using TraceStack = TStack<kStack, kStackShared, pvh::kTraceThreads>;
constexpr int kStackSharedWords = kStackShared > 0 ? kStackShared * pvh::kTraceThreads : 1;
// Wide nodes of the static tree's top levels copied into shared memory by
// every block of the persistent kernels (0: none).  Measured on the city and
// villa workloads, 64, 128 and 192 nodes (8.5-25 KB per block) made the
// re-trace 5-9 % and trace-all 6-14 % slower: the top nodes are L1 hits
// anyway, and the copy takes L1 capacity and turns every node load into a
// generic one.  The default keeps none.
#ifndef PV_TRACE_NODE_CACHE
#define PV_TRACE_NODE_CACHE 0
#endif
constexpr int kNodeCache = PV_TRACE_NODE_CACHE;

// Copy the first min(kNodeCache, static wide nodes) nodes into ``cache``
// (all threads of the block); returns how many.
__device__ __forceinline__ int fill_node_cache(const SceneView& sv, WNode* cache) {
  if (kNodeCache == 0) return 0;
  const int n = (int)min((uint32_t)kNodeCache, sv.n_static_wide);
  const float4* src = reinterpret_cast<const float4*>(sv.nodes);
  float4* dst = reinterpret_cast<float4*>(cache);
  for (int i = threadIdx.x; i < n * 8; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
  return n;
}
constexpr int kStepsPerIter = PV_TRACE_STEPS;
constexpr int kMaxSteps = PV_TRACE_MAX_STEPS;
constexpr int kDoneLanes = PV_TRACE_DONE_LANES;

// Advance the lane's ray; all lanes of the warp call it (lanes without a ray
// pass done = true).  Returns whether the lane's ray has ended.
__device__ __forceinline__ bool step_rays(const SceneView& sv, const Ray& r, Trav& t, TraceStack& stk, int excl, Work& wk,
                                          bool done, const WNode* cache, int n_cache) {
  if (kDoneLanes > 32) {
#pragma unroll 1
    for (int i = 0; i < kStepsPerIter && !done; ++i) done = trav_step(sv, r, t, stk, excl, wk, cache, n_cache);
    return done;
  }
  if (kDoneLanes >= 32) return step_warp<kMaxSteps>(sv, r, t, stk, excl, wk, done, cache, n_cache);
#pragma unroll 1
  for (int i = 0; i < kMaxSteps; ++i) {
    if (!done) done = trav_step(sv, r, t, stk, excl, wk, cache, n_cache);
    const unsigned dm = __ballot_sync(0xffffffffu, done);
    if (dm == 0xffffffffu) break;
    if (i + 1 >= kStepsPerIter && __popc(dm) >= kDoneLanes) break;
  }
  return done;
}

// Re-trace (A.list) or trace-all; with kDep every photon stored is also
// deposited into am's atlas as it is stored (the fused trace-all frame).
template <bool kDep>
__global__ void __launch_bounds__(pvh::kTraceThreads, kDep ? PV_TRACE_DEP_MIN_BLOCKS : PV_TRACE_MIN_BLOCKS)
    k_trace(SceneView sv, FrameLights L, TraceArgs A, AtlasMap am) {
  __shared__ uint32_t s_red[32 * 2];
  __shared__ unsigned long long s_red64[32];
  const int root = *sv.root;
  const uint32_t total = A.list ? *A.count : A.n;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  Work wk;
  PathState s;
  Ray r;
  Trav t;
  __shared__ int s_stk[kStackSharedWords];
  TraceStack stk;
  stk.sh = s_stk + threadIdx.x;
  __shared__ WNode s_nodes[kNodeCache > 0 ? kNodeCache : 1];
  const int n_cache = fill_node_cache(sv, s_nodes);
  const WNode* const cache = kNodeCache > 0 ? s_nodes : nullptr;
  bool has_ray = false, exhausted = false;
  uint32_t c_rays = 0, c_photons = 0;
  for (uint32_t guard = 0; guard < (1u << 30); ++guard) {
    const bool need = !has_ray && !exhausted;
    const unsigned nm = __ballot_sync(0xffffffffu, need);
    if (nm) {
      const int leader = __ffs(nm) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(A.ticket, (uint32_t)__popc(nm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const uint32_t idx = base + __popc(nm & lt);
        if (idx < total) {
          if (init_path(sv, L, A, idx, s, r)) {
            trav_begin(t, root);
            has_ray = true;
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted && !has_ray)) break;
    if (kDoneLanes > 32 && !has_ray) continue;
    const bool done = step_rays(sv, r, t, stk, s.excl, wk, !has_ray, cache, n_cache);
    if (!has_ray || !done) continue;
    ++c_rays;
    if (trace_hit<kDep>(sv, A, s, r, t, c_photons, &am)) trav_begin(t, root);
    else has_ray = false;
  }
  uint32_t* const ctr[2] = {A.stats ? &A.stats->trace_rays : nullptr, A.stats ? &A.stats->photons_written : nullptr};
  const uint32_t val[2] = {c_rays, c_photons};
  block_add_n<2>(ctr, val, s_red);
  block_add64(A.stats ? (unsigned long long*)&A.stats->node_visits : nullptr, wk.nodes, s_red64);
  block_add64(A.stats ? (unsigned long long*)&A.stats->tri_tests : nullptr, wk.tris, s_red64);
}


// Alg. 1 (Sec. 3.3) fused with the re-trace.  The work items are the paths
// the box test sent to Alg. 1, then the paths verification itself marked for
// re-tracing.  A continuation lane runs Alg. 1's closest-hit queries through
// the same resumable traversal as the re-trace rays, so its queries
// interleave with other lanes' rays instead of holding a separate kernel to
// its slowest chain; a path whose Eq. 2 test fails goes on to its re-trace
// from the failing vertex in the same lane.  Every path sees the same
// arithmetic as in k_continue followed by k_trace, so the records are
// identical; only the order in which paths are processed differs.
//
// With a deposit (kDep 1) the atlas deposit joins the kernel.  A lane deposits each path it
// finishes as soon as it is final; after the re-trace items come the paths
// verification left untouched (touched[p] == 0), whose deposit fills the
// lanes that have no more rays to trace.  Every path is deposited once, by
// the same per-photon arithmetic as k_deposit, into integer sums: the atlas
// is the same bit for bit.
//
// kDep 2: the atlas already holds the deposit of the records as they were on
// entry, and k_verify has taken the touched paths' entry photons out of it.
// A lane deposits the final photons of each path it finishes; untouched
// paths are not visited.  Integer sums make the result the same, bit for
// bit, as a cleared atlas with every path deposited.
struct DepositArgs {
  pv_atlas at;
  const uint8_t* touched;
};

__device__ __forceinline__ void cont_flush(ContCounters& cc, uint32_t* s_cnt) {
  if (cc.rays) atomicAdd(s_cnt + 0, cc.rays);
  if (cc.tail) atomicAdd(s_cnt + 1, cc.tail);
  if (cc.upd) atomicAdd(s_cnt + 2, cc.upd);
  if (cc.trunc) atomicAdd(s_cnt + 3, cc.trunc);
}

// kDep: 0 no deposit, 1 deposit into a cleared atlas, 2 carried atlas (delta).
//
// Launched as a programmatic dependent of k_verify (PV_CONT_TRACE_PDL), its
// blocks may be placed on the SMs while k_verify's last blocks run, and wait
// below until k_verify has finished and its writes are visible; for the
// default ordinary launch the wait returns at once.
template <int kDep>
__global__ void __launch_bounds__(pvh::kTraceThreads, PV_CONT_TRACE_MIN_BLOCKS)
    k_cont_trace(SceneView sv, FrameLights L, TraceArgs A, ContArgs C, DepositArgs D) {
  __shared__ uint32_t s_red[32 * 2];
  __shared__ unsigned long long s_red64[32];
  __shared__ uint32_t s_cnt[4];
  if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0u;
  grid_dependency_wait();
  __syncthreads();
  const int root = *sv.root;
  const uint32_t n_cont = min(*C.count, C.n);
  const uint32_t n_trace = n_cont + min(*A.count, A.n);
  constexpr bool kDeposit = kDep != 0;
  const uint32_t total = n_trace + (kDep == 1 ? A.n : 0u);
  const int lane = threadIdx.x & 31;
  uint32_t dep = 0xFFFFFFFFu;                // a final path this lane still has to deposit
  auto deposit = [&](uint32_t p) {
    if (kDeposit) dep = p;
  };
  const unsigned lt = (1u << lane) - 1u;
  Work wk;
  PathState s;
  Ray r;
  Trav t;
  __shared__ int s_stk[kStackSharedWords];
  TraceStack stk;
  stk.sh = s_stk + threadIdx.x;
  __shared__ WNode s_nodes[kNodeCache > 0 ? kNodeCache : 1];
  const int n_cache = fill_node_cache(sv, s_nodes);
  const WNode* const cache = kNodeCache > 0 ? s_nodes : nullptr;
  uint32_t cmask = 0, cmeta = 0;             // Alg. 1 state beyond s.k (segment), s.E (a_orig), s.excl (a_prim)
  bool has_ray = false, exhausted = false, cont = false;
  uint32_t c_rays = 0, c_photons = 0;
  for (uint32_t guard = 0; guard < (1u << 30); ++guard) {
    if (PV_DEP_WARP && kDeposit && __any_sync(0xffffffffu, dep != 0xFFFFFFFFu)) {
      deposit_warp(atlas_map(D.at), A.n, sv.B, A.info, A.pa, A.pb, dep);   // scales per call: no registers held
      dep = 0xFFFFFFFFu;
    }
    if (!PV_DEP_WARP && kDeposit && dep != 0xFFFFFFFFu) {
      deposit_path(atlas_map(D.at), A.n, sv.B, A.info, A.pa, A.pb, dep);   // scales per path: no registers held
      dep = 0xFFFFFFFFu;
    }
    const bool need = !has_ray && !exhausted;
    const unsigned nm = __ballot_sync(0xffffffffu, need);
    if (nm) {
      const int leader = __ffs(nm) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(A.ticket, (uint32_t)__popc(nm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const uint32_t idx = base + __popc(nm & lt);
        if (idx < n_cont) {
          ContCounters cc;
          s.pid = C.list[idx];
          if (cont_begin(sv, C, s.pid, s.cell, s.k, cmask, cmeta, s.E, s.excl, r, cc)) {
            trav_begin(t, root);
            has_ray = true;
            cont = true;
          } else {
            deposit(s.pid);
          }
          cont_flush(cc, s_cnt);
        } else if (idx < n_trace) {
          if (init_path(sv, L, A, idx - n_cont, s, r)) {
            trav_begin(t, root);
            has_ray = true;
            cont = false;
          } else {
            deposit(s.pid);
          }
        } else if (idx < total) {                // deposit of a path this frame left untouched
          const uint32_t p = idx - n_trace;
          if (!D.touched[p]) deposit(p);
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted && !has_ray && dep == 0xFFFFFFFFu)) break;
    if (kDoneLanes > 32 && !has_ray) continue;
    const bool done = step_rays(sv, r, t, stk, s.excl, wk, !has_ray, cache, n_cache);
    if (!has_ray || !done) continue;
    if (cont) {
      ContCounters cc;
      float3 a_cur;
      int o = cont_hit(sv, C, s.pid, s.cell, s.k, cmask, cmeta, s.E, s.excl, r, t.best, t.tbest, a_cur, cc);
      if (o == kContNext && !cont_next(sv, C, s.pid, s.cell, s.k, cmask, cmeta, s.E, s.excl, a_cur, r, cc))
        o = kContDone;
      cont_flush(cc, s_cnt);
      if (o == kContNext) {
        trav_begin(t, root);
      } else if (o == kContTail && init_pid(sv, L, A, s.pid, false, s, r)) {
        cont = false;                            // Eq. 2 failed: re-trace from the failing vertex
        trav_begin(t, root);
      } else {
        has_ray = false;
        deposit(s.pid);
      }
      continue;
    }
    ++c_rays;
    if (trace_hit(sv, A, s, r, t, c_photons)) {
      trav_begin(t, root);
    } else {
      has_ray = false;
      deposit(s.pid);
    }
  }
  uint32_t* const ctr[2] = {A.stats ? &A.stats->trace_rays : nullptr, A.stats ? &A.stats->photons_written : nullptr};
  const uint32_t val[2] = {c_rays, c_photons};
  block_add_n<2>(ctr, val, s_red);           // synchronises the block: s_cnt is complete
  if (threadIdx.x == 0 && A.stats) {
    if (s_cnt[0]) atomicAdd(&A.stats->cont_rays, s_cnt[0]);
    if (s_cnt[1]) {                            // the tails join the re-trace list
      atomicAdd(&A.stats->n_tail, s_cnt[1]);
      atomicAdd(&A.stats->n_listed, s_cnt[1]);
    }
    if (s_cnt[2]) atomicAdd(&A.stats->n_updated, s_cnt[2]);
    if (s_cnt[3]) atomicAdd(&A.stats->n_truncated, s_cnt[3]);
  }
  block_add64(A.stats ? (unsigned long long*)&A.stats->node_visits : nullptr, wk.nodes, s_red64);
  block_add64(A.stats ? (unsigned long long*)&A.stats->tri_tests : nullptr, wk.tris, s_red64);
}

}  // namespace

namespace pvh {

namespace {

// persistent blocks of a kernel: its occupancy limit on every SM, or fewer
// when PV_TRACE_BLOCKS_PER_SM asks for fewer (a tuning override)
template <typename K>
int persistent_blocks(const pv_scene* s, K kernel) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kTraceThreads, 0);
  if (const char* e = std::getenv("PV_TRACE_BLOCKS_PER_SM")) {
    const int want = std::atoi(e);
    if (want > 0 && want < per) per = want;
  }
  return (per > 0 ? per : 1) * s->num_sms;
}

TraceArgs trace_args(pv_scene* s, const pv_paths* p, const uint32_t* list, const uint32_t* count, uint64_t seed,
                     uint32_t frame, pv_frame_stats* stats) {
  TraceArgs A;
  A.n = p->n;
  A.info = p->info;
  A.origin = p->origin;
  A.pa = reinterpret_cast<float4*>(p->pa);
  A.pb = reinterpret_cast<float4*>(p->pb);
  A.list = list;
  A.count = count;
  A.ticket = s->ws_ctr + CTR_TRACE;
  A.seed = seed;
  A.frame = frame;
  A.stats = stats;
  return A;
}

}  // namespace

void launch_trace(pv_scene* s, const pv_paths* p, const uint32_t* list, const uint32_t* count, uint64_t seed,
                  uint32_t frame, pv_frame_stats* stats, cudaStream_t st, const pv_atlas* atlas) {
  const TraceArgs A = trace_args(s, p, list, count, seed, frame, stats);
  cudaMemsetAsync(A.ticket, 0, sizeof(uint32_t), st);
  if (!p->n) return;
  AtlasMap am;
  std::memset(&am, 0, sizeof am);
  if (atlas) {
    // the texel scales of atlas_map, in the same IEEE single-precision operations on the host
    am.at = *atlas;
    am.sx = (float)atlas->width / (atlas->x1 - atlas->x0);
    am.sz = (float)atlas->height / (atlas->z1 - atlas->z0);
    if (!s->trace_dep_blocks) s->trace_dep_blocks = persistent_blocks(s, k_trace<true>);
    k_trace<true><<<s->trace_dep_blocks, kTraceThreads, 0, st>>>(view(s), frame_lights(s), A, am);
  } else {
    if (!s->trace_blocks) s->trace_blocks = persistent_blocks(s, k_trace<false>);
    k_trace<false><<<s->trace_blocks, kTraceThreads, 0, st>>>(view(s), frame_lights(s), A, am);
  }
}

// k_cont_trace right after k_verify.  With PV_CONT_TRACE_PDL it is a
// programmatic dependent launch, which may start while k_verify is finishing.
// That made back-to-back frames 3 % slower (villa 1.182 against 1.147 ms per
// frame, city 0.440 against 0.427 ms) with the same time from a frame's first
// launch to its last: the cost fell between frames.  So the launch is an
// ordinary one by default.
#ifndef PV_CONT_TRACE_PDL
#define PV_CONT_TRACE_PDL 0
#endif
template <int kDep>
void launch_cont_trace_pdl(int blocks, const SceneView& sv, const FrameLights& L, const TraceArgs& A,
                           const ContArgs& C, const DepositArgs& D, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kTraceThreads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = PV_CONT_TRACE_PDL;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_cont_trace<kDep>, sv, L, A, C, D);
}

void launch_cont_trace(pv_scene* s, const pv_paths* p, const ContArgs& C, const uint32_t* list, const uint32_t* count,
                       uint64_t seed, uint32_t frame, pv_frame_stats* stats, const pv_atlas* atlas,
                       const uint8_t* touched, bool delta, cudaStream_t st) {
  // the ticket was cleared with the other work counters before k_verify
  const TraceArgs A = trace_args(s, p, list, count, seed, frame, stats);
  if (!p->n) return;
  DepositArgs D;
  std::memset(&D, 0, sizeof D);
  if (atlas) {
    D.at = *atlas;
    D.touched = touched;
    if (delta) {
      if (!s->cont_trace_delta_blocks) s->cont_trace_delta_blocks = persistent_blocks(s, k_cont_trace<2>);
      launch_cont_trace_pdl<2>(s->cont_trace_delta_blocks, view(s), frame_lights(s), A, C, D, st);
    } else {
      if (!s->cont_trace_dep_blocks) s->cont_trace_dep_blocks = persistent_blocks(s, k_cont_trace<1>);
      launch_cont_trace_pdl<1>(s->cont_trace_dep_blocks, view(s), frame_lights(s), A, C, D, st);
    }
  } else {
    if (!s->cont_trace_blocks) s->cont_trace_blocks = persistent_blocks(s, k_cont_trace<0>);
    launch_cont_trace_pdl<0>(s->cont_trace_blocks, view(s), frame_lights(s), A, C, D, st);
  }
}

}  // namespace pvh

extern "C" int pv_retrace_invalid(pv_scene* s, const pv_paths* paths, const uint32_t* d_list, const uint32_t* d_count,
                                  uint64_t seed, uint32_t frame, pv_frame_stats* d_stats, void* stream) {
  const int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!d_list || !d_count) return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  pvh::launch_trace(s, paths, d_list, d_count, seed, frame, d_stats, st);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

extern "C" int pv_trace_all(pv_scene* s, const pv_paths* paths, uint64_t seed, uint32_t frame, pv_frame_stats* d_stats,
                            void* stream) {
  const int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  pvh::launch_trace(s, paths, nullptr, nullptr, seed, frame, d_stats, st);
  if (s->has_dm) pvh::dm_reset(s, st);            // a full trace is stratified: DM_C = DM_T
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

extern "C" int pv_trace_all_deposit(pv_scene* s, const pv_paths* paths, uint64_t seed, uint32_t frame,
                                    const pv_atlas* atlas, pv_frame_stats* d_stats, void* stream) {
  int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if ((rc = pvh::check_atlas(atlas)) != PV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (cudaMemsetAsync(atlas->data, 0, (size_t)atlas->width * atlas->height * 3 * sizeof(uint64_t), st) != cudaSuccess)
    return PV_ERR_CUDA;
  pvh::launch_trace(s, paths, nullptr, nullptr, seed, frame, d_stats, st, atlas);
  if (s->has_dm) pvh::dm_reset(s, st);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
