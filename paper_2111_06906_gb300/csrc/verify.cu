// Per-frame verification of stored photon paths.
//
// k_verify_box / k_verify (resident blocks looping over tiles of paths,
// streaming the 2-D photon array row by row): Sec. 3.1 "update path
// origins" fused with Sec. 3.2 "dynamic occlusions" as in Sec. 4 (origins
// first, then the segment tests).
// k_continue (persistent, over the paths k_verify flagged in error mode):
//   the error-based threshold continuation of Sec. 3.3, Alg. 1 and Eq. 2.
// Then the replace bits are compacted into the re-trace list (compact.cu).
#include <algorithm>
#include <cstring>

#include "verify_core.cuh"

using namespace pvk;

namespace {

// PV_VERIFY_FLAT: error mode deals the warp's segments out to its lanes
// (verify_block_flat); 0 keeps thread per path throughout.
// PV_VERIFY_PERSISTENT: each block loops over tiles of paths, so the block
// prologue and the counter reductions run once per block.
#ifndef PV_VERIFY_FLAT
#define PV_VERIFY_FLAT 1
#endif
#ifndef PV_VERIFY_PERSISTENT
#define PV_VERIFY_PERSISTENT 1
#endif
// Resident blocks asked of the register allocator for the box-only kernel:
// 5 (51 registers) beat the 4 that 56 registers allow by 7 % on the villa
// workload.  The variants with traversal code keep their registers (they
// would spill).
#ifndef PV_VERIFY_MIN_BLOCKS
#define PV_VERIFY_MIN_BLOCKS 5
#endif
constexpr bool kVerifyLoop = PV_VERIFY_FLAT && PV_VERIFY_PERSISTENT;

// Flat segment mapping in error mode, else thread per path; with
// kVerifyLoop a grid of resident blocks looping over tiles.  A re-trace kernel launched as its
// programmatic dependent (PV_CONT_TRACE_PDL) may be scheduled as soon as every block has started.
template <bool kPointVis, bool kExact>
__device__ __forceinline__ void verify_kernel(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                              VerifySmem& sm) {
  launch_dependents();
  const bool flat = PV_VERIFY_FLAT && A.mode == PV_MODE_ERROR;
  if (kVerifyLoop) {
    if (flat) verify_tiles<kPointVis, kExact, 2>(sv, L, A, blockIdx.x, gridDim.x, sm);
    else verify_tiles<kPointVis, kExact, 0>(sv, L, A, blockIdx.x, gridDim.x, sm);
  } else {
    if (flat) verify_block_flat<kPointVis, kExact>(sv, L, A, blockIdx.x * blockDim.x + threadIdx.x, sm);
    else verify_block<kPointVis, kExact>(sv, L, A, blockIdx.x * blockDim.x + threadIdx.x, sm);
  }
}

// With visibility rays or triangle tests (traversal code inside).
template <bool kPointVis, bool kExact>
__global__ void __launch_bounds__(pvh::kVerifyThreads) k_verify(SceneView sv, FrameLights L, VerifyArgs A) {
  __shared__ VerifySmem sm;
  verify_kernel<kPointVis, kExact>(sv, L, A, sm);
}

// Box tests only, the common case.
__global__ void __launch_bounds__(pvh::kVerifyThreads, PV_VERIFY_MIN_BLOCKS) k_verify_box(SceneView sv, FrameLights L,
                                                                                         VerifyArgs A) {
  __shared__ VerifySmem sm;
  verify_kernel<false, false>(sv, L, A, sm);
}

// Blocks of a k_verify kernel for n paths: every tile, or with the tile
// loop at most the resident blocks of all SMs (fewer when PV_VERIFY_MAX_BLOCKS
// asks for fewer: a testing and tuning override).
template <typename K>
uint32_t verify_grid(pv_scene* s, K kernel, int& per, uint32_t n) {
  const uint32_t tiles = (n + pvh::kVerifyThreads - 1) / pvh::kVerifyThreads;
  if (!kVerifyLoop) return tiles;
  if (!per) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, pvh::kVerifyThreads, 0);
    if (per < 1) per = 1;
  }
  return std::min<uint32_t>(tiles, pvh::verify_block_cap((uint32_t)per * (uint32_t)s->num_sms));
}

template <bool kPointVis, bool kExact>
void launch_k_verify(pv_scene* s, const SceneView& sv, const FrameLights& L, const VerifyArgs& A, cudaStream_t st) {
  int& per = s->verify_blocks_per_sm[(kPointVis ? 2 : 0) + (kExact ? 1 : 0)];
  if (!kPointVis && !kExact) {
    const uint32_t grid = verify_grid(s, k_verify_box, per, A.n);
    k_verify_box<<<grid, pvh::kVerifyThreads, 0, st>>>(sv, L, A);
  } else {
    const uint32_t grid = verify_grid(s, k_verify<kPointVis, kExact>, per, A.n);
    k_verify<kPointVis, kExact><<<grid, pvh::kVerifyThreads, 0, st>>>(sv, L, A);
  }
}

__global__ void __launch_bounds__(128, 6) k_continue(SceneView sv, ContArgs A) {
  __shared__ uint32_t s_red[32 * 4];
  __shared__ unsigned long long s_red64[32];
  const int root = *sv.root;
  const uint32_t total = *A.count;
  const int lane = threadIdx.x & 31;
  ContCounters cc;
  Work wk;
  for (uint32_t guard = 0; guard < (1u << 26); ++guard) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(A.ticket, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= total) break;
    const uint32_t i = base + lane;
    if (i < total) continue_path(sv, root, A, A.list[i], cc, wk);
    __syncwarp();
  }
  uint32_t* const ctr[4] = {A.stats ? &A.stats->cont_rays : nullptr, A.stats ? &A.stats->n_tail : nullptr,
                            A.stats ? &A.stats->n_updated : nullptr, A.stats ? &A.stats->n_truncated : nullptr};
  const uint32_t val[4] = {cc.rays, cc.tail, cc.upd, cc.trunc};
  block_add_n<4>(ctr, val, s_red);
  block_add64(A.stats ? (unsigned long long*)&A.stats->node_visits : nullptr, wk.nodes, s_red64);
  block_add64(A.stats ? (unsigned long long*)&A.stats->tri_tests : nullptr, wk.tris, s_red64);
}

}  // namespace

namespace pvh {
int check_paths(const pv_scene* s, const pv_paths* p) {
  if (!s || !p || !p->info || !p->origin || !p->pa || !p->pb) return PV_ERR_ARG;
  if (p->n != s->n_paths_total || p->max_bounces != s->B) return PV_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(p->pa) | reinterpret_cast<uintptr_t>(p->pb)) & 15u) return PV_ERR_ARG;
  return PV_OK;
}
}  // namespace pvh

namespace {

int check_verify(const pv_scene* s, const pv_paths* paths, const pv_verify_params* params) {
  const int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!params) return PV_ERR_ARG;
  if (params->mode < PV_MODE_NAIVE_AABB || params->mode > PV_MODE_ERROR || !(params->tau >= 0.0f)) return PV_ERR_ARG;
  return PV_OK;
}

ContArgs cont_args(pv_scene* s, const pv_paths* paths, const pv_verify_params* params, pv_frame_stats* d_stats) {
  ContArgs C;
  C.n = paths->n;
  C.info = paths->info;
  C.origin = paths->origin;
  C.pa = reinterpret_cast<float4*>(paths->pa);
  C.pb = reinterpret_cast<const float4*>(paths->pb);
  C.mask = s->ws_mask;
  C.list = s->ws_cont;
  C.count = s->ws_ctr + pvh::CTR_ALL;
  C.ticket = s->ws_ctr + pvh::CTR_CONT;
  C.tau = params->tau;
  C.stats = d_stats;
  return C;
}

// Work counters reset, DM_C of moved lights with a map cleared, then k_verify
// (Sec. 3.1 + 3.2).  ``cont``: Alg. 1 has paths to look at this frame.
template <typename OnCleared = void (*)()>
int launch_verify(pv_scene* s, const pv_paths* paths, const pv_verify_params* params, pv_frame_stats* d_stats,
                  const SceneView& sv, const FrameLights& L, cudaStream_t st, bool& cont, uint8_t* touched = nullptr,
                  bool direct_list = false, const pv_atlas* sub = nullptr, OnCleared on_cleared = [] {}) {
  const uint32_t n = paths->n;
  if (cudaMemsetAsync(s->ws_ctr, 0, 16 * sizeof(uint32_t), st) != cudaSuccess) return PV_ERR_CUDA;
  for (uint32_t l = 0; l < s->n_lights; ++l)       // DM_C of moved lights with a map is counted afresh
    if (L.dm[l].dims && ((L.moved_mask >> l) & 1u))
      if (cudaMemsetAsync(L.dm[l].dmc, 0, (size_t)L.dm[l].cells * sizeof(uint32_t), st) != cudaSuccess)
        return PV_ERR_CUDA;
  on_cleared();
  VerifyArgs A;
  A.n = n;
  A.info = paths->info;
  A.origin = paths->origin;
  A.pa = reinterpret_cast<float4*>(paths->pa);
  A.pb = reinterpret_cast<const float4*>(paths->pb);
  A.mode = params->mode;
  A.tau = params->tau;
  A.flags = params->flags;
  A.mask_out = s->ws_mask;
  A.cont_list = s->ws_cont;
  A.cont_count = s->ws_ctr + pvh::CTR_ALL;
  A.stats = d_stats;
  A.touched = touched;
  std::memset(&A.sub, 0, sizeof A.sub);
  if (sub && touched) A.sub = *sub;             // a carried atlas: touched paths' entry photons leave it here
  A.list_out = direct_list ? s->ws_list : nullptr;           // the marked paths, appended (no compaction)
  A.list_count = direct_list ? s->ws_ctr + pvh::CTR_LIST : nullptr;
  if (n) {
    bool point_vis = false;
    for (uint32_t l = 0; l < s->n_lights; ++l)
      if (((L.moved_mask >> l) & 1u) && s->lights_new[l].type == PV_LIGHT_POINT) point_vis = true;
    const bool exact = params->mode == PV_MODE_NAIVE_EXACT ||
                       (params->mode == PV_MODE_ERROR && (params->flags & PV_FLAG_ERROR_EXACT));
    if (point_vis && exact) launch_k_verify<true, true>(s, sv, L, A, st);
    else if (point_vis) launch_k_verify<true, false>(s, sv, L, A, st);
    else if (exact) launch_k_verify<false, true>(s, sv, L, A, st);
    else launch_k_verify<false, false>(s, sv, L, A, st);
  }
  cont = n && params->mode == PV_MODE_ERROR && (s->moved || L.moved_mask);
  return PV_OK;
}

void launch_continue(pv_scene* s, const SceneView& sv, const ContArgs& C, cudaStream_t st) {
  if (!s->cont_blocks) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_continue, 128, 0);
    s->cont_blocks = (per > 0 ? per : 1) * s->num_sms;
  }
  k_continue<<<s->cont_blocks, 128, 0, st>>>(sv, C);
}

}  // namespace

extern "C" int pv_verify_paths(pv_scene* s, const pv_paths* paths, const pv_verify_params* params, uint32_t* d_list,
                               uint32_t* d_count, pv_frame_stats* d_stats, void* stream) {
  int rc = check_verify(s, paths, params);
  if (rc != PV_OK) return rc;
  if (!d_list || !d_count) return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  const SceneView sv = pvh::view(s);
  const FrameLights L = pvh::frame_lights(s);
  bool cont = false;
  if ((rc = launch_verify(s, paths, params, d_stats, sv, L, st, cont)) != PV_OK) return rc;
  if (cont) launch_continue(s, sv, cont_args(s, paths, params, d_stats), st);
  if (s->has_dm && (rc = pvh::dm_frame(s, paths, L, params, d_stats, st)) != PV_OK) return rc;
  pvh::launch_compact(s, paths->info, paths->n, d_list, d_count, d_stats ? &d_stats->n_listed : nullptr, st);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

namespace {

// pv_verify_retrace, and with an atlas pv_verify_retrace_deposit.
int verify_retrace(pv_scene* s, const pv_paths* paths, const pv_verify_params* params, const pv_atlas* atlas,
                   bool delta, pv_frame_stats* d_stats, cudaStream_t st) {
  int rc = check_verify(s, paths, params);
  if (rc != PV_OK) return rc;
  if (atlas && (rc = pvh::check_atlas(atlas)) != PV_OK) return rc;
  s->last_stream = st;
  const SceneView sv = pvh::view(s);
  const FrameLights L = pvh::frame_lights(s);
  cudaEvent_t* ev = s->stage_n ? &s->stage_ev[pvh::kStageEvents * s->stage_next] : nullptr;
  auto mark = [&](int k) {
    if (ev) cudaEventRecord(ev[k], st);
  };
  mark(0);
  // with maps the deposit runs as its own kernel over every path: the delta form starts from a cleared atlas too
  if (s->has_dm) delta = false;
  // with maps, prune and fill need Alg. 1's final answer for every path before the list is made
  const bool fuse_deposit = atlas && !s->has_dm;
  const bool will_cont = paths->n && params->mode == PV_MODE_ERROR && (s->moved || L.moved_mask);
  const bool fused = (will_cont || fuse_deposit) && !s->has_dm;
  if (atlas && !delta &&
      cudaMemsetAsync(atlas->data, 0, (size_t)atlas->width * atlas->height * 3 * sizeof(uint64_t), st) != cudaSuccess)
    return PV_ERR_CUDA;
  bool cont = false;
  if ((rc = launch_verify(s, paths, params, d_stats, sv, L, st, cont, fuse_deposit ? s->ws_touched : nullptr, fused,
                          delta ? atlas : nullptr, [&] { mark(1); })) != PV_OK)
    return rc;
  mark(2);
  const ContArgs C = cont_args(s, paths, params, d_stats);
  uint32_t* const list = s->ws_list;
  uint32_t* const count = s->ws_ctr + pvh::CTR_LIST;
  uint32_t* const listed = d_stats ? &d_stats->n_listed : nullptr;
  if (fused) {
    // k_verify appended the paths it marked; then Alg. 1, the re-trace (and the deposit) in one kernel
    mark(3);
    pvh::launch_cont_trace(s, paths, C, list, count, params->seed, params->frame, d_stats,
                           fuse_deposit ? atlas : nullptr, s->ws_touched, delta, st);
  } else {
    if (cont) launch_continue(s, sv, C, st);
    if (s->has_dm && (rc = pvh::dm_frame(s, paths, L, params, d_stats, st)) != PV_OK) return rc;
    pvh::launch_compact(s, paths->info, paths->n, list, count, listed, st);
    mark(3);
    pvh::launch_trace(s, paths, list, count, params->seed, params->frame, d_stats, st);
    if (atlas) pvh::launch_deposit(s, paths, atlas, st);
  }
  mark(4);
  if (ev) {
    s->stage_next = (s->stage_next + 1) % s->stage_n;
    s->stage_count = std::min(s->stage_count + 1, s->stage_n);
  }
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

}  // namespace

extern "C" int pv_verify_retrace(pv_scene* s, const pv_paths* paths, const pv_verify_params* params,
                                 pv_frame_stats* d_stats, void* stream) {
  return verify_retrace(s, paths, params, nullptr, false, d_stats, (cudaStream_t)stream);
}

extern "C" int pv_verify_retrace_deposit(pv_scene* s, const pv_paths* paths, const pv_verify_params* params,
                                         const pv_atlas* atlas, pv_frame_stats* d_stats, void* stream) {
  if (!atlas) return PV_ERR_ARG;
  return verify_retrace(s, paths, params, atlas, false, d_stats, (cudaStream_t)stream);
}

extern "C" int pv_verify_retrace_deposit_delta(pv_scene* s, const pv_paths* paths, const pv_verify_params* params,
                                               const pv_atlas* atlas, pv_frame_stats* d_stats, void* stream) {
  if (!atlas) return PV_ERR_ARG;
  return verify_retrace(s, paths, params, atlas, true, d_stats, (cudaStream_t)stream);
}

extern "C" int pv_stage_timing(pv_scene* s, uint32_t n) {
  if (!s || n > 4096) return PV_ERR_ARG;
  if (s->last_stream && cudaStreamSynchronize(s->last_stream) != cudaSuccess) return PV_ERR_CUDA;
  for (cudaEvent_t e : s->stage_ev)
    if (e) cudaEventDestroy(e);
  s->stage_ev.assign(pvh::kStageEvents * (size_t)n, nullptr);
  s->stage_n = s->stage_next = s->stage_count = 0;
  for (auto& e : s->stage_ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
      return PV_ERR_CUDA;
    }
  s->stage_n = n;
  return PV_OK;
}

extern "C" int pv_stage_times(pv_scene* s, float* ms, uint32_t* count) {
  if (!s || !ms || !count) return PV_ERR_ARG;
  const uint32_t c = s->stage_count;
  for (uint32_t i = 0; i < c; ++i) {
    constexpr int E = pvh::kStageEvents;
    const uint32_t k = (s->stage_next + s->stage_n - c + i) % s->stage_n;
    cudaEvent_t* ev = &s->stage_ev[E * k];
    if (cudaEventSynchronize(ev[E - 1]) != cudaSuccess) return PV_ERR_CUDA;
    for (int j = 0; j < E - 1; ++j)
      if (cudaEventElapsedTime(ms + E * i + j, ev[j], ev[j + 1]) != cudaSuccess) return PV_ERR_CUDA;
    if (cudaEventElapsedTime(ms + E * i + E - 1, ev[0], ev[E - 1]) != cudaSuccess) return PV_ERR_CUDA;
  }
  *count = c;
  return PV_OK;
}
