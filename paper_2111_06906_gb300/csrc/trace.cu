// Persistent re-trace of the listed paths (and the trace-all baseline).
//
// "Generate rays" and "trace rays" of Fig. 2 fused into one kernel.  Each
// lane owns one path and one ray at a time and advances its traversal a few
// steps per loop iteration; as soon as a lane's ray is done it stores the
// photon and starts its next ray (the next bounce, or the next list entry,
// taken with one atomic per warp), so lanes never wait for the slowest ray
// of the warp.  Rays are generated where the paper generates them (Sec. 4):
// from the light (start 0), or by Russian roulette and a cosine-weighted
// bounce at the first photon to re-trace.
#include <cstdlib>

#include "trace_core.cuh"

using namespace pvk;

namespace {

// compile-time tuning: traversal steps between refills, minimum resident blocks
#ifndef PV_TRACE_STEPS
#define PV_TRACE_STEPS 8
#endif
#ifndef PV_TRACE_MIN_BLOCKS
#define PV_TRACE_MIN_BLOCKS 7
#endif
constexpr int kStepsPerIter = PV_TRACE_STEPS;

__global__ void __launch_bounds__(pvh::kTraceThreads, PV_TRACE_MIN_BLOCKS) k_trace(SceneView sv, FrameLights L, TraceArgs A) {
  __shared__ uint32_t s_red[32 * 2];
  __shared__ unsigned long long s_red64[32];
  const int root = *sv.root;
  const uint32_t total = A.list ? *A.count : A.n;
  const uint32_t n = A.n;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  Work wk;
  PathState s;
  Ray r;
  Trav t;
  int stk[kStack];
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
    if (!has_ray) continue;
    bool done = false;
#pragma unroll 1
    for (int i = 0; i < kStepsPerIter && !done; ++i) done = trav_step(sv, r, t, stk, s.excl, wk);
    if (!done) continue;
    ++c_rays;
    if (t.best < 0) {                         // escaped: the path ends
      finish(A, s);
      has_ray = false;
      continue;
    }
    const Tri T = load_tri(sv.tris, t.best);
    const int prim = __float_as_int(T.v0.w);
    const float3 x = make_float3(fmaf(t.tbest, r.d.x, r.o.x), fmaf(t.tbest, r.d.y, r.o.y), fmaf(t.tbest, r.d.z, r.o.z));
    const float rad = s.radius + t.tbest;
    A.pa[(size_t)s.k * n + s.pid] = make_float4(x.x, x.y, x.z, __int_as_float(prim));
    A.pb[(size_t)s.k * n + s.pid] = make_float4(s.E.x, s.E.y, s.E.z, rad);
    ++s.k;
    ++c_photons;
    if (s.k >= sv.B || !scatter(sv, A, s, r, x, prim, cross(f3(T.e1), f3(T.e2)), r.d, s.E, rad)) {
      finish(A, s);
      has_ray = false;
    } else {
      trav_begin(t, root);
    }
  }
  uint32_t* const ctr[2] = {A.stats ? &A.stats->trace_rays : nullptr, A.stats ? &A.stats->photons_written : nullptr};
  const uint32_t val[2] = {c_rays, c_photons};
  block_add_n<2>(ctr, val, s_red);
  block_add64(A.stats ? (unsigned long long*)&A.stats->node_visits : nullptr, wk.nodes, s_red64);
  block_add64(A.stats ? (unsigned long long*)&A.stats->tri_tests : nullptr, wk.tris, s_red64);
}

}  // namespace

namespace pvh {

void launch_trace(pv_scene* s, const pv_paths* p, const uint32_t* list, const uint32_t* count, uint64_t seed,
                  uint32_t frame, pv_frame_stats* stats, cudaStream_t st) {
  if (!s->trace_blocks) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace, kTraceThreads, 0);
    // tuning override: persistent blocks per SM (at most the occupancy limit)
    if (const char* e = std::getenv("PV_TRACE_BLOCKS_PER_SM")) {
      const int want = std::atoi(e);
      if (want > 0 && want < per) per = want;
    }
    s->trace_blocks = (per > 0 ? per : 1) * s->num_sms;
  }
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
  cudaMemsetAsync(A.ticket, 0, sizeof(uint32_t), st);
  if (p->n) k_trace<<<s->trace_blocks, kTraceThreads, 0, st>>>(view(s), frame_lights(s), A);
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
