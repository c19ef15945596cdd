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

#include "pv_scene.h"

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

struct TraceArgs {
  uint32_t n;
  uint32_t* info;
  float* origin;
  float4* pa;
  float4* pb;
  const uint32_t* list;     // nullptr: every path from the light (trace-all)
  const uint32_t* count;
  uint32_t* ticket;
  uint64_t seed;
  uint32_t frame;
  pv_frame_stats* stats;
};

struct PathState {
  uint32_t pid, k, cell;
  float3 E;
  float radius;
  int excl;
};

// Russian roulette (q = max albedo) and a cosine-weighted bounce about the
// facing normal at photon s.k; E_{k+1} = E_k * albedo / q.  Sets the next ray.
__device__ __forceinline__ bool scatter(const SceneView& sv, const TraceArgs& A, PathState& s, Ray& r, float3 x,
                                        int prim, float3 nrm, float3 d_in, float3 Ek, float radius) {
  const float4 u = rng4(A.seed, s.pid, s.k, A.frame);
  const float4 alb = __ldg(sv.prim_alb + prim);
  if (!(u.z < alb.w)) return false;
  const float3 nn = normalize(nrm);
  const float3 ns = dot(nn, d_in) < 0.0f ? nn : -1.0f * nn;
  float3 b1, b2;
  onb(ns, b1, b2);
  r = make_ray(x, cosine_dir(ns, b1, b2, u.x, u.y), sv.tmin);
  s.E = make_float3(Ek.x * alb.x / alb.w, Ek.y * alb.y / alb.w, Ek.z * alb.z / alb.w);
  s.excl = prim;
  s.radius = radius;
  return true;
}

__device__ __forceinline__ void finish(const TraceArgs& A, const PathState& s) {
  A.info[s.pid] = info_make(s.cell, s.k, 0, false, false);
}

__device__ __forceinline__ float3 load_origin(const TraceArgs& A, uint32_t p) {
  return make_float3(A.origin[p], A.origin[A.n + p], A.origin[2 * (size_t)A.n + p]);
}

// Set up the first ray of list entry idx; false if the path ends at once.
__device__ bool init_path(const SceneView& sv, const FrameLights& L, const TraceArgs& A, uint32_t idx, PathState& s,
                          Ray& r) {
  const bool all = A.list == nullptr;
  const uint32_t pid = all ? idx : A.list[idx];
  const uint32_t n = A.n;
  s.pid = pid;
  const uint32_t w = all ? 0u : A.info[pid];
  uint32_t l = 0;
  if (all) {
    while (l + 1 < L.n && pid >= L.first[l + 1]) ++l;
    s.cell = l << 20;
  } else {
    l = info_light(w);
    s.cell = w & PV_INFO_CELL_MASK;
  }
  const uint32_t start = all ? 0u : info_start(w);
  if (start == 0) {
    s.k = 0;
    s.radius = 0.0f;
    s.excl = -1;
    if (!all && (w & PV_INFO_REUSE_LIGHT)) {     // same light sample and direction
      const float3 o = load_origin(A, pid);
      r = make_ray(o, normalize_exact(f3(A.pa[pid]) - o), sv.tmin);
      s.E = f3(A.pb[pid]);
    } else {                                     // fresh emission
      const LightPose& Lp = L.cur[l];
      float3 o, d;
      emit(Lp, rng4(A.seed, pid, 0, A.frame), o, d);
      A.origin[pid] = o.x;
      A.origin[n + pid] = o.y;
      A.origin[2 * (size_t)n + pid] = o.z;
      r = make_ray(o, d, sv.tmin);
      const float np = (float)Lp.n_paths;
      s.E = make_float3(Lp.power.x / np, Lp.power.y / np, Lp.power.z / np);
    }
    return true;
  }
  s.k = start;
  if (start >= sv.B) {
    finish(A, s);
    return false;
  }
  const float4 v = A.pa[(size_t)(start - 1) * n + pid];
  const float4 e = A.pb[(size_t)(start - 1) * n + pid];
  const float3 xprev = start >= 2 ? f3(A.pa[(size_t)(start - 2) * n + pid]) : load_origin(A, pid);
  const int prim = __float_as_int(v.w);
  if (!scatter(sv, A, s, r, f3(v), prim, prim_normal(sv, prim, false), normalize_exact(f3(v) - xprev), f3(e), e.w)) {
    finish(A, s);
    return false;
  }
  return true;
}

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
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
