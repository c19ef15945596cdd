// Device code of path (re-)tracing shared by the single-scene persistent
// kernel (trace.cu) and the batched one (batch.cu): ray generation where the
// paper generates rays (Sec. 4), from the light (start 0) or by Russian
// roulette and a cosine-weighted bounce at the first photon to re-trace.
#pragma once
#include "deposit_core.cuh"
#include "dm_core.cuh"
#include "pv_scene.h"

namespace pvk {

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

// Set up the first ray of path pid (``all``: a full trace from the light,
// else a re-trace as its info word says); false if the path ends at once.
__device__ __forceinline__ bool init_pid(const SceneView& sv, const FrameLights& L, const TraceArgs& A, uint32_t pid,
                                         bool all, PathState& s, Ray& r) {
  const uint32_t n = A.n;
  s.pid = pid;
  const uint32_t w = all ? 0u : A.info[pid];
  uint32_t l = 0;
  if (all) {
    while (l + 1 < L.n && pid >= L.first[l + 1]) ++l;
    // a full trace is stratified over the light's distribution map (DM_C = DM_T)
    s.cell = (l << 20) | (L.dm[l].dims ? dm_stratified(L.dm[l], pid - L.first[l]) : 0u);
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
    } else {                                     // fresh emission, inside the path's cell if the light has a map
      const LightPose& Lp = L.cur[l];
      float3 o, d;
      float4 u = rng4(A.seed, pid, 0, A.frame);
      if (L.dm[l].dims) dm_restrict(L.dm[l], s.cell & 0xFFFFFu, u);
      emit(Lp, u, o, d);
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

// Set up the first ray of list entry idx; false if the path ends at once.
__device__ __forceinline__ bool init_path(const SceneView& sv, const FrameLights& L, const TraceArgs& A, uint32_t idx,
                                          PathState& s, Ray& r) {
  const bool all = A.list == nullptr;
  return init_pid(sv, L, A, all ? idx : A.list[idx], all, s, r);
}

// The ray of path s ended (hit t.best at t.tbest, or escaped): store its
// photon (with kDep, also deposit it into am's atlas) and set up the next
// bounce.  False once the path is finished (its info word written).
template <bool kDep = false>
__device__ __forceinline__ bool trace_hit(const SceneView& sv, const TraceArgs& A, PathState& s, Ray& r, const Trav& t,
                                          uint32_t& c_photons, const AtlasMap* am = nullptr) {
  if (t.best < 0) {                          // escaped: the path ends
    finish(A, s);
    return false;
  }
  const Tri T = load_tri(sv.tris, t.best);
  const int prim = __float_as_int(T.v0.w);
  const float3 x = make_float3(fmaf(t.tbest, r.d.x, r.o.x), fmaf(t.tbest, r.d.y, r.o.y), fmaf(t.tbest, r.d.z, r.o.z));
  const float rad = s.radius + t.tbest;
  const uint32_t n = A.n;
  A.pa[(size_t)s.k * n + s.pid] = make_float4(x.x, x.y, x.z, __int_as_float(prim));
  A.pb[(size_t)s.k * n + s.pid] = make_float4(s.E.x, s.E.y, s.E.z, rad);
  if (kDep) deposit_point(*am, x, s.E);
  ++s.k;
  ++c_photons;
  if (s.k >= sv.B || !scatter(sv, A, s, r, x, prim, cross(f3(T.e1), f3(T.e2)), r.d, s.E, rad)) {
    finish(A, s);
    return false;
  }
  return true;
}

// Advance every lane's ray until all rays of the warp have ended, or for at
// most kMax steps; called by all lanes of the warp (a lane without a ray
// passes done = true).  Returns whether this lane's ray has ended.  Waiting
// for the whole warp lets the ray-end code that follows run with all lanes.
template <int kMax, int S = kStack, class Stk>
__device__ __forceinline__ bool step_warp(const SceneView& sv, const Ray& r, Trav& t, Stk& stk, int excl, Work& wk,
                                          bool done, const WNode* cache = nullptr, int n_cache = 0) {
#pragma unroll 1
  for (int i = 0; i < kMax; ++i) {
    if (!done) done = trav_step<S>(sv, r, t, stk, excl, wk, cache, n_cache);
    if (__all_sync(0xffffffffu, done)) break;
  }
  return done;
}

}  // namespace pvk
