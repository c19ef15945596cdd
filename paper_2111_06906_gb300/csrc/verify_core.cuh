// Device code of path verification shared by the single-scene kernels
// (verify.cu) and the batched kernels (batch.cu).
//
// verify_tile_thread / _warp / _flat: Sec. 3.1 "update path origins" fused
//   with Sec. 3.2 "dynamic occlusions" as in Sec. 4 (origins first, then the
//   segment tests) for one tile of paths, thread per path, warp per path or
//   with the warp's segments dealt out to its lanes; verify_tiles loops a
//   block over tiles, verify_block* runs one tile as a whole block.
// continue_path: the error-based threshold continuation of Sec. 3.3, Alg. 1
//   and Eq. 2, for one path flagged by the verification in error mode.
#pragma once
#include "deposit_core.cuh"
#include "dm_core.cuh"
#include "pv_scene.h"

namespace pvk {

struct VerifyArgs {
  uint32_t n;
  uint32_t* info;
  float* origin;
  float4* pa;
  const float4* pb;
  int32_t mode;
  float tau;
  uint32_t flags;
  uint32_t* mask_out;
  uint32_t* cont_list;
  uint32_t* cont_count;
  pv_frame_stats* stats;
  uint8_t* touched;            // optional [n]: 0 for a path this frame leaves as it is; for one it re-traces or
                               // hands to Alg. 1, 1 + the photon count it had on entry (at most 16)
  pv_atlas sub;                // optional (sub.data non-null, with touched): a carried atlas from which each
                               // touched path's entry photons are subtracted here, before anything rewrites them
  uint32_t* list_out;          // optional: the paths marked for re-tracing are appended here (unordered),
  uint32_t* list_count;        // counted here and in stats->n_listed (instead of a compaction)
};

// Closed segment a + s (b - a), s in [0,1], against a closed box: slab test
// with the reciprocal direction precomputed (a component below 1e-20 gets the
// reciprocal 1e20 of its sign, which keeps the axis' interval around [0,1]
// when a lies inside the slab and away from it when a lies outside; only a
// segment lying exactly in a face plane can be decided differently).
__device__ __forceinline__ bool seg_box(float3 inv, float3 aoi, const float* bx) {
  const float x0 = fmaf(bx[0], inv.x, aoi.x), x1 = fmaf(bx[3], inv.x, aoi.x);
  const float y0 = fmaf(bx[1], inv.y, aoi.y), y1 = fmaf(bx[4], inv.y, aoi.y);
  const float z0 = fmaf(bx[2], inv.z, aoi.z), z1 = fmaf(bx[5], inv.z, aoi.z);
  const float t0 = fmax3(fminf(x0, x1), fminf(y0, y1), fmaxf(fminf(z0, z1), 0.0f));
  const float t1 = fmin3(fmaxf(x0, x1), fmaxf(y0, y1), fminf(fmaxf(z0, z1), 1.0f));
  return t0 <= t1;
}

// Segment a->b prepared once for all moved-object tests of it.
struct Seg {
  float3 inv, aoi;     // box tests: reciprocal direction, -a * inv
  Ray r;               // exact tests: unit ray from a, open interval (tmin, tmax)
  float tmax;
  bool ok;             // exact tests: the segment is longer than 2 tmin
};

__device__ __forceinline__ Seg seg_prep(const SceneView& sv, float3 a, float3 b, bool boxes) {
  Seg g;
  const float3 dv = b - a;
  if (boxes) {
    // |1/d| <= 1e20 keeps a * inv finite for any scene size.  An approximate reciprocal (one special-function
    // instruction, not the correctly rounded division) suffices: its error moves the slab bounds by a few
    // units in the last place, far inside the band within which a box decision counts as ambiguous
    const float e = 1e-20f;
    g.inv = make_float3(__fdividef(1.0f, fabsf(dv.x) > e ? dv.x : copysignf(e, dv.x)),
                        __fdividef(1.0f, fabsf(dv.y) > e ? dv.y : copysignf(e, dv.y)),
                        __fdividef(1.0f, fabsf(dv.z) > e ? dv.z : copysignf(e, dv.z)));
    g.aoi = make_float3(-a.x * g.inv.x, -a.y * g.inv.y, -a.z * g.inv.z);
    g.ok = true;
    return g;
  }
  const float len = sqrtf(dot(dv, dv));
  g.ok = len > 0.0f;
  if (!g.ok) return g;
  const float3 d = make_float3(dv.x / len, dv.y / len, dv.z / len);
  g.r = make_ray(a, d, sv.tmin);
  g.tmax = len - sv.tmin;
  g.ok = g.tmax > sv.tmin;
  return g;
}

// The prepared segment against moved object s: box test (old u new tight
// box) or exact any-hit over the object's triangles at the new pose (and the
// old pose with PV_FLAG_TEST_OLD_TRIS, by brute force over object-local
// corners).
template <int S = kStack>
__device__ __forceinline__ bool seg_vs_object(const SceneView& sv, const Seg& g, const float* cull, const float* uni,
                                              bool boxes, bool test_old, int s, Work& wk) {
  if (boxes) return seg_box(g.inv, g.aoi, uni + 6 * s);
  if (!g.ok) return false;
  float te;
  if (sv.objs[s].wroot != INT32_MIN && box1(g.r, g.tmax, cull + 6 * s, te)) {
    float tb = g.tmax;
    int best = -1;
    traverse<true, S>(sv.nodes, sv.tris, sv.objs[s].wroot, g.r, tb, best, -1, sv.max_visits, sv.status, wk);
    if (best >= 0) return true;
  }
  if (test_old) {
    const float* x = sv.xf_old + 12 * s;
    const uint32_t b0 = sv.objs[s].tri_begin, e0 = b0 + sv.objs[s].tri_count;
    for (uint32_t i = b0; i < e0; ++i) {
      const float* v = sv.d_local + 9 * (size_t)i;
      float w[9];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
          w[3 * k + rr] = fmaf(x[4 * rr], v[3 * k], fmaf(x[4 * rr + 1], v[3 * k + 1], fmaf(x[4 * rr + 2], v[3 * k + 2], x[4 * rr + 3])));
      Tri T;
      T.v0 = make_float4(w[0], w[1], w[2], 0.f);
      T.e1 = make_float4(w[3] - w[0], w[4] - w[1], w[5] - w[2], 0.f);
      T.e2 = make_float4(w[6] - w[0], w[7] - w[1], w[8] - w[2], 0.f);
      float t;
      if (tri_hit(g.r, T, g.tmax, t) && t < g.tmax) return true;
    }
  }
  return false;
}

// Moved-object groups staged in shared memory (MovedGroups).
struct GroupSmem {
  float box[kMaxGroups][6];
  int8_t slot[kMaxGroups][kGroupSize];
  int n;
};

// Axis-aligned bounds of the segment a->b, widened by m = 2^-18 max|coord|
// + 1e-19, so that every box seg_box accepts overlaps them.  Why m covers
// seg_box's rounding: a plane distance there is fma(plane, inv, -a inv) with
// inv within 2^-22 of 1/d and d = fl(b - a); an accepted box has, on each
// axis, its near distance <= 1 and its far distance >= 0, which puts its
// near face at most 2^-20 (|b - a| + |a|) <= 3 x 2^-20 max|coord| beyond b
// and its far face at most 2^-24 |a| short of a (for a direction component
// clamped to 1e-20, at most 1.01e-20 beyond a).  The overlap test is exact,
// so it culls no box that seg_box would accept.
struct SegBounds {
  float3 lo, hi;
};

__device__ __forceinline__ SegBounds seg_bounds(float3 a, float3 b) {
  const float mag = fmax3(fmax3(fabsf(a.x), fabsf(a.y), fabsf(a.z)), fmax3(fabsf(b.x), fabsf(b.y), fabsf(b.z)), 0.0f);
  const float m = fmaf(mag, 3.814697265625e-06f, 1e-19f);
  SegBounds s;
  s.lo = make_float3(fminf(a.x, b.x) - m, fminf(a.y, b.y) - m, fminf(a.z, b.z) - m);
  s.hi = make_float3(fmaxf(a.x, b.x) + m, fmaxf(a.y, b.y) + m, fmaxf(a.z, b.z) + m);
  return s;
}

// Closed box bx (lo xyz, hi xyz) against the widened segment bounds.
__device__ __forceinline__ bool seg_overlaps(const SegBounds& s, const float* bx) {
  return (s.lo.x <= bx[3]) & (s.hi.x >= bx[0]) & (s.lo.y <= bx[4]) & (s.hi.y >= bx[1]) & (s.lo.z <= bx[5]) &
         (s.hi.z >= bx[2]);
}

// Segment a->b against every moved object.  Box tests cull first by the
// segment's widened bounds against the union of all moved boxes, then
// against each group's box, and run the slab test (seg_box) only on members
// whose box the bounds overlap (its reciprocals computed once the union
// cull has passed).  Neither cull rejects a box that seg_box accepts
// (seg_bounds), and a box that contains another overlaps whatever the inner
// one does, so the result is that of the slab test against every moved
// object.
template <int S = kStack>
__device__ __forceinline__ bool seg_vs_moved(const SceneView& sv, const float* cull, const float* uni,
                                             const GroupSmem& gs, bool boxes, bool test_old, float3 a, float3 b,
                                             Work& wk) {
  if (boxes) {
    const SegBounds sb = seg_bounds(a, b);
    if (!seg_overlaps(sb, uni + 6 * kMaxDyn)) return false;
    const Seg g = seg_prep(sv, a, b, true);
    auto slab = [&](const float* bx) { return seg_box(g.inv, g.aoi, bx); };
    if (gs.n == 0) {                           // no group table: every moved object in turn
      for (uint64_t m = sv.moved; m; m &= m - 1) {
        const float* bx = uni + 6 * (__ffsll((long long)m) - 1);
        if (seg_overlaps(sb, bx) && slab(bx)) return true;
      }
      return false;
    }
    for (int q = 0; q < gs.n; ++q) {
      if (gs.n > 1 && !seg_overlaps(sb, gs.box[q])) continue;   // one group: its box is the union
#pragma unroll
      for (int m = 0; m < kGroupSize; ++m) {
        const int s = gs.slot[q][m];
        if (s < 0) break;
        const float* bx = uni + 6 * s;
        if (seg_overlaps(sb, bx) && slab(bx)) return true;
      }
    }
    return false;
  }
  const Seg g = seg_prep(sv, a, b, false);
  for (uint64_t m = sv.moved; m; m &= m - 1)
    if (seg_vs_object<S>(sv, g, cull, uni, false, test_old, __ffsll((long long)m) - 1, wk)) return true;
  return false;
}

__device__ __forceinline__ uint32_t* field(pv_frame_stats* s, size_t off) {
  return s ? reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(s) + off) : nullptr;
}

// Shared memory of one verify block.
struct VerifySmem {
  float cull[kMaxDyn * 6];
  float uni[(kMaxDyn + 1) * 6];
  GroupSmem groups;
  uint32_t red[32 * 7];
  unsigned long long red64[32];
  int mslot[kMaxDyn];          // moved slots in ascending order (warp mapping)
  int n_moved;
  uint32_t hitmask[256];       // flat mapping: intersected segments of each thread's path
  uint32_t slotmask[256];      // flat mapping: segments decided by a moved primitive at an end
  uint16_t seg_owner[256 / 32][32 * PV_MAX_BOUNCES];   // flat mapping, per warp: segment q's lane | k << 5
};

// Result of the origin stage for one path.
struct PathCheck {
  float3 o;                    // emission point after Sec. 3.1
  uint32_t nseg, cell;
  bool test;                   // the segment stage must run
  bool blocked1;               // a moved point light's visibility ray is blocked
  bool replaced;               // marked for a fresh emission by the origin stage
};

// The touched byte of a path: 0 if untouched, else 1 + the photon count of
// its record on entry (v.nseg is read before any rewrite of the info word).
__device__ __forceinline__ uint8_t touched_code(bool touched, const PathCheck& v) {
  return touched ? (uint8_t)(1u + v.nseg) : (uint8_t)0;
}

// Record path p's touched byte; with a carried atlas, take a touched path's
// entry photons out of it (pa / pb are not written before the re-trace kernel).
__device__ __forceinline__ void mark_touched(const VerifyArgs& A, uint32_t p, bool touched, const PathCheck& v) {
  if (!A.touched) return;
  const uint8_t code = touched_code(touched, v);
  A.touched[p] = code;
  if (code && A.sub.data) deposit_rows<true>(atlas_map(A.sub), A.n, code - 1u, A.pa, A.pb, p);
}

// Sec. 3.1 "update path origins" for path p (< A.n): the moved light's
// emission point is re-derived; a path that cannot be kept is marked for a
// fresh emission.
template <bool kPointVis, int S = kStack>
__device__ __forceinline__ PathCheck origin_stage(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                                  int root, uint32_t p, uint32_t& c_vis, uint32_t& c_reemit, Work& wk) {
  const uint32_t n = A.n;
  const uint32_t w = A.info[p];
  PathCheck v;
  v.nseg = min(info_nseg(w), sv.B);
  v.cell = w & PV_INFO_CELL_MASK;
  const uint32_t l = info_light(w);
  v.o = make_float3(A.origin[p], A.origin[n + p], A.origin[2 * (size_t)n + p]);
  v.blocked1 = false;
  v.replaced = false;
  bool invalid = false;
  if ((L.moved_mask >> l) & 1u) {
    const DmLight& D = L.dm[l];
    int dm_cell = -1;
    if (D.dims && v.nseg > 0) {              // Compute DM_C: the parametrisation decides (Sec. 3.1)
      float u[4];
      if (dm_param(L.cur[l], f3(A.pa[p]), v.o, u)) dm_cell = (int)dm_cell_of_u(D, u);
    }
    if (v.nseg == 0 || (D.dims && dm_cell < 0)) {
      invalid = true;                        // an escaped path has no vertex to re-aim at; or off the map
    } else {
      const bool by_map = D.dims != 0;       // the map has decided validity
      const float4 x1v = A.pa[p];
      const float3 x1 = f3(x1v);
      const LightPose& Ln = L.cur[l];
      float3 o = v.o;
      if (Ln.type == PV_LIGHT_POINT) {
        o = Ln.pos;
        if (kPointVis) {
          const float3 dv = x1 - o;
          const float len = sqrtf(dot(dv, dv));
          if (len > 0.0f) {
            const Ray r = make_ray(o, make_float3(dv.x / len, dv.y / len, dv.z / len), sv.tmin);
            v.blocked1 = any_hit_all<S>(sv, root, r, len - sv.tmin, __float_as_int(x1v.w), wk);
          }
          ++c_vis;
        }
      } else {
        const float3 d = normalize_exact(x1 - o);
        const float nd = dot(Ln.n, d);
        if (!by_map && !(nd > 0.0f)) {
          invalid = true;
        } else {
          const float tp = dot(Ln.n, x1 - Ln.pos) / nd;
          if (!by_map && !(tp > 0.0f)) {
            invalid = true;
          } else {
            const float3 op = make_float3(fmaf(-tp, d.x, x1.x), fmaf(-tp, d.y, x1.y), fmaf(-tp, d.z, x1.z));
            const float3 rel = op - Ln.pos;
            if (!by_map && (fabsf(dot(Ln.t, rel)) > 0.5f * Ln.size.x || fabsf(dot(Ln.b, rel)) > 0.5f * Ln.size.y))
              invalid = true;
            if (!invalid && ((L.tilted_mask >> l) & 1u)) {
              const float ratio = nd / dot(L.old[l].n, d);
              const float4 e = A.pb[p];
              if (!energy_close(ratio * f3(e), f3(e), A.tau)) invalid = true;
            }
            o = op;
          }
        }
      }
      if (!invalid) {
        A.origin[p] = o.x;
        A.origin[n + p] = o.y;
        A.origin[2 * (size_t)n + p] = o.z;
        v.o = o;
      }
    }
    if (invalid) {
      A.info[p] = info_make(v.cell, 0, 0, true, false);
      v.replaced = true;
      ++c_reemit;
    } else if (dm_cell >= 0) {
      atomicAdd(D.dmc + dm_cell, 1u);
      v.cell = (l << 20) | (uint32_t)dm_cell;
      if (v.cell != (w & PV_INFO_CELL_MASK)) A.info[p] = (w & ~PV_INFO_CELL_MASK) | v.cell;
    }
  }
  v.test = !invalid && (sv.moved || v.blocked1);
  return v;
}

// Segment k of a path ends or starts on a moved object's primitive (or is the
// blocked first segment of a moved point light): intersected without a test.
__device__ __forceinline__ bool slot_hit(const SceneView& sv, uint32_t k, int prim_a, int prim_b, bool blocked1) {
  return slot_moved(sv, prim_b) || (k >= 2 && slot_moved(sv, prim_a)) || (k == 1 && blocked1);
}

// Re-trace decision from the intersected-segment mask (bit k = segment k);
// returns whether the path enters the error-based continuation.
__device__ __forceinline__ bool finish_stage(const VerifyArgs& A, uint32_t p, const PathCheck& v, uint32_t mask,
                                             uint32_t& c_reemit, uint32_t& c_tail) {
  if (!mask) return false;
  if (A.mode != PV_MODE_ERROR) {
    const uint32_t first = __ffs(mask) - 1;
    if (first == 1) {
      A.info[p] = info_make(v.cell, 0, 0, true, true);       // keep light position and direction
      ++c_reemit;
    } else {
      A.info[p] = info_make(v.cell, first - 1, first - 1, true, false);
      ++c_tail;
    }
    return false;
  }
  A.mask_out[p] = mask;
  return true;
}

// Block prologue: moved objects' boxes, their union, and the moved-slot list.
__device__ __forceinline__ void verify_smem_init(const SceneView& sv, VerifySmem& sm) {
  load_boxes(sv, sm.cull, sm.uni);
  // this frame's groups of the moved objects (none without a group table)
  const bool have = sv.moved && sv.groups;
  const int ng = have ? (int)min(sv.groups->n, (uint32_t)kMaxGroups) : 0;
  for (int i = threadIdx.x; i < ng * 6; i += blockDim.x) sm.groups.box[i / 6][i % 6] = sv.groups->box[i / 6][i % 6];
  for (int i = threadIdx.x; i < ng * kGroupSize; i += blockDim.x)
    sm.groups.slot[i / kGroupSize][i % kGroupSize] = sv.groups->slot[i / kGroupSize][i % kGroupSize];
  if (threadIdx.x == 0) sm.groups.n = ng;
  if (threadIdx.x == 0) {
    int k = 0;
    for (uint64_t m = sv.moved; m; m &= m - 1) sm.mslot[k++] = __ffsll((long long)m) - 1;
    sm.n_moved = k;
  }
  __syncthreads();
  if (threadIdx.x < 6) {                 // union of the moved objects' old u new boxes
    const int k = threadIdx.x;
    float v = k < 3 ? 3.0e38f : -3.0e38f;
    for (uint64_t m = sv.moved; m; m &= m - 1) {
      const float x = sm.uni[6 * (__ffsll((long long)m) - 1) + k];
      v = k < 3 ? fminf(v, x) : fmaxf(v, x);
    }
    sm.uni[6 * kMaxDyn + k] = v;
  }
  __syncthreads();
}

// Block epilogue: continuation list (one atomic per warp) and counters.
// Append the calling lanes' paths with ``want`` set to list[count] (one
// atomic per warp).
__device__ __forceinline__ void warp_append(bool want, uint32_t p, uint32_t* list, uint32_t* count) {
  const unsigned wm = __ballot_sync(0xffffffffu, want);
  if (!wm) return;
  const int lane = threadIdx.x & 31, leader = __ffs(wm) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(wm));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) list[base + __popc(wm & ((1u << lane) - 1u))] = p;
}

// Verification counters of one thread, summed over the paths it handled.
struct VerifyCount {
  uint32_t paths = 0, tested = 0, vis = 0, reemit = 0, tail = 0, cont = 0, listed = 0;
};

// Per-path end of verification: list appends (one atomic per warp) and counts.
__device__ __forceinline__ void verify_tile_end(const VerifyArgs& A, uint32_t p, bool want_cont, bool listed,
                                                VerifyCount& vc) {
  warp_append(want_cont, p, A.cont_list, A.cont_count);
  if (A.list_out) warp_append(listed, p, A.list_out, A.list_count);
  vc.paths += p < A.n ? 1u : 0u;
  vc.cont += want_cont ? 1u : 0u;
  vc.listed += listed ? 1u : 0u;
}

// Block-wide counter sums, one atomic per counter per block (all threads call).
__device__ __forceinline__ void verify_counts_flush(const VerifyArgs& A, const VerifyCount& vc, const Work& wk,
                                                    bool traversed, VerifySmem& sm) {
  uint32_t* const ctr[7] = {field(A.stats, offsetof(pv_frame_stats, n_paths)),
                            field(A.stats, offsetof(pv_frame_stats, segments_tested)),
                            field(A.stats, offsetof(pv_frame_stats, vis_rays)),
                            field(A.stats, offsetof(pv_frame_stats, n_reemit)),
                            field(A.stats, offsetof(pv_frame_stats, n_tail)),
                            field(A.stats, offsetof(pv_frame_stats, n_cont)),
                            A.list_out ? field(A.stats, offsetof(pv_frame_stats, n_listed)) : nullptr};
  const uint32_t val[7] = {vc.paths, vc.tested, vc.vis, vc.reemit, vc.tail, vc.cont, vc.listed};
  block_add_n<7>(ctr, val, sm.red);
  if (traversed) {
    block_add64(A.stats ? (unsigned long long*)&A.stats->node_visits : nullptr, wk.nodes, sm.red64);
    block_add64(A.stats ? (unsigned long long*)&A.stats->tri_tests : nullptr, wk.tris, sm.red64);
  }
}


// kPointVis: a moved point light needs visibility rays; kExact: segments are
// tested against triangles (not only boxes).  Specialised so the common case
// carries no traversal code.
//
// Thread per path: the whole block verifies paths p (this thread's; p >= A.n
// idles), Sec. 3.2's segments in order from the light; called by every thread
// of the block (block reductions inside).
template <bool kPointVis, bool kExact, int S = kStack>
__device__ __forceinline__ void verify_tile_thread(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                                   int root, uint32_t p, VerifySmem& sm, VerifyCount& vc, Work& wk) {
  const uint32_t n = A.n;
  const bool test_old = kExact && (A.flags & PV_FLAG_TEST_OLD_TRIS) != 0;
  bool want_cont = false, touched = false, listed = false;
  if (p < n) {
    const PathCheck v = origin_stage<kPointVis, S>(sv, L, A, root, p, vc.vis, vc.reemit, wk);
    if (v.test) {
      // ---- Sec. 3.2: segments in order, starting from the light
      uint32_t mask = 0;
      float3 a = v.o;
      int prim_a = -1;
      for (uint32_t k = 1; k <= v.nseg; ++k) {
        const float4 vb = A.pa[(size_t)(k - 1) * n + p];
        const float3 b = f3(vb);
        const int prim_b = __float_as_int(vb.w);
        bool hit = slot_hit(sv, k, prim_a, prim_b, v.blocked1);
        if (!hit && sv.moved) {
          ++vc.tested;
          hit = kExact ? seg_vs_moved<S>(sv, sm.cull, sm.uni, sm.groups, false, test_old, a, b, wk)
                       : seg_vs_moved<S>(sv, sm.cull, sm.uni, sm.groups, true, false, a, b, wk);
        }
        if (hit) {
          mask |= 1u << k;
          if (A.mode != PV_MODE_ERROR) break;
        }
        a = b;
        prim_a = prim_b;
      }
      want_cont = finish_stage(A, p, v, mask, vc.reemit, vc.tail);
      touched = mask != 0;                   // handed to Alg. 1, or (naive modes) marked for re-tracing
      listed = mask != 0 && A.mode != PV_MODE_ERROR;
    }
    mark_touched(A, p, touched || v.replaced, v);
    listed = listed || v.replaced;
  }
  verify_tile_end(A, p, want_cont, listed, vc);
}

template <bool kPointVis, bool kExact, int S = kStack>
__device__ __forceinline__ void verify_block(const SceneView& sv, const FrameLights& L, const VerifyArgs& A, uint32_t p,
                                             VerifySmem& sm) {
  verify_smem_init(sv, sm);
  Work wk;
  VerifyCount vc;
  verify_tile_thread<kPointVis, kExact, S>(sv, L, A, *sv.root, p, sm, vc, wk);
  verify_counts_flush(A, vc, wk, kPointVis || kExact, sm);
}

// Warp per path: each lane runs the origin stage of its own path, then the
// warp takes its paths one at a time and spreads (segment, moved object)
// pairs over its lanes; the intersected-segment mask is the OR over lanes.
// Same masks and decisions as verify_block; the segments-tested counter
// follows verify_block's sequential order, while the traversal counters
// count every pair tested here.
template <bool kPointVis, bool kExact, int S = kStack>
__device__ __forceinline__ void verify_tile_warp(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                                 int root, uint32_t p, VerifySmem& sm, VerifyCount& vc, Work& wk) {
  const uint32_t n = A.n;
  const int lane = threadIdx.x & 31;
  const bool test_old = kExact && (A.flags & PV_FLAG_TEST_OLD_TRIS) != 0;
  const bool error_mode = A.mode == PV_MODE_ERROR;
  const int n_moved = sm.n_moved;
  PathCheck v;
  v.test = false;
  v.nseg = 0;
  v.o = make_float3(0.f, 0.f, 0.f);
  v.blocked1 = false;
  v.replaced = false;
  v.cell = 0;
  if (p < n) v = origin_stage<kPointVis, S>(sv, L, A, root, p, vc.vis, vc.reemit, wk);
  uint32_t my_mask = 0;
  for (unsigned todo = __ballot_sync(0xffffffffu, v.test); todo; todo &= todo - 1) {
    const int j = __ffs(todo) - 1;
    const uint32_t pj = __shfl_sync(0xffffffffu, p, j);
    const uint32_t nseg = __shfl_sync(0xffffffffu, v.nseg, j);
    const bool blocked1 = __shfl_sync(0xffffffffu, v.blocked1, j);
    const float3 o = make_float3(__shfl_sync(0xffffffffu, v.o.x, j), __shfl_sync(0xffffffffu, v.o.y, j),
                                 __shfl_sync(0xffffffffu, v.o.z, j));
    // segments ending or starting on a moved primitive: lane k-1 takes segment k
    bool sh = false;
    if ((uint32_t)lane < nseg) {
      const uint32_t k = lane + 1;
      const int prim_b = __float_as_int(A.pa[(size_t)lane * n + pj].w);
      const int prim_a = k >= 2 ? __float_as_int(A.pa[(size_t)(lane - 1) * n + pj].w) : -1;
      sh = slot_hit(sv, k, prim_a, prim_b, blocked1);
    }
    const uint32_t smask = __ballot_sync(0xffffffffu, sh) << 1;
    // (segment, moved object) pairs not already decided
    uint32_t tmask = 0;
    const uint32_t pairs = nseg * (uint32_t)n_moved;
    for (uint32_t q = lane; q < pairs; q += 32) {
      const uint32_t k = q / (uint32_t)n_moved + 1;
      if ((smask >> k) & 1u) continue;
      if ((tmask >> k) & 1u) continue;
      const int obj = sm.mslot[q % (uint32_t)n_moved];
      const float3 b = f3(A.pa[(size_t)(k - 1) * n + pj]);
      const float3 a = k == 1 ? o : f3(A.pa[(size_t)(k - 2) * n + pj]);
      const Seg g = seg_prep(sv, a, b, !kExact);
      bool hit;
      if (!kExact) hit = seg_box(g.inv, g.aoi, sm.uni + 6 * kMaxDyn) && seg_vs_object<S>(sv, g, sm.cull, sm.uni, true, false, obj, wk);
      else hit = seg_vs_object<S>(sv, g, sm.cull, sm.uni, false, test_old, obj, wk);
      if (hit) tmask |= 1u << k;
    }
    const uint32_t mask = smask | __reduce_or_sync(0xffffffffu, tmask);
    if (lane == j) {
      uint32_t m = mask;
      uint32_t last = nseg;
      if (!error_mode && m) {
        last = __ffs(m) - 1;
        m = 1u << last;
      }
      // segments sequential verification would have tested: 1..last, not slot-hit
      if (sv.moved && last >= 1) vc.tested += __popc(~smask & ((2u << last) - 2u));
      my_mask = m;
    }
  }
  bool want_cont = false;
  if (p < n && v.test) want_cont = finish_stage(A, p, v, my_mask, vc.reemit, vc.tail);
  if (p < n) mark_touched(A, p, (v.test && my_mask != 0) || v.replaced, v);
  const bool listed = p < n && (v.replaced || (v.test && my_mask != 0 && !error_mode));
  verify_tile_end(A, p, want_cont, listed, vc);
}

template <bool kPointVis, bool kExact, int S = kStack>
__device__ __forceinline__ void verify_block_warp(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                                  uint32_t p, VerifySmem& sm) {
  verify_smem_init(sv, sm);
  Work wk;
  VerifyCount vc;
  verify_tile_warp<kPointVis, kExact, S>(sv, L, A, *sv.root, p, sm, vc, wk);
  verify_counts_flush(A, vc, wk, kPointVis || kExact, sm);
}

struct ContArgs {
  uint32_t n;
  uint32_t* info;
  const float* origin;
  float4* pa;
  const float4* pb;
  const uint32_t* mask;
  const uint32_t* list;
  const uint32_t* count;
  uint32_t* ticket;
  float tau;
  pv_frame_stats* stats;
};

// Alg. 1 as a resumable state machine, so that a persistent kernel can
// interleave its ray queries with other rays.  Between two queries a path's
// state is: the segment ``seg`` whose query is in flight; ``mask`` (bits 0-15
// the segments the box test intersected, bits 16-31 the segments whose origin
// moved); ``meta`` (bits 0-3 the path length, then "origin carried" and
// "vertices updated"); the original position ``a_orig`` and primitive
// ``a_prim`` of the segment's origin.  The current origin is the query ray's
// origin, and ``a_prim`` doubles as the query's exclusion (the light origin
// of segment 1 carries -1).  Vertices are read from and updated in the path
// buffer as the loop advances.
constexpr uint32_t kContCarried = 1u << 4;     // the segment's origin moved and is carried in registers
constexpr uint32_t kContUpdated = 1u << 5;     // some vertex was moved
enum { kContNext = 0, kContDone = 1, kContTail = 2 };

struct ContCounters {
  uint32_t rays = 0, tail = 0, upd = 0, trunc = 0;
};

// stored vertex k of path p (0 = origin, primitive -1)
__device__ __forceinline__ float4 cont_vertex(const ContArgs& A, uint32_t p, uint32_t k) {
  const uint32_t n = A.n;
  return k == 0 ? make_float4(A.origin[p], A.origin[n + p], A.origin[2 * (size_t)n + p], __int_as_float(-1))
                : A.pa[(size_t)(k - 1) * n + p];
}

// The path is kept (possibly shortened or with moved vertices).
__device__ __forceinline__ void cont_finish(const ContArgs& A, uint32_t p, uint32_t cell, uint32_t meta,
                                            ContCounters& cc) {
  A.info[p] = info_make(cell, meta & 15u, 0, false, false);
  if (meta & kContUpdated) ++cc.upd;
}

// Set up the query of the next segment from ``seg`` on that needs one; false
// once the path is finished (its info word written).  ``a_cur`` is the
// carried origin (used when kContCarried is set).
__device__ __forceinline__ bool cont_next(const SceneView& sv, const ContArgs& A, uint32_t p, uint32_t cell,
                                          uint32_t& seg, uint32_t& mask, uint32_t& meta, float3& a_orig, int& a_prim,
                                          float3 a_cur, Ray& r, ContCounters& cc) {
  const uint32_t nseg = meta & 15u;
  while (seg <= nseg) {
    if (!((mask >> seg) & 1u) && !((mask >> (16 + seg)) & 1u)) {
      ++seg;
      meta &= ~kContCarried;
      continue;
    }
    if (!(meta & kContCarried)) {
      const float4 v = cont_vertex(A, p, seg - 1);
      a_cur = a_orig = f3(v);
      a_prim = __float_as_int(v.w);
    }
    const float3 b = f3(cont_vertex(A, p, seg));
    r = make_ray(a_cur, normalize_exact(b - a_cur), sv.tmin);
    ++cc.rays;
    return true;
  }
  cont_finish(A, p, cell, meta, cc);
  return false;
}

// Start Alg. 1 on path p; false if it needs no query (finished).
__device__ __forceinline__ bool cont_begin(const SceneView& sv, const ContArgs& A, uint32_t p, uint32_t& cell,
                                           uint32_t& seg, uint32_t& mask, uint32_t& meta, float3& a_orig, int& a_prim,
                                           Ray& r, ContCounters& cc) {
  const uint32_t w = A.info[p];
  cell = w & PV_INFO_CELL_MASK;
  meta = min(info_nseg(w), sv.B);
  mask = A.mask[p] & 0xFFFFu;
  seg = __ffs(mask) - 1;
  return cont_next(sv, A, p, cell, seg, mask, meta, a_orig, a_prim, a_orig, r, cc);
}

// Take the result of the query of segment ``seg`` (hit triangle ``tri`` at
// ``t``, tri < 0 for none).  kContNext: continue with cont_next from the
// returned ``a_cur``; kContDone: the path is kept (info written); kContTail:
// Eq. 2 failed, the path is marked for re-tracing from vertex ``seg``.
__device__ __forceinline__ int cont_hit(const SceneView& sv, const ContArgs& A, uint32_t p, uint32_t cell,
                                        uint32_t& seg, uint32_t& mask, uint32_t& meta, float3& a_orig, int& a_prim,
                                        const Ray& r, int tri, float t, float3& a_cur, ContCounters& cc) {
  const uint32_t n = A.n;
  if (tri < 0) {                                                       // escaped: the path ends here
    meta = (meta & ~15u) | (seg - 1);
    ++cc.trunc;
    cont_finish(A, p, cell, meta, cc);
    return kContDone;
  }
  a_cur = r.o;
  const float3 d = r.d;
  const float4 bv = cont_vertex(A, p, seg);
  const float3 b = f3(bv);
  const int b_prim = __float_as_int(bv.w);
  const Tri T = load_tri(sv.tris, tri);
  const int pn = __float_as_int(T.v0.w);
  const float3 xn = make_float3(fmaf(t, d.x, a_cur.x), fmaf(t, d.y, a_cur.y), fmaf(t, d.z, a_cur.z));
  const bool close = pn == b_prim && maxabs3(xn - b) <= sv.close_tol;
  if (seg == (meta & 15u)) {                                           // last photon: move it
    A.pa[(size_t)(seg - 1) * n + p] = make_float4(xn.x, xn.y, xn.z, __int_as_float(pn));
    meta |= kContUpdated;
    cont_finish(A, p, cell, meta, cc);
    return kContDone;
  }
  const float4 cv = cont_vertex(A, p, seg + 1);                       // stored next photon
  const float3 c = f3(cv);
  const float3 EO = f3(A.pb[(size_t)seg * n + p]);
  float3 EN = EO;
  if (!close) {
    const float4 albn = __ldg(sv.prim_alb + pn);
    const float3 nn = normalize(cross(f3(T.e1), f3(T.e2)));
    const float3 nsn = dot(nn, d) < 0.0f ? nn : -1.0f * nn;
    const float3 wv = c - xn;
    const float wl = sqrtf(dot(wv, wv));
    const float cosn = wl > 0.0f ? fmaxf(0.0f, dot(nsn, __frcp_rn(wl) * wv)) : 0.0f;
    const float4 albo = __ldg(sv.prim_alb + b_prim);
    const float3 no = normalize(prim_normal(sv, b_prim, true));
    const float3 dino = normalize_exact(b - a_orig);
    const float3 nso = dot(no, dino) < 0.0f ? no : -1.0f * no;
    const float coso = dot(nso, normalize_exact(c - b));
    const float3 Ei = f3(A.pb[(size_t)(seg - 1) * n + p]);
    const float f = coso > 0.0f ? cosn / (albo.w * coso) : 0.0f;
    EN = make_float3(Ei.x * albn.x * f, Ei.y * albn.y * f, Ei.z * albn.z * f);
  }
  if (!energy_close(EN, EO, A.tau)) {                                 // Eq. 2 fails: re-trace from here
    A.pa[(size_t)(seg - 1) * n + p] = make_float4(xn.x, xn.y, xn.z, __int_as_float(pn));
    A.info[p] = info_make(cell, seg, seg, true, false);
    ++cc.tail;
    return kContTail;
  }
  if (close && !((mask >> (seg + 1)) & 1u) && !slot_moved(sv, pn) && !slot_moved(sv, __float_as_int(cv.w))) {
    seg += 2;                                                          // next segment known valid
    meta &= ~kContCarried;
    return kContNext;
  }
  A.pa[(size_t)(seg - 1) * n + p] = make_float4(xn.x, xn.y, xn.z, __int_as_float(pn));
  a_cur = xn;                                                          // origin of the next segment moved
  a_orig = b;
  a_prim = pn;
  meta |= kContCarried | kContUpdated;
  mask |= 1u << (16 + seg + 1);
  ++seg;
  return kContNext;
}

// Alg. 1 for one path, its queries run to completion one after the other.
template <int S = kStack>
__device__ __forceinline__ void continue_path(const SceneView& sv, int root, const ContArgs& A, uint32_t p,
                                              ContCounters& cc, Work& wk) {
  uint32_t cell, seg, mask, meta;
  float3 a_orig = make_float3(0.f, 0.f, 0.f);
  int a_prim = -1;
  Ray r;
  bool more = cont_begin(sv, A, p, cell, seg, mask, meta, a_orig, a_prim, r, cc);
  for (uint32_t guard = 0; more && guard < 64; ++guard) {
    Hit h;
    closest_hit<S>(sv, root, r, a_prim, h, wk);
    float3 a_cur;
    const int o = cont_hit(sv, A, p, cell, seg, mask, meta, a_orig, a_prim, r, h.tri, h.t, a_cur, cc);
    more = o == kContNext && cont_next(sv, A, p, cell, seg, mask, meta, a_orig, a_prim, a_cur, r, cc);
  }
}

// Flat segment mapping: each lane runs the origin stage of its own path,
// then the warp deals all segments of its 32 paths out to its lanes, 32 at
// a time, so lanes with short paths do not idle while long ones finish.  A
// segment's answer is OR-ed into its path's mask in shared memory.  Same
// masks, decisions and counters as verify_block: every segment of a tested
// path is tested there too in error mode, the only mode this mapping serves
// (the naive modes stop at a path's first hit).  Blocks of at most 256.
template <bool kPointVis, bool kExact, int S = kStack>
__device__ __forceinline__ void verify_tile_flat(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                                 int root, uint32_t p, VerifySmem& sm, VerifyCount& vc, Work& wk) {
  const uint32_t n = A.n;
  const int lane = threadIdx.x & 31;
  const uint32_t wbase = threadIdx.x & ~31u;
  const bool test_old = kExact && (A.flags & PV_FLAG_TEST_OLD_TRIS) != 0;
  PathCheck v;
  v.test = false;
  v.nseg = 0;
  v.o = make_float3(0.f, 0.f, 0.f);
  v.blocked1 = false;
  v.replaced = false;
  v.cell = 0;
  if (p < n) v = origin_stage<kPointVis, S>(sv, L, A, root, p, vc.vis, vc.reemit, wk);
  sm.hitmask[threadIdx.x] = 0u;
  sm.slotmask[threadIdx.x] = 0u;
  // segments of the warp's tested paths, numbered by an inclusive prefix over the lanes
  const uint32_t cnt = (p < n && v.test) ? v.nseg : 0u;
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  // each lane enters its segments in the warp's table: entry q = the owning lane and the segment number
  uint16_t* const tab = sm.seg_owner[threadIdx.x >> 5];
  for (uint32_t j = 0; j < cnt; ++j) tab[incl - cnt + j] = (uint16_t)(lane | ((j + 1) << 5));
  __syncwarp();
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t q = base + lane;
    const uint32_t e = q < total ? tab[q] : 0u;
    const uint32_t owner = e & 31u;
    const uint32_t po = __shfl_sync(0xffffffffu, p, owner);
    const float ox = __shfl_sync(0xffffffffu, v.o.x, owner), oy = __shfl_sync(0xffffffffu, v.o.y, owner);
    const float oz = __shfl_sync(0xffffffffu, v.o.z, owner);
    const bool blocked1 = __shfl_sync(0xffffffffu, v.blocked1, owner);
    if (q >= total) continue;
    const uint32_t k = e >> 5;                 // segment k of path po, 1 .. nseg
    const float4 vb = A.pa[(size_t)(k - 1) * n + po];
    const float4 va = k >= 2 ? A.pa[(size_t)(k - 2) * n + po] : make_float4(ox, oy, oz, __int_as_float(-1));
    const int prim_b = __float_as_int(vb.w), prim_a = __float_as_int(va.w);
    bool hit = slot_hit(sv, k, prim_a, prim_b, blocked1);
    if (hit) {
      atomicOr(&sm.slotmask[wbase + owner], 1u << k);
    } else if (sv.moved) {
      hit = kExact ? seg_vs_moved<S>(sv, sm.cull, sm.uni, sm.groups, false, test_old, f3(va), f3(vb), wk)
                   : seg_vs_moved<S>(sv, sm.cull, sm.uni, sm.groups, true, false, f3(va), f3(vb), wk);
    }
    if (hit) atomicOr(&sm.hitmask[wbase + owner], 1u << k);
  }
  __syncwarp();
  bool want_cont = false;
  if (p < n && v.test) {
    const uint32_t mask = sm.hitmask[threadIdx.x];
    if (sv.moved && v.nseg >= 1) vc.tested += __popc(~sm.slotmask[threadIdx.x] & ((2u << v.nseg) - 2u));
    want_cont = finish_stage(A, p, v, mask, vc.reemit, vc.tail);
    mark_touched(A, p, mask != 0 || v.replaced, v);
  } else if (p < n) {
    mark_touched(A, p, v.replaced, v);
  }
  verify_tile_end(A, p, want_cont, p < n && v.replaced, vc);
}

template <bool kPointVis, bool kExact, int S = kStack>
__device__ __forceinline__ void verify_block_flat(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                                  uint32_t p, VerifySmem& sm) {
  verify_smem_init(sv, sm);
  Work wk;
  VerifyCount vc;
  verify_tile_flat<kPointVis, kExact, S>(sv, L, A, *sv.root, p, sm, vc, wk);
  verify_counts_flush(A, vc, wk, kPointVis || kExact, sm);
}

// One tile of paths p (this thread's) in mapping kMap: 0 thread per path,
// 1 warp per path, 2 flat segments (error mode).  No block-wide barrier
// inside: the caller staged the block prologue and sums the counters.
template <bool kPointVis, bool kExact, int kMap, int S = kStack>
__device__ __forceinline__ void verify_tile(const SceneView& sv, const FrameLights& L, const VerifyArgs& A, int root,
                                            uint32_t p, VerifySmem& sm, VerifyCount& vc, Work& wk) {
  if (kMap == 2) verify_tile_flat<kPointVis, kExact, S>(sv, L, A, root, p, sm, vc, wk);
  else if (kMap == 1) verify_tile_warp<kPointVis, kExact, S>(sv, L, A, root, p, sm, vc, wk);
  else verify_tile_thread<kPointVis, kExact, S>(sv, L, A, root, p, sm, vc, wk);
}

// Mapping kMap over tiles t = first, first + stride, ... of blockDim.x paths,
// with the block prologue and the counter reductions done once.
template <bool kPointVis, bool kExact, int kMap, int S = kStack>
__device__ __forceinline__ void verify_tiles(const SceneView& sv, const FrameLights& L, const VerifyArgs& A,
                                             uint32_t first, uint32_t stride, VerifySmem& sm) {
  verify_smem_init(sv, sm);
  Work wk;
  VerifyCount vc;
  const int root = *sv.root;
  const uint32_t tiles = (A.n + blockDim.x - 1) / blockDim.x;
  for (uint32_t t = first; t < tiles; t += stride)
    verify_tile<kPointVis, kExact, kMap, S>(sv, L, A, root, t * blockDim.x + threadIdx.x, sm, vc, wk);
  verify_counts_flush(A, vc, wk, kPointVis || kExact, sm);
}

}  // namespace pvk
