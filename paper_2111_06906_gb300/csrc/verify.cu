// Per-frame verification of stored photon paths.
//
// k_verify (one thread per path, streaming the 2-D photon array row by row):
//   Sec. 3.1 "update path origins" fused with Sec. 3.2 "dynamic occlusions"
//   as in Sec. 4 (origins first, then the ordered segment tests).
// k_continue (persistent, over the paths k_verify flagged in error mode):
//   the error-based threshold continuation of Sec. 3.3, Alg. 1 and Eq. 2.
// Then the replace bits are compacted into the re-trace list (compact.cu).
#include "pv_scene.h"

using namespace pvk;

namespace {

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
  const float t0 = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), 0.0f));
  const float t1 = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), 1.0f));
  return t0 <= t1;
}

// Segment a->b against every moved object: box test (old u new tight box)
// or exact any-hit over the object's triangles at the new pose (and the old
// pose with PV_FLAG_TEST_OLD_TRIS, by brute force over object-local corners).
__device__ bool seg_vs_moved(const SceneView& sv, const float* cull, const float* uni, bool boxes, bool test_old,
                             float3 a, float3 b, Work& wk) {
  const float3 dv = b - a;
  uint64_t m = sv.moved;
  if (boxes) {
    const float e = 1e-20f;                 // |1/d| <= 1e20 keeps a * inv finite for any scene size
    const float3 inv = make_float3(__frcp_rn(fabsf(dv.x) > e ? dv.x : copysignf(e, dv.x)),
                                   __frcp_rn(fabsf(dv.y) > e ? dv.y : copysignf(e, dv.y)),
                                   __frcp_rn(fabsf(dv.z) > e ? dv.z : copysignf(e, dv.z)));
    const float3 aoi = make_float3(-a.x * inv.x, -a.y * inv.y, -a.z * inv.z);
    if (!seg_box(inv, aoi, uni + 6 * kMaxDyn)) return false;     // union of all moved boxes
    while (m) {
      const int s = __ffsll((long long)m) - 1;
      m &= m - 1;
      if (seg_box(inv, aoi, uni + 6 * s)) return true;
    }
    return false;
  }
  const float len = sqrtf(dot(dv, dv));
  if (!(len > 0.0f)) return false;
  const float3 d = make_float3(dv.x / len, dv.y / len, dv.z / len);
  const Ray r = make_ray(a, d, sv.tmin);
  const float tmax = len - sv.tmin;
  if (!(tmax > sv.tmin)) return false;
  while (m) {
    const int s = __ffsll((long long)m) - 1;
    m &= m - 1;
    float te;
    if (sv.objs[s].wroot != INT32_MIN && box1(r, tmax, cull + 6 * s, te)) {
      float tb = tmax;
      int best = -1;
      traverse<true>(sv.nodes, sv.tris, sv.objs[s].wroot, r, tb, best, -1, sv.max_visits, sv.status, wk);
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
        if (tri_hit(r, T, tmax, t)) return true;
      }
    }
  }
  return false;
}

__device__ __forceinline__ uint32_t* field(pv_frame_stats* s, size_t off) {
  return s ? reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(s) + off) : nullptr;
}

// kPointVis: a moved point light needs visibility rays; kExact: segments are
// tested against triangles (not only boxes).  Specialised so the common case
// carries no traversal code.
template <bool kPointVis, bool kExact>
__global__ void __launch_bounds__(pvh::kVerifyThreads) k_verify(SceneView sv, FrameLights L, VerifyArgs A) {
  __shared__ float s_cull[kMaxDyn * 6];
  __shared__ float s_uni[(kMaxDyn + 1) * 6];
  __shared__ uint32_t s_red[32 * 6];
  __shared__ unsigned long long s_red64[32];
  load_boxes(sv, s_cull, s_uni);
  __syncthreads();
  if (threadIdx.x < 6) {                 // union of the moved objects' old u new boxes
    const int k = threadIdx.x;
    float v = k < 3 ? 3.0e38f : -3.0e38f;
    for (uint64_t m = sv.moved; m; m &= m - 1) {
      const float x = s_uni[6 * (__ffsll((long long)m) - 1) + k];
      v = k < 3 ? fminf(v, x) : fmaxf(v, x);
    }
    s_uni[6 * kMaxDyn + k] = v;
  }
  __syncthreads();
  Work wk;
  const int root = *sv.root;
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = A.n;
  const bool test_old = kExact && (A.flags & PV_FLAG_TEST_OLD_TRIS) != 0;
  uint32_t c_tested = 0, c_vis = 0, c_reemit = 0, c_tail = 0;
  bool want_cont = false;
  if (p < n) {
    const uint32_t w = A.info[p];
    const uint32_t nseg = min(info_nseg(w), sv.B), l = info_light(w), cell = w & PV_INFO_CELL_MASK;
    float3 o = make_float3(A.origin[p], A.origin[n + p], A.origin[2 * (size_t)n + p]);
    bool blocked1 = false, invalid = false;
    if ((L.moved_mask >> l) & 1u) {
      // ---- Sec. 3.1: update path origins
      if (nseg == 0) {
        invalid = true;                        // an escaped path has no vertex to re-aim at
      } else {
        const float4 x1v = A.pa[p];
        const float3 x1 = f3(x1v);
        const LightPose& Ln = L.cur[l];
        if (Ln.type == PV_LIGHT_POINT) {
          o = Ln.pos;
          if (kPointVis) {
            const float3 dv = x1 - o;
            const float len = sqrtf(dot(dv, dv));
            if (len > 0.0f) {
              const Ray r = make_ray(o, make_float3(dv.x / len, dv.y / len, dv.z / len), sv.tmin);
              blocked1 = any_hit_all(sv, root, r, len - sv.tmin, __float_as_int(x1v.w), wk);
            }
            ++c_vis;
          }
        } else {
          const float3 d = normalize_exact(x1 - o);
          const float nd = dot(Ln.n, d);
          if (!(nd > 0.0f)) {
            invalid = true;
          } else {
            const float tp = dot(Ln.n, x1 - Ln.pos) / nd;
            if (!(tp > 0.0f)) {
              invalid = true;
            } else {
              const float3 op = make_float3(fmaf(-tp, d.x, x1.x), fmaf(-tp, d.y, x1.y), fmaf(-tp, d.z, x1.z));
              const float3 rel = op - Ln.pos;
              if (fabsf(dot(Ln.t, rel)) > 0.5f * Ln.size.x || fabsf(dot(Ln.b, rel)) > 0.5f * Ln.size.y) invalid = true;
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
        }
      }
      if (invalid) {
        A.info[p] = info_make(cell, 0, 0, true, false);
        ++c_reemit;
      }
    }
    if (!invalid && (sv.moved || blocked1)) {
      // ---- Sec. 3.2: segments in order, starting from the light
      uint32_t mask = 0;
      float3 a = o;
      int prim_a = -1;
      for (uint32_t k = 1; k <= nseg; ++k) {
        const float4 v = A.pa[(size_t)(k - 1) * n + p];
        const float3 b = f3(v);
        const int prim_b = __float_as_int(v.w);
        bool hit = slot_moved(sv, prim_b) || (k >= 2 && slot_moved(sv, prim_a)) || (k == 1 && blocked1);
        if (!hit && sv.moved) {
          ++c_tested;
          hit = kExact ? seg_vs_moved(sv, s_cull, s_uni, false, test_old, a, b, wk)
                       : seg_vs_moved(sv, s_cull, s_uni, true, false, a, b, wk);
        }
        if (hit) {
          mask |= 1u << k;
          if (A.mode != PV_MODE_ERROR) break;
        }
        a = b;
        prim_a = prim_b;
      }
      if (mask) {
        if (A.mode != PV_MODE_ERROR) {
          const uint32_t first = __ffs(mask) - 1;
          if (first == 1) {
            A.info[p] = info_make(cell, 0, 0, true, true);     // keep light position and direction
            ++c_reemit;
          } else {
            A.info[p] = info_make(cell, first - 1, first - 1, true, false);
            ++c_tail;
          }
        } else {
          A.mask_out[p] = mask;
          want_cont = true;
        }
      }
    }
  }
  // append the error-mode candidates to the continuation list (one atomic per warp)
  const unsigned wm = __ballot_sync(0xffffffffu, want_cont);
  if (wm) {
    const int lane = threadIdx.x & 31, leader = __ffs(wm) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(A.cont_count, (uint32_t)__popc(wm));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want_cont) A.cont_list[base + __popc(wm & ((1u << lane) - 1u))] = p;
  }
  uint32_t* const ctr[6] = {field(A.stats, offsetof(pv_frame_stats, n_paths)),
                            field(A.stats, offsetof(pv_frame_stats, segments_tested)),
                            field(A.stats, offsetof(pv_frame_stats, vis_rays)),
                            field(A.stats, offsetof(pv_frame_stats, n_reemit)),
                            field(A.stats, offsetof(pv_frame_stats, n_tail)),
                            field(A.stats, offsetof(pv_frame_stats, n_cont))};
  const uint32_t val[6] = {p < n ? 1u : 0u, c_tested, c_vis, c_reemit, c_tail, want_cont ? 1u : 0u};
  block_add_n<6>(ctr, val, s_red);
  if (kPointVis || kExact) {
    block_add64(A.stats ? (unsigned long long*)&A.stats->node_visits : nullptr, wk.nodes, s_red64);
    block_add64(A.stats ? (unsigned long long*)&A.stats->tri_tests : nullptr, wk.tris, s_red64);
  }
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

// Alg. 1 for one path whose intersected segments are ``mask``.  Vertices are
// read from and updated in the path buffer as the loop advances; only the
// origin of the current segment (current and original position) is carried
// in registers.
__device__ void continue_path(const SceneView& sv, int root, const ContArgs& A, uint32_t p, uint32_t& c_rays,
                              uint32_t& c_tail, uint32_t& c_upd, uint32_t& c_trunc, Work& wk) {
  const uint32_t n = A.n;
  const uint32_t w = A.info[p];
  const uint32_t cell = w & PV_INFO_CELL_MASK;
  uint32_t nseg = min(info_nseg(w), sv.B);
  const uint32_t mask = A.mask[p];
  const float3 org = make_float3(A.origin[p], A.origin[n + p], A.origin[2 * (size_t)n + p]);
  auto vertex = [&](uint32_t k) -> float4 {        // stored vertex k (0 = origin)
    return k == 0 ? make_float4(org.x, org.y, org.z, __int_as_float(-1)) : A.pa[(size_t)(k - 1) * n + p];
  };
  uint32_t moved_origin = 0;
  bool updated = false, a_valid = false;
  int done = 0;
  float3 a_cur = org, a_orig = org;
  int a_prim = -1;
  uint32_t seg = __ffs(mask) - 1;
  while (seg <= nseg) {
    if (!((mask >> seg) & 1u) && !((moved_origin >> seg) & 1u)) {
      ++seg;
      a_valid = false;
      continue;
    }
    if (!a_valid) {
      const float4 v = vertex(seg - 1);
      a_cur = a_orig = f3(v);
      a_prim = __float_as_int(v.w);
    }
    const float4 bv = vertex(seg);
    const float3 b = f3(bv);
    const int b_prim = __float_as_int(bv.w);
    const float3 d = normalize_exact(b - a_cur);
    const Ray r = make_ray(a_cur, d, sv.tmin);
    Hit h;
    ++c_rays;
    if (!closest_hit(sv, root, r, seg == 1 ? -1 : a_prim, h, wk)) {   // escaped: the path ends here
      nseg = seg - 1;
      ++c_trunc;
      done = 1;
      break;
    }
    const Tri T = load_tri(sv.tris, h.tri);
    const int pn = __float_as_int(T.v0.w);
    const float3 xn = make_float3(fmaf(h.t, d.x, a_cur.x), fmaf(h.t, d.y, a_cur.y), fmaf(h.t, d.z, a_cur.z));
    const bool close = pn == b_prim && maxabs3(xn - b) <= sv.close_tol;
    if (seg == nseg) {                                                  // last photon: move it
      A.pa[(size_t)(seg - 1) * n + p] = make_float4(xn.x, xn.y, xn.z, __int_as_float(pn));
      updated = true;
      done = 1;
      break;
    }
    const float4 cv = vertex(seg + 1);                                  // stored next photon
    const float3 c = f3(cv);
    const float3 EO = f3(A.pb[(size_t)seg * n + p]);
    float3 EN = EO;
    if (!close) {
      const float4 albn = __ldg(sv.prim_alb + pn);
      const float3 nn = normalize(cross(f3(T.e1), f3(T.e2)));
      const float3 nsn = dot(nn, d) < 0.0f ? nn : -1.0f * nn;
      const float3 wv = c - xn;
      const float wl = sqrtf(dot(wv, wv));
      const float cosn = wl > 0.0f ? fmaxf(0.0f, dot(nsn, (1.0f / wl) * wv)) : 0.0f;
      const float4 albo = __ldg(sv.prim_alb + b_prim);
      const float3 no = normalize(prim_normal(sv, b_prim, true));
      const float3 dino = normalize_exact(b - a_orig);
      const float3 nso = dot(no, dino) < 0.0f ? no : -1.0f * no;
      const float coso = dot(nso, normalize_exact(c - b));
      const float3 Ei = f3(A.pb[(size_t)(seg - 1) * n + p]);
      const float f = coso > 0.0f ? cosn / (albo.w * coso) : 0.0f;
      EN = make_float3(Ei.x * albn.x * f, Ei.y * albn.y * f, Ei.z * albn.z * f);
    }
    if (!energy_close(EN, EO, A.tau)) {                                // Eq. 2 fails: re-trace from here
      A.pa[(size_t)(seg - 1) * n + p] = make_float4(xn.x, xn.y, xn.z, __int_as_float(pn));
      A.info[p] = info_make(cell, seg, seg, true, false);
      ++c_tail;
      done = 2;
      break;
    }
    if (close && !((mask >> (seg + 1)) & 1u) && !slot_moved(sv, pn) && !slot_moved(sv, __float_as_int(cv.w))) {
      seg += 2;                                                         // next segment known valid
      a_valid = false;
      continue;
    }
    A.pa[(size_t)(seg - 1) * n + p] = make_float4(xn.x, xn.y, xn.z, __int_as_float(pn));
    a_cur = xn;                                                         // origin of the next segment moved
    a_orig = b;
    a_prim = pn;
    a_valid = true;
    updated = true;
    moved_origin |= 1u << (seg + 1);
    ++seg;
  }
  if (done != 2) {
    A.info[p] = info_make(cell, nseg, 0, false, false);
    if (updated) ++c_upd;
  }
}

__global__ void __launch_bounds__(128) k_continue(SceneView sv, ContArgs A) {
  __shared__ uint32_t s_red[32 * 4];
  __shared__ unsigned long long s_red64[32];
  const int root = *sv.root;
  const uint32_t total = *A.count;
  const int lane = threadIdx.x & 31;
  uint32_t c_rays = 0, c_tail = 0, c_upd = 0, c_trunc = 0;
  Work wk;
  for (uint32_t guard = 0; guard < (1u << 26); ++guard) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(A.ticket, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= total) break;
    const uint32_t i = base + lane;
    if (i < total) continue_path(sv, root, A, A.list[i], c_rays, c_tail, c_upd, c_trunc, wk);
    __syncwarp();
  }
  uint32_t* const ctr[4] = {A.stats ? &A.stats->cont_rays : nullptr, A.stats ? &A.stats->n_tail : nullptr,
                            A.stats ? &A.stats->n_updated : nullptr, A.stats ? &A.stats->n_truncated : nullptr};
  const uint32_t val[4] = {c_rays, c_tail, c_upd, c_trunc};
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

extern "C" int pv_verify_paths(pv_scene* s, const pv_paths* paths, const pv_verify_params* params, uint32_t* d_list,
                               uint32_t* d_count, pv_frame_stats* d_stats, void* stream) {
  int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!params || !d_list || !d_count) return PV_ERR_ARG;
  if (params->mode < PV_MODE_NAIVE_AABB || params->mode > PV_MODE_ERROR || !(params->tau >= 0.0f)) return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  const uint32_t n = paths->n;
  const SceneView sv = pvh::view(s);
  const FrameLights L = pvh::frame_lights(s);
  if (cudaMemsetAsync(s->ws_ctr, 0, 16 * sizeof(uint32_t), st) != cudaSuccess) return PV_ERR_CUDA;
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
  if (n) {
    bool point_vis = false;
    for (uint32_t l = 0; l < s->n_lights; ++l)
      if (((L.moved_mask >> l) & 1u) && s->lights_new[l].type == PV_LIGHT_POINT) point_vis = true;
    const bool exact = params->mode == PV_MODE_NAIVE_EXACT ||
                       (params->mode == PV_MODE_ERROR && (params->flags & PV_FLAG_ERROR_EXACT));
    const dim3 grid((n + pvh::kVerifyThreads - 1) / pvh::kVerifyThreads);
    if (point_vis && exact) k_verify<true, true><<<grid, pvh::kVerifyThreads, 0, st>>>(sv, L, A);
    else if (point_vis) k_verify<true, false><<<grid, pvh::kVerifyThreads, 0, st>>>(sv, L, A);
    else if (exact) k_verify<false, true><<<grid, pvh::kVerifyThreads, 0, st>>>(sv, L, A);
    else k_verify<false, false><<<grid, pvh::kVerifyThreads, 0, st>>>(sv, L, A);
  }
  if (n && params->mode == PV_MODE_ERROR && (s->moved || L.moved_mask)) {
    if (!s->cont_blocks) {
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_continue, 128, 0);
      s->cont_blocks = (per > 0 ? per : 1) * s->num_sms;
    }
    ContArgs C;
    C.n = n;
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
    k_continue<<<s->cont_blocks, 128, 0, st>>>(sv, C);
  }
  pvh::launch_compact(s, paths->info, n, d_list, d_count, d_stats ? &d_stats->n_listed : nullptr, st);
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}
