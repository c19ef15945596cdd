// Scene construction, per-frame pose update and status handling (C ABI).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "pv_scene.h"

using namespace pvk;

namespace {

__global__ void k_invert(const uint32_t* tri_prim, uint32_t n, uint32_t* prim_dyn) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) prim_dyn[tri_prim[i]] = i;
}

bool same_pose(const pv_light& a, const pv_light& b) {
  return std::memcmp(a.pos, b.pos, sizeof a.pos) == 0 && std::memcmp(a.normal, b.normal, sizeof a.normal) == 0 &&
         std::memcmp(a.tangent, b.tangent, sizeof a.tangent) == 0 && std::memcmp(a.size, b.size, sizeof a.size) == 0;
}

LightPose to_pose(const pv_light& l) {
  LightPose p;
  p.type = l.type;
  p.pos = make_float3(l.pos[0], l.pos[1], l.pos[2]);
  p.n = make_float3(l.normal[0], l.normal[1], l.normal[2]);
  p.t = make_float3(l.tangent[0], l.tangent[1], l.tangent[2]);
  // bitangent = normal x tangent, in double then rounded once
  const double n0 = l.normal[0], n1 = l.normal[1], n2 = l.normal[2];
  const double t0 = l.tangent[0], t1 = l.tangent[1], t2 = l.tangent[2];
  p.b = make_float3((float)(n1 * t2 - n2 * t1), (float)(n2 * t0 - n0 * t2), (float)(n0 * t1 - n1 * t0));
  p.size = make_float2(l.size[0], l.size[1]);
  p.power = make_float3(l.power[0], l.power[1], l.power[2]);
  p.n_paths = l.n_paths;
  return p;
}

int check_lights(const pv_light* l, uint32_t n) {
  for (uint32_t i = 0; i < n; ++i) {
    if (l[i].type != PV_LIGHT_POINT && l[i].type != PV_LIGHT_RECT) return PV_ERR_ARG;
    if (l[i].n_paths == 0) return PV_ERR_ARG;
  }
  return PV_OK;
}

void free_scene(pv_scene* s) {
  if (!s) return;
  for (cudaEvent_t e : s->stage_ev)
    if (e) cudaEventDestroy(e);
  void* ptrs[] = {s->nodes, s->wnodes, s->wsrc, s->wcount, s->cq, s->tris, s->root, s->d_local, s->d_tri_prim, s->d_leaf_parent, s->d_node_parent,
                  s->d_fit_flags, s->w_link, s->w_nch, s->w_arrive, s->t_link, s->pair_link, s->pair_tri, s->pair_warps, s->pair_acc, s->pair_count, s->obox, s->d_tri_slot, s->objs, s->groups, s->r_keys[0], s->r_keys[1], s->r_vals[0], s->r_vals[1],
                  s->r_hist, s->r_tris, s->r_local, s->r_prim, s->prim_slot, s->prim_dyn, s->prim_alb, s->prim_nrm,
                  s->xf_old, s->xf_new, s->ws_mask, s->ws_cont, s->ws_list, s->ws_touched, s->ws_tiles, s->ws_ctr, s->status, s->b_keys[0], s->b_keys[1],
                  s->b_vals[0], s->b_vals[1], s->b_hist, s->dm_c[0], s->dm_c[1], s->dm_c[2], s->dm_c[3],
                  s->dm_flag, s->dm_free, s->dm_scan, s->dm_ctr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
}

}  // namespace

namespace pvh {

SceneView view(const pv_scene* s) {
  SceneView v;
  v.nodes = s->wnodes;
  v.tris = s->tris;
  v.root = s->root;
  v.objs = s->objs;
  v.groups = s->groups;
  v.n_dyn = s->n_dyn;
  v.prim_slot = s->prim_slot;
  v.prim_dyn = s->prim_dyn;
  v.prim_alb = s->prim_alb;
  v.prim_nrm = s->prim_nrm;
  v.d_local = s->d_local;
  v.xf_old = s->xf_old;
  v.xf_new = s->xf_new;
  v.B = s->B;
  v.tmin = s->tmin;
  v.close_tol = s->close_tol;
  v.moved = s->moved;
  v.max_visits = s->visit_limit ? s->visit_limit : 2u * (s->n_static_refs + s->n_dyn_tris) + 256u;
  v.status = s->status;
  v.n_static_wide = s->w_dyn_off;
  return v;
}

FrameLights frame_lights(const pv_scene* s) {
  FrameLights L;
  std::memset(&L, 0, sizeof L);
  L.n = s->n_lights;
  L.first[0] = 0;
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    L.cur[l] = to_pose(s->lights_new[l]);
    L.old[l] = to_pose(s->lights_old[l]);
    L.first[l + 1] = L.first[l] + s->lights_new[l].n_paths;
    if (!same_pose(s->lights_old[l], s->lights_new[l])) L.moved_mask |= 1u << l;
    if (std::memcmp(s->lights_old[l].normal, s->lights_new[l].normal, sizeof(float) * 3) != 0) L.tilted_mask |= 1u << l;
  }
  for (uint32_t l = s->n_lights; l < PV_MAX_LIGHTS; ++l) L.first[l + 1] = L.first[l];
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    DmLight& D = L.dm[l];
    D.dims = s->dm_dims[l];
    D.cells = s->dm_cells[l];
    D.n_paths = s->lights_new[l].n_paths;
    D.dmc = s->dm_c[l];
    for (int k = 0; k < 4; ++k) D.res[k] = s->dm_res[l][k];
  }
  return L;
}

}  // namespace pvh

extern "C" int pv_build_scene(const pv_scene_desc* d, void* stream, pv_scene** out) {
  if (!out) return PV_ERR_ARG;
  *out = nullptr;
  if (!d || !d->verts || !d->tri_object || !d->object_dynamic || !d->object_albedo || !d->lights) return PV_ERR_ARG;
  if (d->n_tris == 0 || d->n_objects == 0 || d->n_lights == 0) return PV_ERR_ARG;
  if (!(d->scene_diag > 0.f) || !std::isfinite(d->scene_diag)) return PV_ERR_ARG;
  if (d->n_lights > PV_MAX_LIGHTS || d->max_bounces == 0 || d->max_bounces > PV_MAX_BOUNCES) return PV_ERR_LIMIT;
  if (check_lights(d->lights, d->n_lights) != PV_OK) return PV_ERR_ARG;
  uint64_t total = 0;
  for (uint32_t l = 0; l < d->n_lights; ++l) total += d->lights[l].n_paths;
  if (total >= (1ull << 31)) return PV_ERR_LIMIT;
  for (uint32_t t = 0; t < d->n_tris; ++t)
    if (d->tri_object[t] >= d->n_objects) return PV_ERR_ARG;
  if (d->n_tris >= (1u << 31)) return PV_ERR_LIMIT;

  uint32_t dm_res[PV_MAX_LIGHTS][4] = {}, dm_dims[PV_MAX_LIGHTS] = {}, dm_cells[PV_MAX_LIGHTS] = {};
  for (uint32_t l = 0; l < d->n_lights; ++l) {
    const bool rect = d->lights[l].type == PV_LIGHT_RECT;
    const uint32_t dims = rect ? 4u : 2u;
    uint64_t cells = 1;
    for (uint32_t k = 0; k < dims; ++k) {
      const uint32_t r = rect ? d->dm_rect[k] : d->dm_point[k];
      dm_res[l][k] = r;
      cells *= r;
    }
    if (cells == 0) continue;                  // no map for this light
    if (cells > (1u << 20)) return PV_ERR_LIMIT;
    dm_dims[l] = dims;
    dm_cells[l] = (uint32_t)cells;
  }
  cudaStream_t st = (cudaStream_t)stream;
  pv_scene* s = new pv_scene;
  s->flags = d->flags;
  uint32_t dm_max = 0;
  for (uint32_t l = 0; l < PV_MAX_LIGHTS; ++l) {
    for (int k = 0; k < 4; ++k) s->dm_res[l][k] = dm_res[l][k];
    s->dm_dims[l] = dm_dims[l];
    s->dm_cells[l] = dm_cells[l];
    if (dm_cells[l]) s->has_dm = true;
    dm_max = std::max(dm_max, dm_cells[l]);
  }
  s->n_tris = d->n_tris;
  s->n_objects = d->n_objects;
  s->B = d->max_bounces;
  s->diag = d->scene_diag;
  s->tmin = 1e-5f * d->scene_diag;
  s->close_tol = 1e-5f * d->scene_diag;
  s->n_lights = d->n_lights;
  s->n_paths_total = (uint32_t)total;
  for (uint32_t l = 0; l < d->n_lights; ++l) s->lights_old[l] = s->lights_new[l] = d->lights[l];
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
    delete s;
    return PV_ERR_CUDA;
  }

  // slots of the dynamic objects, in object order
  std::vector<int> slot_of(d->n_objects, -1);
  for (uint32_t o = 0; o < d->n_objects; ++o)
    if (d->object_dynamic[o]) {
      if (s->n_dyn == PV_MAX_DYN_OBJECTS) {
        delete s;
        return PV_ERR_LIMIT;
      }
      slot_of[o] = (int)s->n_dyn++;
      s->dyn_object.push_back(o);
    }
  s->dyn_tris_of.assign(s->n_dyn, {});
  s->h_objs.assign(s->n_dyn, DynObj{});
  std::vector<uint32_t> static_prims;
  std::vector<uint8_t> pslot(d->n_tris, 255);
  std::vector<float4> palb(d->n_tris), pnrm(d->n_tris);
  for (uint32_t t = 0; t < d->n_tris; ++t) {
    const uint32_t o = d->tri_object[t];
    const float* a = d->object_albedo + 3 * (size_t)o;
    palb[t] = make_float4(a[0], a[1], a[2], std::fmax(a[0], std::fmax(a[1], a[2])));
    const float* v = d->verts + 9 * (size_t)t;
    const double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
    const double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
    pnrm[t] = make_float4((float)(e1[1] * e2[2] - e1[2] * e2[1]), (float)(e1[2] * e2[0] - e1[0] * e2[2]),
                          (float)(e1[0] * e2[1] - e1[1] * e2[0]), 0.f);
    if (slot_of[o] >= 0) {
      pslot[t] = (uint8_t)slot_of[o];
      s->dyn_tris_of[slot_of[o]].push_back(t);
      s->n_dyn_tris++;
    } else {
      static_prims.push_back(t);
    }
  }
  for (uint32_t sl = 0; sl < s->n_dyn; ++sl) s->h_objs[sl].user_object = s->dyn_object[sl];
  // initial poses
  s->h_xf_new.assign(12 * (size_t)s->n_dyn, 0.f);
  for (uint32_t sl = 0; sl < s->n_dyn; ++sl) {
    float* x = &s->h_xf_new[12 * sl];
    if (d->object_xform) {
      std::memcpy(x, d->object_xform + 12 * (size_t)s->dyn_object[sl], 12 * sizeof(float));
    } else {
      x[0] = x[5] = x[10] = 1.f;
    }
  }
  s->h_xf_old = s->h_xf_new;

  int rc = PV_OK;
  auto fail = [&](cudaError_t e) { if (e != cudaSuccess && rc == PV_OK) rc = e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA; };
  fail(cudaMalloc(&s->prim_slot, d->n_tris));
  fail(cudaMalloc(&s->prim_dyn, d->n_tris * sizeof(uint32_t)));
  fail(cudaMalloc(&s->prim_alb, d->n_tris * sizeof(float4)));
  fail(cudaMalloc(&s->prim_nrm, d->n_tris * sizeof(float4)));
  fail(cudaMalloc(&s->xf_old, kMaxDyn * 12 * sizeof(float)));
  fail(cudaMalloc(&s->xf_new, kMaxDyn * 12 * sizeof(float)));
  fail(cudaMalloc(&s->status, sizeof(int)));
  fail(cudaMalloc(&s->ws_ctr, 16 * sizeof(uint32_t)));
  s->n_tiles = (s->n_paths_total + pvh::kTile - 1) / pvh::kTile;
  fail(cudaMalloc(&s->ws_mask, (size_t)s->n_paths_total * sizeof(uint32_t)));
  fail(cudaMalloc(&s->ws_cont, (size_t)s->n_paths_total * sizeof(uint32_t)));
  fail(cudaMalloc(&s->ws_list, (size_t)s->n_paths_total * sizeof(uint32_t)));
  fail(cudaMalloc(&s->ws_touched, (size_t)s->n_paths_total));
  fail(cudaMalloc(&s->ws_tiles, (size_t)(s->n_tiles + 1) * sizeof(uint64_t)));
  for (uint32_t l = 0; l < PV_MAX_LIGHTS; ++l)
    if (s->dm_cells[l]) {
      fail(cudaMalloc(&s->dm_c[l], (size_t)s->dm_cells[l] * sizeof(uint32_t)));
      if (s->dm_c[l]) fail(cudaMemsetAsync(s->dm_c[l], 0, (size_t)s->dm_cells[l] * sizeof(uint32_t), st));
    }
  if (s->has_dm) {
    fail(cudaMalloc(&s->dm_flag, (size_t)s->n_paths_total * sizeof(uint32_t)));
    fail(cudaMalloc(&s->dm_free, (size_t)s->n_paths_total * sizeof(uint32_t)));
    fail(cudaMalloc(&s->dm_scan, ((size_t)dm_max + 1) * sizeof(uint32_t)));
    fail(cudaMalloc(&s->dm_ctr, 8 * sizeof(uint32_t)));
  }
  for (int b = 0; b < 2; ++b) {
    fail(cudaMalloc(&s->b_keys[b], (size_t)s->n_paths_total * sizeof(uint64_t)));
    fail(cudaMalloc(&s->b_vals[b], (size_t)s->n_paths_total * sizeof(uint32_t)));
  }
  fail(cudaMalloc(&s->b_hist, 256 * (size_t)pvh::radix_tiles(s->n_paths_total) * sizeof(uint32_t)));
  if (rc != PV_OK) {
    free_scene(s);
    return rc;
  }
  fail(cudaMemcpyAsync(s->prim_slot, pslot.data(), d->n_tris, cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(s->prim_alb, palb.data(), d->n_tris * sizeof(float4), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(s->prim_nrm, pnrm.data(), d->n_tris * sizeof(float4), cudaMemcpyHostToDevice, st));
  fail(cudaMemsetAsync(s->prim_dyn, 0xff, d->n_tris * sizeof(uint32_t), st));
  fail(cudaMemsetAsync(s->xf_old, 0, kMaxDyn * 12 * sizeof(float), st));
  fail(cudaMemsetAsync(s->xf_new, 0, kMaxDyn * 12 * sizeof(float), st));
  fail(cudaMemsetAsync(s->status, 0, sizeof(int), st));
  fail(cudaMemsetAsync(s->ws_ctr, 0, 16 * sizeof(uint32_t), st));
  s->n_static = (uint32_t)static_prims.size();
  if (rc == PV_OK) rc = pvh::build_bvh(s, d->verts, static_prims, st);
  if (rc == PV_OK) {
    // world triangles, boxes and top level of the initial pose, then make it the old pose too
    s->moved = s->n_dyn == 64 ? ~0ull : ((1ull << s->n_dyn) - 1ull);
    pvh::launch_update_dynamic(s, st);
    s->moved = 0;
    pvh::launch_update_dynamic(s, st);
    if (s->n_dyn_tris)
      k_invert<<<(s->n_dyn_tris + 255) / 256, 256, 0, st>>>(s->d_tri_prim, s->n_dyn_tris, s->prim_dyn);
    fail(cudaGetLastError());
  }
  if (rc == PV_OK) fail(cudaStreamSynchronize(st));
  if (rc == PV_OK) rc = pvh::build_refit_pairs(s, st);
  s->dyn_tris_of.clear();
  s->dyn_tris_of.shrink_to_fit();
  if (rc != PV_OK) {
    free_scene(s);
    return rc;
  }
  s->last_stream = st;
  *out = s;
  return PV_OK;
}

namespace pvh {

// Host half of a pose update: the new poses become current, the previous
// ones old, and the moved bits are found by bitwise comparison.
int stage_poses(pv_scene* s, const float* xforms, const pv_light* lights) {
  if (!s) return PV_ERR_ARG;
  if (lights) {
    if (check_lights(lights, s->n_lights) != PV_OK) return PV_ERR_ARG;
    for (uint32_t l = 0; l < s->n_lights; ++l)
      if (lights[l].n_paths != s->lights_new[l].n_paths) return PV_ERR_ARG;
  }
  s->h_xf_old = s->h_xf_new;
  uint64_t moved = 0;
  if (xforms)
    for (uint32_t sl = 0; sl < s->n_dyn; ++sl) {
      const float* x = xforms + 12 * (size_t)s->dyn_object[sl];
      if (std::memcmp(x, &s->h_xf_new[12 * sl], 12 * sizeof(float)) != 0) moved |= 1ull << sl;
      std::memcpy(&s->h_xf_new[12 * sl], x, 12 * sizeof(float));
    }
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    s->lights_old[l] = s->lights_new[l];
    if (lights) s->lights_new[l] = lights[l];
  }
  s->moved = moved;
  return PV_OK;
}

int stack_need(pv_scene* s, uint32_t* out) {
  if (!s || !out) return PV_ERR_ARG;
  if (!s->stack_need) {
    if (cudaStreamSynchronize(s->last_stream) != cudaSuccess) return PV_ERR_CUDA;
    int root = INT32_MIN;
    if (cudaMemcpy(&root, s->root, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PV_ERR_CUDA;
    std::vector<int4> ch(s->n_wide);
    if (s->n_wide && cudaMemcpy2D(ch.data(), sizeof(int4), &s->wnodes[0].child, sizeof(WNode), sizeof(int4), s->n_wide,
                                  cudaMemcpyDeviceToHost) != cudaSuccess)
      return PV_ERR_CUDA;
    // deepest root-to-leaf path, counted in wide nodes (iterative, bounded)
    uint32_t height = 0;
    std::vector<std::pair<int, uint32_t>> todo;
    if (root >= 0) todo.push_back({root, 1u});
    for (size_t guard = 0; !todo.empty() && guard < 4 * (size_t)s->n_wide + 16; ++guard) {
      const auto [node, depth] = todo.back();
      todo.pop_back();
      if (node < 0 || (uint32_t)node >= s->n_wide) continue;
      height = std::max(height, depth);
      const int c[4] = {ch[node].x, ch[node].y, ch[node].z, ch[node].w};
      for (int k = 0; k < 4; ++k)
        if (c[k] >= 0) todo.push_back({c[k], depth + 1});
    }
    s->stack_need = std::max<uint32_t>(3 * height, 1);
  }
  *out = s->stack_need;
  return PV_OK;
}

}  // namespace pvh

extern "C" int pv_update_dynamic(pv_scene* s, const float* xforms, const pv_light* lights, void* stream) {
  const int rc = pvh::stage_poses(s, xforms, lights);
  if (rc != PV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t moved = s->moved;
  pvh::launch_update_dynamic(s, st);
  if (moved && (s->flags & PV_BUILD_DYN_REBUILD))
    k_invert<<<(s->n_dyn_tris + 255) / 256, 256, 0, st>>>(s->d_tri_prim, s->n_dyn_tris, s->prim_dyn);
  s->last_stream = st;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

extern "C" int pv_set_traversal_limit(pv_scene* s, uint32_t max_visits) {
  if (!s) return PV_ERR_ARG;
  s->visit_limit = max_visits;
  return PV_OK;
}

extern "C" int pv_distribution_map_cells(const pv_scene* s, uint32_t light) {
  if (!s || light >= s->n_lights) return PV_ERR_ARG;
  return (int)s->dm_cells[light];
}

extern "C" int pv_read_distribution_map(pv_scene* s, uint32_t light, uint32_t* h_counts) {
  if (!s || light >= s->n_lights || !h_counts) return PV_ERR_ARG;
  if (!s->dm_cells[light]) return PV_OK;
  if (cudaStreamSynchronize(s->last_stream) != cudaSuccess) return PV_ERR_CUDA;
  return pvh::cuda_status(cudaMemcpy(h_counts, s->dm_c[light], (size_t)s->dm_cells[light] * sizeof(uint32_t),
                                     cudaMemcpyDeviceToHost));
}

extern "C" int pv_read_device_status(pv_scene* s) {
  if (!s) return PV_ERR_ARG;
  if (cudaStreamSynchronize(s->last_stream) != cudaSuccess) return PV_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, s->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PV_ERR_CUDA;
  if (v != 0 && cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess) return PV_ERR_CUDA;
  return v;
}

extern "C" void pv_destroy_scene(pv_scene* s) {
  if (!s) return;
  cudaStreamSynchronize(s->last_stream);
  free_scene(s);
}

extern "C" const char* pv_status_string(int status) {
  switch (status) {
    case PV_OK: return "ok";
    case PV_ERR_ARG: return "invalid argument";
    case PV_ERR_CUDA: return "CUDA runtime error";
    case PV_ERR_OOM: return "out of device memory";
    case PV_ERR_STACK: return "BVH traversal stack overflow";
    case PV_ERR_ITER_CAP: return "iteration cap reached";
    case PV_ERR_LIMIT: return "format limit exceeded";
    case PV_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}
