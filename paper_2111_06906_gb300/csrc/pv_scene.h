// Host-side scene object and launch helpers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cstdlib>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "pv.h"
#include "pv_device.cuh"

struct pv_scene {
  int device = 0;
  int num_sms = 0;
  int verify_blocks_per_sm[4] = {0, 0, 0, 0};   // resident k_verify blocks per SM, by (point vis, exact)
  uint32_t n_tris = 0, n_objects = 0, n_static = 0, n_dyn_tris = 0, n_dyn = 0;
  uint32_t B = 0;
  float diag = 0.f, tmin = 0.f, close_tol = 0.f;
  uint32_t flags = 0;

  // shared BVH arrays: triangles [static references | dynamic]; binary nodes
  // [static | dynamic] (build and refit); wide nodes [static | dynamic | top] (traversal)
  pvk::Node* nodes = nullptr;
  pvk::WNode* wnodes = nullptr;
  pvk::Tri* tris = nullptr;
  int* root = nullptr;               // device word: wide root of the whole scene
  int32_t s_root = INT32_MIN;        // static binary root (child index)
  int32_t s_wroot = INT32_MIN;       // static wide root (reference)
  uint32_t n_static_refs = 0, d_tri_off = 0, d_node_off = 0;
  uint32_t w_dyn_off = 0, w_top_off = 0, n_wide = 0;
  int* wsrc = nullptr;               // [n_wide][4] binary slot of each wide child (refit source)
  uint32_t* wcount = nullptr;        // device: [0] static wide count, [1] dynamic wide count
  int* cq = nullptr;                 // collapse queues, 2 x [q_cap][2]
  uint32_t q_cap = 0;
  bool top_built = false;

  // dynamic objects (one LBVH over all dynamic triangles, keyed by slot first)
  float* d_local = nullptr;          // [n_dyn_tris][9] object-local corners, BVH order
  uint32_t* d_tri_prim = nullptr;    // [n_dyn_tris] primitive id, BVH order
  uint32_t* d_leaf_parent = nullptr; // [n_dyn_tris] parent << 1 | side
  uint32_t* d_node_parent = nullptr; // [n_dyn_tris] parent << 1 | side of internal nodes
  uint32_t* d_fit_flags = nullptr;   // [n_dyn_tris] arrival counters for the bottom-up pass
  // direct refit of the dynamic wide nodes (after the first collapse)
  uint32_t* w_link = nullptr;        // [n_dyn_tris] dynamic wide node -> parent (local << 2 | slot), ~0u at a root
  uint8_t* w_nch = nullptr;          // [n_dyn_tris] children in use per dynamic wide node
  uint32_t* w_arrive = nullptr;      // [n_dyn_tris] children refitted this frame (reset by the last), then the
                                     // refit's finished-block count
  uint32_t* t_link = nullptr;        // [n_dyn_tris] dynamic triangle -> parent wide node (local << 2 | slot)
  // pair table of the refit without dependent levels (k_refit_wide, refit_pair)
  uint32_t* pair_link = nullptr;     // [n_pairs] parent slot of the pair's wide node (| kPairOne)
  uint32_t* pair_tri = nullptr;      // [n_pairs] local dynamic triangle under the node
  uint32_t* pair_warps = nullptr;    // [4 x dynamic wide nodes] warps over each node's pairs, by parent slot
  int* pair_acc = nullptr;           // [4 x dynamic wide nodes][6] box of a node over several warps
  uint32_t* pair_count = nullptr;    // [4 x dynamic wide nodes] warps still to arrive
  uint32_t n_pairs = 0;
  bool pairs_ok = false;             // the table is built (else the refit climbs)
  int* obox = nullptr;               // [kMaxDyn][6] exact new boxes of the frame, order-preserving integers
  uint8_t* d_tri_slot = nullptr;     // [n_dyn_tris] slot per dynamic triangle
  pvk::DynObj* objs = nullptr;       // [n_dyn]
  pvk::MovedGroups* groups = nullptr;  // the moved objects' groups of this frame
  std::vector<pvk::DynObj> h_objs;
  std::vector<std::vector<uint32_t>> dyn_tris_of;   // slot -> primitive ids (build only)
  // rebuild scratch (PV_BUILD_DYN_REBUILD)
  uint64_t* r_keys[2] = {nullptr, nullptr};
  uint32_t* r_vals[2] = {nullptr, nullptr};
  uint32_t* r_hist = nullptr;
  pvk::Tri* r_tris = nullptr;
  float* r_local = nullptr;
  uint32_t* r_prim = nullptr;

  // per primitive
  uint8_t* prim_slot = nullptr;
  uint32_t* prim_dyn = nullptr;
  float4* prim_alb = nullptr;
  float4* prim_nrm = nullptr;        // [n_tris] e1 x e2 of the given corners (object-local for dynamic)

  // poses: host copies of the object table's dynamic transforms and lights
  std::vector<uint32_t> dyn_object;          // slot -> user object id
  std::vector<float> h_xf_old, h_xf_new;     // [n_dyn][12]
  float* xf_old = nullptr;                   // device [kMaxDyn][12]
  float* xf_new = nullptr;
  uint64_t moved = 0;
  uint32_t n_lights = 0;
  pv_light lights_old[PV_MAX_LIGHTS], lights_new[PV_MAX_LIGHTS];
  uint32_t n_paths_total = 0;

  // per-frame workspace
  uint32_t* ws_mask = nullptr;       // [n_paths] intersected-segment masks (error mode)
  uint32_t* ws_cont = nullptr;       // [n_paths] continuation list
  uint32_t* ws_list = nullptr;       // [n_paths] re-trace list of pv_verify_retrace
  uint8_t* ws_touched = nullptr;     // [n_paths] paths the frame re-traces or hands to Alg. 1 (fused deposit)
  uint64_t* ws_tiles = nullptr;      // [n_tiles + 1] decoupled look-back tile states
  uint32_t n_tiles = 0;
  uint32_t* ws_ctr = nullptr;        // [16] work counters
  // distribution maps (Sec. 3.1), per light; workspace shared by the lights
  uint32_t dm_res[PV_MAX_LIGHTS][4] = {};
  uint32_t dm_dims[PV_MAX_LIGHTS] = {}, dm_cells[PV_MAX_LIGHTS] = {};
  uint32_t* dm_c[PV_MAX_LIGHTS] = {};         // DM_C [cells]
  uint32_t* dm_flag = nullptr;                // [n_paths] pruned mark, then free-path flags
  uint32_t* dm_free = nullptr;                // [n_paths] free paths, ascending
  uint32_t* dm_scan = nullptr;                // [max cells + 1] deficits, then their exclusive prefix
  uint32_t* dm_ctr = nullptr;                 // [8] free paths per light, free-list length
  bool has_dm = false;
  uint64_t* b_keys[2] = {nullptr, nullptr};   // [n_paths] budget ranking sort keys (ping-pong)
  uint32_t* b_vals[2] = {nullptr, nullptr};
  uint32_t* b_hist = nullptr;                 // [256][radix tiles of n_paths]
  int* status = nullptr;             // sticky device status
  cudaStream_t last_stream = nullptr;

  int verify_blocks = 0, trace_blocks = 0, trace_dep_blocks = 0, cont_blocks = 0, cont_trace_blocks = 0,
      cont_trace_dep_blocks = 0, cont_trace_delta_blocks = 0;
  // stage timing of pv_verify_retrace: a ring of stage_n calls, pvh::kStageEvents events each
  std::vector<cudaEvent_t> stage_ev;
  uint32_t stage_n = 0, stage_next = 0, stage_count = 0;
  uint32_t visit_limit = 0;          // 0 = default cap (see view())
  uint32_t stack_need = 0;           // traversal stack entries the wide tree can need (0 = not yet measured)
};

namespace pvk {
struct ContArgs;                     // verify_core.cuh
}

namespace pvh {

constexpr int kStageEvents = 5;      // events per timed pv_verify_retrace call
constexpr int kTraceThreads = 128;
constexpr int kVerifyThreads = 256;
constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 16;    // paths per thread in the compaction tile
constexpr uint32_t kTile = kCompactThreads * kCompactItems;

// Verify blocks for a tile loop: ``resident``, or fewer when the environment
// variable PV_VERIFY_MAX_BLOCKS asks for fewer (testing and tuning).
inline uint32_t verify_block_cap(uint32_t resident) {
  if (const char* e = std::getenv("PV_VERIFY_MAX_BLOCKS")) {
    const long m = std::strtol(e, nullptr, 10);
    if (m > 0 && (uint32_t)m < resident) return (uint32_t)m;
  }
  return resident;
}

// work counter slots in ws_ctr
enum { CTR_CONT = 0, CTR_TRACE = 1, CTR_TILE = 2, CTR_ALL = 3, CTR_LIST = 4 };

pvk::SceneView view(const pv_scene* s);
pvk::FrameLights frame_lights(const pv_scene* s);
// scene.cu: host half of pv_update_dynamic (validation, pose bookkeeping, moved bits)
int stage_poses(pv_scene* s, const float* xforms, const pv_light* lights);
// scene.cu: traversal stack entries the scene's wide tree can need (three per
// wide node on its deepest root-to-leaf path), measured once (synchronous)
int stack_need(pv_scene* s, uint32_t* out);

// dm.cu: distribution maps.  dm_reset sets DM_C = DM_T for every light with a
// map; dm_frame runs count-independent steps after verification of a frame in
// which lights with maps moved (prune, edit, free list, fill).
void dm_reset(pv_scene* s, cudaStream_t st);
int dm_frame(pv_scene* s, const pv_paths* p, const pvk::FrameLights& L, const pv_verify_params* prm,
             pv_frame_stats* stats, cudaStream_t st);

// bvh.cu
// exclusive prefix sum of m counters in place (one block)
void exclusive_scan(uint32_t* data, uint32_t m, cudaStream_t st);
// stable LSD radix sort of (key, value) pairs on key bits [lo_bit, hi_bit);
// the buffers swap so that k0/v0 hold the result; hist holds 256 * radix_tiles(n)
void radix_sort(uint64_t*& k0, uint32_t*& v0, uint64_t*& k1, uint32_t*& v1, uint32_t n, uint32_t* hist, int lo_bit,
                int hi_bit, cudaStream_t st);
uint32_t radix_tiles(uint32_t n);
int build_bvh(pv_scene* s, const float* h_verts, const std::vector<uint32_t>& static_prims, cudaStream_t st);
void launch_update_dynamic(pv_scene* s, cudaStream_t st);
int build_refit_pairs(pv_scene* s, cudaStream_t st);

// compact.cu
void launch_compact(pv_scene* s, const uint32_t* info, uint32_t n, uint32_t* list, uint32_t* count,
                    uint32_t* stats_listed, cudaStream_t st);

// trace.cu
// k_trace over ``list`` (nullptr: every path from its light); with an atlas,
// every photon stored is also deposited into it (the atlas is not cleared here).
void launch_trace(pv_scene* s, const pv_paths* p, const uint32_t* list, const uint32_t* count, uint64_t seed,
                  uint32_t frame, pv_frame_stats* stats, cudaStream_t st, const pv_atlas* atlas = nullptr);
// Alg. 1 over the continuation list C fused with the re-trace of ``list``;
// with an atlas, every path is also deposited (touched: verification's marks;
// delta: the atlas holds the entry records' deposit, only listed paths change it)
void launch_cont_trace(pv_scene* s, const pv_paths* p, const pvk::ContArgs& C, const uint32_t* list,
                       const uint32_t* count, uint64_t seed, uint32_t frame, pv_frame_stats* stats,
                       const pv_atlas* atlas, const uint8_t* touched, bool delta, cudaStream_t st);
// deposit.cu: argument checks of an atlas, and the plain deposit of every path
int check_atlas(const pv_atlas* a);
void launch_deposit(pv_scene* s, const pv_paths* p, const pv_atlas* a, cudaStream_t st);

// verify.cu: argument checks shared by the entry points
int check_paths(const pv_scene* s, const pv_paths* p);

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? PV_OK : PV_ERR_CUDA; }

}  // namespace pvh

#define PV_CHECK(call)                         \
  do {                                         \
    cudaError_t _e = (call);                   \
    if (_e != cudaSuccess) return PV_ERR_CUDA; \
  } while (0)
