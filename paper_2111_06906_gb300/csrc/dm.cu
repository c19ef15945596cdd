// Distribution maps (Sec. 3.1), the steps after "compute DM_C" (which is
// fused with the origin update in the verify kernel, as in Sec. 4):
//   prune paths (Eq. 1) in two passes (Sec. 4): k_dm_prune marks, reading the
//     counts as computed; k_dm_commit edits the counts and flags the free
//     paths (pruned, or no longer from the light);
//   the free paths are compacted into an ascending list;
//   fill DM_C: k_dm_deficit + an exclusive scan give each cell's range of
//     deficit slots; k_dm_fill gives the j-th free path of a light the cell
//     whose range holds j (any further ones spread evenly) and counts it.
// Every decision is an integer one (counts, the 24-bit draw), so the result
// does not depend on the order of the atomics.
#include "dm_core.cuh"
#include "pv_scene.h"

using namespace pvk;

namespace {

__global__ void k_dm_reset(DmLight D) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < D.cells; c += gridDim.x * blockDim.x)
    D.dmc[c] = dm_target(D, c);
}

// Pass 1 (dm_prune_path), flag[p] = 1 for a pruned path.
__global__ void __launch_bounds__(256) k_dm_prune(FrameLights L, uint32_t n, uint32_t* info, uint32_t* flag,
                                                  uint64_t seed, uint32_t frame, pv_frame_stats* stats) {
  __shared__ uint32_t s_red[32];
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t pruned = 0;
  if (p < n) {
    pruned = dm_prune_path(L, p, info, seed, frame);
    flag[p] = pruned;
  }
  uint32_t* const ctr[1] = {stats ? &stats->n_pruned : nullptr};
  const uint32_t val[1] = {pruned};
  block_add_n<1>(ctr, val, s_red);
}

// Pass 2 (dm_commit_path): the pruned paths leave their cells; every fresh
// emission of a light with a moved map is flagged free (bit 30, for the
// compaction) and counted.
__global__ void __launch_bounds__(256) k_dm_commit(FrameLights L, uint32_t n, const uint32_t* info, uint32_t* flag,
                                                   uint32_t* free_count) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  flag[p] = dm_commit_path(L, p, info, flag[p], free_count);
}

__global__ void k_dm_deficit(DmLight D, uint32_t* def) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= D.cells; c += gridDim.x * blockDim.x)
    def[c] = dm_deficit(D, c);
}

// Fill (dm_fill_path) for the free paths of light l, listed after those of
// the lights before it.
__global__ void __launch_bounds__(256) k_dm_fill(FrameLights L, uint32_t l, const uint32_t* free_list,
                                                 const uint32_t* free_count, const uint32_t* pre, uint32_t* info,
                                                 pv_frame_stats* stats) {
  __shared__ uint32_t s_red[32];
  const DmLight& D = L.dm[l];
  const uint32_t F = free_count[l];
  uint32_t off = 0;
  for (uint32_t k = 0; k < l; ++k) off += free_count[k];
  uint32_t filled = 0;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < F; j += gridDim.x * blockDim.x) {
    dm_fill_path(D, l, free_list[off + j], j, F, pre, info);
    ++filled;
  }
  uint32_t* const ctr[1] = {stats ? &stats->n_filled : nullptr};
  const uint32_t val[1] = {filled};
  block_add_n<1>(ctr, val, s_red);
}

}  // namespace

namespace pvh {

void dm_reset(pv_scene* s, cudaStream_t st) {
  const FrameLights L = frame_lights(s);
  for (uint32_t l = 0; l < s->n_lights; ++l)
    if (L.dm[l].dims) k_dm_reset<<<(L.dm[l].cells + 255) / 256, 256, 0, st>>>(L.dm[l]);
}

int dm_frame(pv_scene* s, const pv_paths* p, const FrameLights& L, const pv_verify_params* prm, pv_frame_stats* stats,
             cudaStream_t st) {
  uint32_t moved = 0;
  for (uint32_t l = 0; l < s->n_lights; ++l)
    if (L.dm[l].dims && ((L.moved_mask >> l) & 1u)) moved |= 1u << l;
  if (!moved || p->n == 0) return PV_OK;
  const uint32_t n = p->n, blocks = (n + 255) / 256;
  PV_CHECK(cudaMemsetAsync(s->dm_ctr, 0, 8 * sizeof(uint32_t), st));
  k_dm_prune<<<blocks, 256, 0, st>>>(L, n, p->info, s->dm_flag, prm->seed, prm->frame, stats);
  k_dm_commit<<<blocks, 256, 0, st>>>(L, n, p->info, s->dm_flag, s->dm_ctr);
  launch_compact(s, s->dm_flag, n, s->dm_free, s->dm_ctr + 4, nullptr, st);
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    if (!((moved >> l) & 1u)) continue;
    const DmLight& D = L.dm[l];
    k_dm_deficit<<<(D.cells + 256) / 256, 256, 0, st>>>(D, s->dm_scan);
    exclusive_scan(s->dm_scan, D.cells + 1, st);
    const uint32_t fb = std::min<uint32_t>((s->lights_new[l].n_paths + 255) / 256, 8u * (uint32_t)s->num_sms);
    k_dm_fill<<<std::max<uint32_t>(fb, 1u), 256, 0, st>>>(L, l, s->dm_free, s->dm_ctr, s->dm_scan, p->info, stats);
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace pvh
