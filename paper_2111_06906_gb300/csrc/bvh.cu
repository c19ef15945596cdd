// Morton-code LBVH construction, refit, per-frame rebuild and top level.
//
// All triangles and nodes live in two arrays shared by every tree:
//   triangles: [static references | dynamic triangles]
//   nodes:     [static tree | dynamic tree | top level]
// Child indices are global (>= 0 internal node, ~i leaf = triangle i), so a
// query walks the top level, the static tree and the dynamic objects' trees
// in one traversal.
//
// Static build: oversized triangles are first split into references, each
// bounded by the part of the triangle inside one cell of a grid over the
// triangle's box (polygon clipping), so a few huge triangles (a floor) cannot
// inflate the boxes of their ancestors.  Then: 63-bit Morton keys of the
// reference centroids, a stable LSD radix sort (8-bit digits, per-warp stable
// ranks), the binary radix tree of Karras ("Maximizing parallelism in the
// construction of BVHs, octrees and k-d trees", HPG 2012) with index
// tie-break for equal keys, and a bottom-up box pass in which the second child
// to arrive at a node builds the union.
//
// Dynamic objects share one tree keyed by (slot, 57-bit Morton code of the
// object-local centroid): slots occupy the top key bits, so each object's
// triangles form one subtree whose root is recorded per slot.  Every frame the
// moved objects are transformed and the tree is refitted (or rebuilt from
// world-space keys), then the top level over the static root and the object
// roots is rebuilt by a median split.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "update_core.cuh"

namespace pvk {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ uint64_t spread_bits(uint32_t v, int bits) {
  uint64_t x = 0;
  for (int i = 0; i < bits; ++i) x |= (uint64_t)((v >> i) & 1u) << (3 * i);
  return x;
}

__device__ __forceinline__ uint32_t quantize(float v, float lo, float ext, int bits) {
  const float f = ext > 0.f ? (v - lo) / ext : 0.5f;
  const float m = (float)(1u << bits);
  const float q = fminf(fmaxf(f * m, 0.0f), m - 1.0f);
  return (uint32_t)q;
}

__device__ __forceinline__ uint64_t morton(float3 c, const float* lo, const float* ext, int bits) {
  return spread_bits(quantize(c.x, lo[0], ext[0], bits), bits) | (spread_bits(quantize(c.y, lo[1], ext[1], bits), bits) << 1) |
         (spread_bits(quantize(c.z, lo[2], ext[2], bits), bits) << 2);
}

struct Frame6 {
  float lo[3], ext[3];
};

// keys for the static references: centroid of the reference box
__global__ void k_morton_static(const float* ref_box, uint32_t n, Frame6 f, uint64_t* keys, uint32_t* vals) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* b = ref_box + 6 * (size_t)i;
  const float3 c = make_float3(0.5f * (b[0] + b[3]), 0.5f * (b[1] + b[4]), 0.5f * (b[2] + b[5]));
  keys[i] = morton(c, f.lo, f.ext, 21);
  vals[i] = i;
}

// keys for the dynamic triangles: slot in the top 6 bits, then a 57-bit
// Morton code of the centroid inside the object's frame (object-local box at
// build, current world box when rebuilding)
__global__ void k_morton_dyn(const float* local, const Tri* world, const uint8_t* slot_of, uint32_t n,
                             const Frame6* frames, const DynObj* objs, int use_world, uint64_t* keys, uint32_t* vals) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t s = slot_of[i];
  float3 c;
  float lo[3], ext[3];
  if (use_world) {
    const Tri T = world[i];
    const float3 v0 = f3(T.v0), v1 = v0 + f3(T.e1), v2 = v0 + f3(T.e2);
    c = (1.f / 3.f) * (v0 + v1 + v2);
    for (int k = 0; k < 3; ++k) {
      lo[k] = objs[s].box_new[k];
      ext[k] = objs[s].box_new[3 + k] - objs[s].box_new[k];
    }
  } else {
    const float* v = local + 9 * (size_t)i;
    c = make_float3((v[0] + v[3] + v[6]) * (1.f / 3.f), (v[1] + v[4] + v[7]) * (1.f / 3.f),
                    (v[2] + v[5] + v[8]) * (1.f / 3.f));
    for (int k = 0; k < 3; ++k) {
      lo[k] = frames[s].lo[k];
      ext[k] = frames[s].ext[k];
    }
  }
  keys[i] = ((uint64_t)s << 57) | morton(c, lo, ext, 19);
  vals[i] = i;
}

// ------------------------------------------------------------------ radix sort
__global__ void k_rs_hist(const uint64_t* keys, uint32_t n, int shift, uint32_t* hist, uint32_t n_tiles) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t base = blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += blockDim.x) {
    const uint32_t j = base + i;
    if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[(size_t)i * n_tiles + blockIdx.x] = h[i];
}

// exclusive scan of m counters in place (one block of 1024 threads)
__global__ void k_rs_scan(uint32_t* hist, uint32_t m) {
  __shared__ uint32_t sums[1024];
  const uint32_t per = (m + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = min(b + per, m);
  uint32_t s = 0;
  for (uint32_t i = b; i < e; ++i) s += hist[i];
  sums[threadIdx.x] = s;
  __syncthreads();
  for (uint32_t off = 1; off < blockDim.x; off <<= 1) {
    const uint32_t v = threadIdx.x >= off ? sums[threadIdx.x - off] : 0u;
    __syncthreads();
    sums[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = sums[threadIdx.x] - s;
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t v = hist[i];
    hist[i] = run;
    run += v;
  }
}

// stable scatter: warp w of a tile ranks its 512 keys in order, 32 at a time
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                                                             uint32_t* vout, uint32_t n, int shift, const uint32_t* hist,
                                                             uint32_t n_tiles) {
  __shared__ uint32_t wcnt[kRsWarps][256];
  __shared__ uint32_t goff[256];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kRsWarps * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) goff[i] = hist[(size_t)i * n_tiles + blockIdx.x];
  __syncthreads();
  const uint32_t base = blockIdx.x * kRsTile + w * (kRsItems * 32);
  const unsigned lt = (1u << lane) - 1u;
  uint64_t k[kRsItems];
  uint32_t v[kRsItems], rank[kRsItems];
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const uint32_t j = base + r * 32 + lane;
    const bool valid = j < n;
    k[r] = valid ? kin[j] : 0ull;
    v[r] = valid ? vin[j] : 0u;
    const uint32_t d = valid ? (uint32_t)((k[r] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? wcnt[w][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt) == 0u) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    uint32_t run = 0;
    for (int q = 0; q < kRsWarps; ++q) {
      const uint32_t c = wcnt[q][d];
      wcnt[q][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const uint32_t j = base + r * 32 + lane;
    if (j < n) {
      const uint32_t d = (uint32_t)((k[r] >> shift) & 255u);
      const uint32_t pos = goff[d] + wcnt[w][d] + rank[r];
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
  }
}

// ------------------------------------------------------------------ hierarchy
__device__ __forceinline__ int lcp(const uint64_t* keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint64_t a = keys[i], b = keys[j];
  if (a == b) return 64 + __clz((unsigned)(i ^ j));
  return __clzll((long long)(a ^ b));
}

// Internal node i of the radix tree over n sorted keys: its key range, split
// and children (global indices: nodes at node_off, leaves at tri_off), the
// parent links of the bottom-up pass (local indices) and per-object roots.
__global__ void k_karras(const uint64_t* keys, int n, Node* nodes, int node_off, int tri_off, uint32_t* node_parent,
                         uint32_t* leaf_parent, const uint8_t* tri_slot, DynObj* objs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = (lcp(keys, n, i, i + 1) - lcp(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = lcp(keys, n, i, i - d);
  int lmax = 2;
  while (lcp(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (lcp(keys, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = lcp(keys, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (lcp(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  const int gamma = i + s * d + min(d, 0);
  const int first = min(i, j), last = max(i, j);
  const bool lleaf = first == gamma, rleaf = last == gamma + 1;
  const int left = lleaf ? ~(tri_off + gamma) : node_off + gamma;
  const int right = rleaf ? ~(tri_off + gamma + 1) : node_off + gamma + 1;
  nodes[node_off + i].d = make_int4(left, right, first, last);
  if (lleaf) leaf_parent[gamma] = ((uint32_t)i << 1); else node_parent[gamma] = ((uint32_t)i << 1);
  if (rleaf) leaf_parent[gamma + 1] = ((uint32_t)i << 1) | 1u; else node_parent[gamma + 1] = ((uint32_t)i << 1) | 1u;
  if (tri_slot) {
    const uint32_t sl = tri_slot[first];
    if (objs[sl].tri_begin == (uint32_t)first && objs[sl].tri_begin + objs[sl].tri_count - 1 == (uint32_t)last)
      objs[sl].root = node_off + i;
  }
}

// sorted references -> triangle records and leaf boxes
__global__ void k_gather_static(const float* verts, const uint32_t* ref_tri, const float* ref_box, const uint32_t* order,
                                const uint32_t* prim_of, uint32_t n, Tri* out, float* leaf_box) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t r = order[i];
  const uint32_t src = ref_tri[r];
  const float* v = verts + 9 * (size_t)src;
  Tri T;
  T.v0 = make_float4(v[0], v[1], v[2], __int_as_float((int)prim_of[src]));
  T.e1 = make_float4(v[3] - v[0], v[4] - v[1], v[5] - v[2], 0.f);
  T.e2 = make_float4(v[6] - v[0], v[7] - v[1], v[8] - v[2], 0.f);
  out[i] = T;
  for (int k = 0; k < 6; ++k) leaf_box[6 * (size_t)i + k] = ref_box[6 * (size_t)r + k];
}

// permute the dynamic arrays into the sorted order
__global__ void k_gather_dyn(const uint32_t* order, uint32_t n, const float* local_in, const uint32_t* prim_in,
                             const Tri* tri_in, float* local_out, uint32_t* prim_out, Tri* tri_out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t src = order[i];
  for (int k = 0; k < 9; ++k) local_out[9 * (size_t)i + k] = local_in[9 * (size_t)src + k];
  prim_out[i] = prim_in[src];
  if (tri_in) tri_out[i] = tri_in[src];
}

__global__ void k_fit(Node* nodes, const uint32_t* node_parent, const uint32_t* leaf_parent, uint32_t* flags,
                      const Tri* tris, const float* leaf_box, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || n < 2) return;
  fit_leaf(nodes, node_parent, leaf_parent, flags, tris, leaf_box, i);
}

// ------------------------------------------------------------------ per-frame update
__global__ void __launch_bounds__(256) k_update_objects(XformParams P, const float* local, const uint32_t* prim,
                                                          Tri* tris, DynObj* objs, float* xf_old, float* xf_new) {
  const uint32_t s = blockIdx.x;
  update_object(P.xf[s], ((P.moved >> s) & 1ull) != 0, local, prim, tris, objs, xf_old, xf_new, s);
}

// ------------------------------------------------------------------ wide (4-child) nodes
__device__ __forceinline__ int range_size(const Node* bnodes, int b) {
  const int4 d = bnodes[b].d;
  return d.w - d.z + 1;
}

// Collapse a binary tree into wide nodes, one block, level by level.  Each
// wide node starts from its binary node's two children and repeatedly opens
// the child of largest surface area until it has four children; a child whose
// subtree holds at most kLeafMax triangles becomes a leaf range (subtrees of a
// radix tree cover consecutive sorted triangles).  ``wsrc`` records, for every
// wide child, the binary slot its box comes from (binary node << 1 | side), so
// a refit of the binary tree can refresh the wide boxes.
//   static tree: one seed, binary root ``seed_root``, wide index ``wbase``;
//   dynamic objects: one seed per object with more than kLeafMax triangles.
// A wide node takes up to four children by opening, one at a time, the child
// with the largest surface area (the static tree: a cheaper traversal), or
// for the dynamic objects with PV_DYN_OPEN_BY_COUNT the child with the most
// triangles: a shallower tree, whose refit climbs fewer dependent levels
// (8 in place of 9 for the villa's 5000-triangle tori, 0.7 us less).
#ifndef PV_DYN_OPEN_BY_COUNT
#define PV_DYN_OPEN_BY_COUNT 1
#endif
__global__ void __launch_bounds__(1024) k_collapse(const Node* bnodes, int tri_off, int seed_root, DynObj* objs, int n_dyn,
                                                   int* qa, int* qb, uint32_t q_cap, WNode* wnodes, int* wsrc,
                                                   int wbase, uint32_t* wcount, int* status) {
  __shared__ uint32_t s_in, s_out, s_next;
  const int leaf_max = objs ? kLeafMax : kStaticLeafMax;
  if (threadIdx.x == 0) {
    uint32_t cnt = 0, next = 0;
    if (objs) {
      for (int s = 0; s < n_dyn; ++s) {
        const DynObj& o = objs[s];
        if (o.tri_count == 0) {
          objs[s].wroot = INT32_MIN;
        } else if (o.tri_count <= (uint32_t)kLeafMax) {
          objs[s].wroot = leaf_ref(tri_off + o.tri_begin, o.tri_count);
        } else {
          objs[s].wroot = wbase + (int)next;
          qa[2 * cnt] = o.root;
          qa[2 * cnt + 1] = wbase + (int)next;
          ++cnt;
          ++next;
        }
      }
    } else {
      qa[0] = seed_root;
      qa[1] = wbase;
      cnt = 1;
      next = 1;
    }
    s_in = cnt;
    s_next = next;
  }
  __syncthreads();
  for (int level = 0; level < 128; ++level) {
    const uint32_t n_in = s_in;
    if (n_in == 0) break;
    if (threadIdx.x == 0) s_out = 0;
    __syncthreads();
    for (uint32_t it = threadIdx.x; it < n_in; it += blockDim.x) {
      const int b = qa[2 * it], w = qa[2 * it + 1];
      float box[4][6];
      int ref[4], src[4];
      int m = 2;
      const int4 d = bnodes[b].d;
      ref[0] = d.x;
      ref[1] = d.y;
      slot_box(bnodes, b, 0, box[0]);
      slot_box(bnodes, b, 1, box[1]);
      src[0] = b << 1;
      src[1] = (b << 1) | 1;
      while (m < 4) {
        int pick = -1;
        float best = -1.f;
        for (int i = 0; i < m; ++i) {
          if (ref[i] < 0 || range_size(bnodes, ref[i]) <= leaf_max) continue;
          const float ex = box[i][3] - box[i][0], ey = box[i][4] - box[i][1], ez = box[i][5] - box[i][2];
          const float size = PV_DYN_OPEN_BY_COUNT && objs ? (float)range_size(bnodes, ref[i]) : ex * ey + ey * ez + ez * ex;
          if (size > best) {
            best = size;
            pick = i;
          }
        }
        if (pick < 0) break;
        const int c = ref[pick];
        const int4 dc = bnodes[c].d;
        ref[pick] = dc.x;
        slot_box(bnodes, c, 0, box[pick]);
        src[pick] = c << 1;
        ref[m] = dc.y;
        slot_box(bnodes, c, 1, box[m]);
        src[m] = (c << 1) | 1;
        ++m;
      }
      int wref[4];
      for (int i = 0; i < m; ++i) {
        const int c = ref[i];
        if (c < 0) {
          wref[i] = leaf_ref((uint32_t)(~c), 1);
        } else {
          const int4 dc = bnodes[c].d;
          const int size = dc.w - dc.z + 1;
          if (size <= leaf_max) {
            wref[i] = leaf_ref((uint32_t)(tri_off + dc.z), (uint32_t)size);
          } else {
            const uint32_t slot = atomicAdd(&s_out, 1u);
            const int nw = wbase + (int)atomicAdd(&s_next, 1u);
            if (slot < q_cap) {
              qb[2 * slot] = c;
              qb[2 * slot + 1] = nw;
            } else {
              record_error(status, PV_ERR_ITER_CAP);
            }
            wref[i] = nw;
          }
        }
      }
      write_wide(wnodes + w, box, wref, m);
      for (int i = 0; i < 4; ++i) wsrc[4 * (w - wbase) + i] = i < m ? src[i] : -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_in = min(s_out, q_cap);
    int* t = qa;
    qa = qb;
    qb = t;
    __syncthreads();
  }
  if (threadIdx.x == 0) *wcount = s_next;
}

// Refresh the boxes of wide nodes [0, n) of one tree from the refitted
// binary slots recorded by k_collapse.
__global__ void k_wide_refit(const Node* bnodes, const int* wsrc, const uint32_t* n_wide, WNode* wnodes) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= *n_wide) return;
  wide_refit_node(bnodes, wsrc, wnodes, w);
}

__global__ void k_build_top(WNode* wnodes, const Tri* tris, int top_off, int static_root, const DynObj* objs, int n_dyn,
                            int* root_out, uint64_t moved, MovedGroups* groups) {
  build_top_and_groups(wnodes, tris, top_off, static_root, objs, n_dyn, root_out, moved, groups);
}

// Parent links of the dynamic objects' wide nodes and of their triangles,
// after a collapse (the links start all ~0u: roots, one-triangle objects).
__global__ void k_wide_links(const WNode* wdyn, const uint32_t* n_wide, int w_off, uint32_t tri_off, uint32_t* w_link,
                             uint8_t* w_nch, uint32_t* t_link) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= *n_wide) return;
  const int4 ch = wdyn[w].child;
  const int c4[4] = {ch.x, ch.y, ch.z, ch.w};
  uint32_t m = 0;
  for (int c = 0; c < 4; ++c) {
    const int r = c4[c];
    if (r == INT32_MIN) continue;
    ++m;
    const uint32_t link = (w << 2) | (uint32_t)c;
    if (r >= 0) {
      w_link[r - w_off] = link;
    } else {
      const uint32_t f = leaf_first(r) - tri_off;
      for (uint32_t k = 0; k < leaf_count(r); ++k) t_link[f + k] = link;
    }
  }
  w_nch[w] = (uint8_t)m;
}

// Refit frames in one launch: the direct refit, then the last block to
// finish runs the frame's pose bookkeeping, the top level and the
// moved-object groups (what k_frame_top does alone when nothing moved).
struct TopArgs {
  uint32_t* done;              // blocks finished (reset by the last)
  DynObj* objs;
  float* xf_old;
  float* xf_new;
  WNode* wnodes;               // the whole wide array
  const Tri* tris;
  int top_off, static_root;
  int* root_out;
  MovedGroups* groups;
};

// The end of a refit launch, called by every thread of every block.
__device__ __forceinline__ void refit_finish(const XformParams& P, const RefitArgs& R, const TopArgs& T) {
  __shared__ bool s_last;
  __threadfence();                             // this block's triangles, boxes and object-box atomics
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(T.done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();                             // every block's writes are visible from here
  if (threadIdx.x == 0) *T.done = 0u;
  pose_bookkeeping(P.xf, P.moved, P.n_dyn, T.objs, T.xf_old, T.xf_new, R.obox);
  build_top_and_groups(T.wnodes, T.tris, T.top_off, T.static_root, T.objs, (int)P.n_dyn, T.root_out, P.moved,
                       T.groups);
}

// Resident blocks per SM asked of k_refit_wide (the block count it launches
// grows with the pairs).  6, and 8 (32 registers, 132 bytes of spills),
// measured the same as 5 within 1 us on the city and the villa.
#ifndef PV_REFIT_MIN_BLOCKS
#define PV_REFIT_MIN_BLOCKS 5
#endif

// Blocks [0, blocks_tri): one thread per dynamic triangle (refit_leaf); the
// blocks after them: one thread per pair of the pair table (refit_pair, the
// slots of the wide nodes above the triangles).
__global__ void __launch_bounds__(256, PV_REFIT_MIN_BLOCKS) k_refit_wide(XformParams P, RefitArgs R, PairArgs Q,
                                                                          TopArgs T, uint32_t blocks_tri) {
  if (blockIdx.x < blocks_tri) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t s = i < R.n ? R.tri_slot[i] : 0u;
    const bool mv = i < R.n && ((P.moved >> s) & 1ull);
    float3 blo, bhi;
    refit_leaf(P.xf[mv ? s : 0], mv, s, R, i, blo, bhi);
  } else {
    refit_pair(P, R, Q, (blockIdx.x - blocks_tri) * blockDim.x + threadIdx.x);
  }
  refit_finish(P, R, T);
}

// The same with the climb of refit_tri, one thread per dynamic triangle (for
// a scene built with PV_BUILD_REFIT_CLIMB, or without a pair table).
__global__ void __launch_bounds__(256) k_refit_climb(XformParams P, RefitArgs R, TopArgs T) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t s = i < R.n ? R.tri_slot[i] : 0u;
  const bool mv = i < R.n && ((P.moved >> s) & 1ull);
  refit_tri(P.xf[mv ? s : 0], mv, s, R, i);
  refit_finish(P, R, T);
}

// Pose bookkeeping of every slot, then (when objects moved) the top level
// and the moved objects' groups.  One block of 32 threads.
__global__ void k_frame_top(XformParams P, DynObj* objs, float* xf_old, float* xf_new, int* obox, WNode* wnodes,
                            const Tri* tris, int top_off, int static_root, int* root_out, MovedGroups* groups) {
  pose_bookkeeping(P.xf, P.moved, P.n_dyn, objs, xf_old, xf_new, obox);
  if (!P.moved) return;
  build_top_and_groups(wnodes, tris, top_off, static_root, objs, (int)P.n_dyn, root_out, P.moved, groups);
}


}  // namespace pvk

using namespace pvk;

namespace pvh {

void radix_sort(uint64_t*& k0, uint32_t*& v0, uint64_t*& k1, uint32_t*& v1, uint32_t n, uint32_t* hist,
                       int lo_bit, int hi_bit, cudaStream_t st) {
  const uint32_t n_tiles = (n + kRsTile - 1) / kRsTile;
  for (int shift = lo_bit; shift < hi_bit; shift += 8) {
    k_rs_hist<<<n_tiles, kRsThreads, 0, st>>>(k0, n, shift, hist, n_tiles);
    k_rs_scan<<<1, 1024, 0, st>>>(hist, 256u * n_tiles);
    k_rs_scatter<<<n_tiles, kRsThreads, 0, st>>>(k0, v0, k1, v1, n, shift, hist, n_tiles);
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
}

uint32_t radix_tiles(uint32_t n) { return (n + kRsTile - 1) / kRsTile; }

void exclusive_scan(uint32_t* data, uint32_t m, cudaStream_t st) { k_rs_scan<<<1, 1024, 0, st>>>(data, m); }

static inline uint32_t blocks(uint32_t n, uint32_t t) { return (n + t - 1) / t; }

// ---- oversized-triangle references (host)

// Clip the convex polygon P (n vertices) against the half-space s*x[axis] <= s*v.
static int clip_plane(const double (*P)[3], int n, int axis, double v, double s, double (*Q)[3]) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const double* a = P[i];
    const double* b = P[(i + 1) % n];
    const double da = s * (a[axis] - v), db = s * (b[axis] - v);
    if (da <= 0.0) {
      std::memcpy(Q[m++], a, sizeof(double) * 3);
    }
    if ((da < 0.0 && db > 0.0) || (da > 0.0 && db < 0.0)) {
      const double t = da / (da - db);
      for (int k = 0; k < 3; ++k) Q[m][k] = a[k] + t * (b[k] - a[k]);
      ++m;
    }
  }
  return m;
}

// References of the static triangles: one per triangle, except that a
// triangle whose box diagonal exceeds 8x the median is split over a grid of
// cells of that size, one reference per non-empty clipped part (at most 4096).
static void make_refs(const float* verts, const std::vector<uint32_t>& prims, std::vector<uint32_t>& ref_tri,
                      std::vector<float>& ref_box) {
  const size_t n = prims.size();
  std::vector<float> diag(n);
  for (size_t i = 0; i < n; ++i) {
    const float* v = verts + 9 * (size_t)prims[i];
    float d2 = 0.f;
    for (int k = 0; k < 3; ++k) {
      const float lo = std::min(v[k], std::min(v[3 + k], v[6 + k]));
      const float hi = std::max(v[k], std::max(v[3 + k], v[6 + k]));
      d2 += (hi - lo) * (hi - lo);
    }
    diag[i] = std::sqrt(d2);
  }
  std::vector<float> tmp(diag);
  std::nth_element(tmp.begin(), tmp.begin() + n / 2, tmp.end());
  const double cell = std::max(8.0 * tmp[n / 2], 1e-6);
  ref_tri.reserve(n);
  ref_box.reserve(6 * n);
  for (size_t i = 0; i < n; ++i) {
    const float* v = verts + 9 * (size_t)prims[i];
    float lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(v[k], std::min(v[3 + k], v[6 + k]));
      hi[k] = std::max(v[k], std::max(v[3 + k], v[6 + k]));
    }
    if (diag[i] <= cell) {
      ref_tri.push_back((uint32_t)i);
      ref_box.insert(ref_box.end(), {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]});
      continue;
    }
    int m[3];
    for (int k = 0; k < 3; ++k) m[k] = std::max(1, std::min(64, (int)std::ceil((hi[k] - lo[k]) / cell)));
    while ((long)m[0] * m[1] * m[2] > 4096)
      for (int k = 0; k < 3; ++k) m[k] = std::max(1, m[k] / 2);
    for (int a = 0; a < m[0]; ++a)
      for (int b = 0; b < m[1]; ++b)
        for (int c = 0; c < m[2]; ++c) {
          const int idx[3] = {a, b, c};
          double P[16][3], Q[16][3];
          for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) P[j][k] = v[3 * j + k];
          int cnt = 3;
          for (int k = 0; k < 3 && cnt; ++k) {
            const double c0 = lo[k] + (double)(hi[k] - lo[k]) * idx[k] / m[k];
            const double c1 = idx[k] + 1 == m[k] ? (double)hi[k] : lo[k] + (double)(hi[k] - lo[k]) * (idx[k] + 1) / m[k];
            cnt = clip_plane(P, cnt, k, c1, 1.0, Q);
            cnt = clip_plane(Q, cnt, k, c0, -1.0, P);
          }
          if (cnt == 0) continue;
          double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
          for (int j = 0; j < cnt; ++j)
            for (int k = 0; k < 3; ++k) {
              blo[k] = std::min(blo[k], P[j][k]);
              bhi[k] = std::max(bhi[k], P[j][k]);
            }
          ref_tri.push_back((uint32_t)i);
          float fb[6];
          for (int k = 0; k < 3; ++k) {   // round outward, never past the triangle's own box
            fb[k] = std::max(lo[k], std::nextafter((float)blo[k], -INFINITY));
            fb[3 + k] = std::min(hi[k], std::nextafter((float)bhi[k], INFINITY));
          }
          ref_box.insert(ref_box.end(), fb, fb + 6);
        }
  }
}

// ---- static tree by binned surface-area heuristic (host, once per scene)
//
// Top-down: each range of references is split where sum(area(child box) x
// references) over PV_SAH_BINS centroid bins per axis is smallest (Wald, "On fast
// construction of SAH-based bounding volume hierarchies", 2007); a range with
// coincident centroids splits at its middle.  Output: the references in leaf
// order, and per internal node (root 0, creation order) its two children
// (internal index, or ~leaf position), its leaf range and the parent links
// the bottom-up fit uses.  The fit computes the boxes and the collapse to
// wide nodes follows, as for the Morton tree.
struct SahOut {
  std::vector<uint32_t> order;
  std::vector<int4> d;
  std::vector<uint32_t> node_parent, leaf_parent;
};

// Centroid bins per axis and split: measured on the villa, 128 bins took node
// visits per re-trace ray from 22.1 (32 bins) to 21.7 and the reuse and
// trace-all frames 1-2 % faster, for 3.0 s of host build in place of 1.6 s;
// 256 gained nothing more.
#ifndef PV_SAH_BINS
#define PV_SAH_BINS 128
#endif
static void sah_build(const std::vector<float>& box, uint32_t n, SahOut& out) {
  constexpr int K = PV_SAH_BINS;
  out.order.resize(n);
  for (uint32_t i = 0; i < n; ++i) out.order[i] = i;
  out.d.assign(n > 1 ? n - 1 : 0, make_int4(0, 0, 0, 0));
  out.node_parent.assign(n, 0u);
  out.leaf_parent.assign(n, 0u);
  if (n < 2) return;
  std::vector<float> cen(3 * (size_t)n);
  for (uint32_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) cen[3 * (size_t)i + k] = 0.5f * (box[6 * (size_t)i + k] + box[6 * (size_t)i + 3 + k]);
  auto area = [](const float* b) {
    const float ex = std::max(b[3] - b[0], 0.f), ey = std::max(b[4] - b[1], 0.f), ez = std::max(b[5] - b[2], 0.f);
    return ex * ey + ey * ez + ez * ex;
  };
  auto grow = [](float* b, const float* c) {
    for (int k = 0; k < 3; ++k) {
      b[k] = std::min(b[k], c[k]);
      b[3 + k] = std::max(b[3 + k], c[3 + k]);
    }
  };
  struct Task { uint32_t b, e; int node; };
  std::vector<Task> todo{{0u, n, 0}};
  int next = 1;
  uint32_t* idx = out.order.data();
  while (!todo.empty()) {
    const Task t = todo.back();
    todo.pop_back();
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = t.b; i < t.e; ++i)
      for (int k = 0; k < 3; ++k) {
        clo[k] = std::min(clo[k], cen[3 * (size_t)idx[i] + k]);
        chi[k] = std::max(chi[k], cen[3 * (size_t)idx[i] + k]);
      }
    int best_axis = -1, best_bin = 0;
    float best_cost = INFINITY;
    for (int a = 0; a < 3; ++a) {
      const float ext = chi[a] - clo[a];
      if (!(ext > 0.f)) continue;
      uint32_t cnt[K] = {};
      float bb[K][6];
      for (int q = 0; q < K; ++q) {
        bb[q][0] = bb[q][1] = bb[q][2] = INFINITY;
        bb[q][3] = bb[q][4] = bb[q][5] = -INFINITY;
      }
      const float sc = (float)K / ext;
      for (uint32_t i = t.b; i < t.e; ++i) {
        const int q = std::min(K - 1, (int)((cen[3 * (size_t)idx[i] + a] - clo[a]) * sc));
        ++cnt[q];
        grow(bb[q], &box[6 * (size_t)idx[i]]);
      }
      float rarea[K];
      uint32_t rcnt[K];
      float acc[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
      uint32_t c = 0;
      for (int q = K - 1; q > 0; --q) {
        grow(acc, bb[q]);
        c += cnt[q];
        rarea[q] = area(acc);
        rcnt[q] = c;
      }
      float lacc[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
      uint32_t lc = 0;
      for (int q = 0; q < K - 1; ++q) {            // split between bins q and q + 1
        grow(lacc, bb[q]);
        lc += cnt[q];
        if (lc == 0 || rcnt[q + 1] == 0) continue;
        const float cost = area(lacc) * (float)lc + rarea[q + 1] * (float)rcnt[q + 1];
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = a;
          best_bin = q;
        }
      }
    }
    uint32_t mid;
    if (best_axis < 0) {
      mid = t.b + (t.e - t.b) / 2;                  // coincident centroids: split the range
    } else {
      const float sc = (float)K / (chi[best_axis] - clo[best_axis]);
      uint32_t* m = std::partition(idx + t.b, idx + t.e, [&](uint32_t r) {
        return std::min(K - 1, (int)((cen[3 * (size_t)r + best_axis] - clo[best_axis]) * sc)) <= best_bin;
      });
      mid = (uint32_t)(m - idx);
      if (mid == t.b || mid == t.e) mid = t.b + (t.e - t.b) / 2;
    }
    int child[2];
    const uint32_t lo[2] = {t.b, mid}, hi[2] = {mid, t.e};
    for (int side = 0; side < 2; ++side) {
      if (hi[side] - lo[side] == 1) {
        child[side] = ~(int)lo[side];
        out.leaf_parent[lo[side]] = ((uint32_t)t.node << 1) | (uint32_t)side;
      } else {
        child[side] = next++;
        out.node_parent[child[side]] = ((uint32_t)t.node << 1) | (uint32_t)side;
        todo.push_back({lo[side], hi[side], child[side]});
      }
    }
    out.d[t.node] = make_int4(child[0], child[1], (int)t.b, (int)t.e - 1);
  }
}

int build_bvh(pv_scene* s, const float* h_verts, const std::vector<uint32_t>& static_prims, cudaStream_t st) {
  int rc = PV_OK;
  auto fail = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == PV_OK) rc = e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA;
  };
  // ---- sizes and the shared arrays
  std::vector<uint32_t> ref_tri;
  std::vector<float> ref_box;
  if (!static_prims.empty()) make_refs(h_verts, static_prims, ref_tri, ref_box);
  const uint32_t ns = (uint32_t)ref_tri.size();
  const uint32_t nd = s->n_dyn_tris;
  s->n_static_refs = ns;
  s->d_tri_off = ns;
  s->d_node_off = ns > 1 ? ns - 1 : 0;
  const uint32_t n_nodes = s->d_node_off + (nd > 1 ? nd - 1 : 0) + 1;
  s->w_dyn_off = ns > 1 ? ns - 1 : 0;
  s->w_top_off = s->w_dyn_off + (nd > 1 ? nd - 1 : 0);
  s->n_wide = s->w_top_off + kMaxDyn + 1;
  s->q_cap = std::max<uint32_t>(ns, nd) + 64;
  fail(cudaMalloc(&s->tris, std::max<uint32_t>(ns + nd, 1) * sizeof(Tri)));
  fail(cudaMalloc(&s->nodes, n_nodes * sizeof(Node)));
  fail(cudaMalloc(&s->wnodes, s->n_wide * sizeof(WNode)));
  fail(cudaMalloc(&s->wsrc, 4 * (size_t)s->n_wide * sizeof(int)));
  fail(cudaMalloc(&s->wcount, 2 * sizeof(uint32_t)));
  fail(cudaMalloc(&s->cq, 4 * (size_t)s->q_cap * sizeof(int)));
  fail(cudaMalloc(&s->root, sizeof(int)));
  if (rc != PV_OK) return rc;
  fail(cudaMemsetAsync(s->nodes, 0, n_nodes * sizeof(Node), st));
  fail(cudaMemsetAsync(s->wnodes, 0, s->n_wide * sizeof(WNode), st));
  fail(cudaMemsetAsync(s->wcount, 0, 2 * sizeof(uint32_t), st));

  // ---- static tree
  s->s_root = INT32_MIN;
  if (ns) {
    Frame6 f;
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = 0; i < ns; ++i)
      for (int k = 0; k < 3; ++k) {
        const float c = 0.5f * (ref_box[6 * i + k] + ref_box[6 * i + 3 + k]);
        clo[k] = std::min(clo[k], c);
        chi[k] = std::max(chi[k], c);
      }
    for (int k = 0; k < 3; ++k) {
      f.lo[k] = clo[k];
      f.ext[k] = chi[k] - clo[k];
    }
    std::vector<float> sv(9 * static_prims.size());
    for (size_t i = 0; i < static_prims.size(); ++i)
      std::memcpy(&sv[9 * i], h_verts + 9 * (size_t)static_prims[i], 9 * sizeof(float));
    float *d_v = nullptr, *d_rbox = nullptr, *d_lbox = nullptr;
    uint32_t *d_prim = nullptr, *d_rtri = nullptr;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *hist = nullptr, *np = nullptr, *lp = nullptr, *flags = nullptr;
    const uint32_t n_tiles = blocks(ns, kRsTile);
    fail(cudaMalloc(&d_v, sv.size() * sizeof(float)));
    fail(cudaMalloc(&d_prim, static_prims.size() * sizeof(uint32_t)));
    fail(cudaMalloc(&d_rtri, ns * sizeof(uint32_t)));
    fail(cudaMalloc(&d_rbox, 6 * (size_t)ns * sizeof(float)));
    fail(cudaMalloc(&d_lbox, 6 * (size_t)ns * sizeof(float)));
    fail(cudaMalloc(&k0, ns * sizeof(uint64_t)));
    fail(cudaMalloc(&k1, ns * sizeof(uint64_t)));
    fail(cudaMalloc(&v0, ns * sizeof(uint32_t)));
    fail(cudaMalloc(&v1, ns * sizeof(uint32_t)));
    fail(cudaMalloc(&hist, 256 * (size_t)n_tiles * sizeof(uint32_t)));
    fail(cudaMalloc(&np, ns * sizeof(uint32_t)));
    fail(cudaMalloc(&lp, ns * sizeof(uint32_t)));
    fail(cudaMalloc(&flags, ns * sizeof(uint32_t)));
    if (rc == PV_OK) {
      fail(cudaMemcpyAsync(d_v, sv.data(), sv.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      fail(cudaMemcpyAsync(d_prim, static_prims.data(), static_prims.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
      fail(cudaMemcpyAsync(d_rtri, ref_tri.data(), ns * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
      fail(cudaMemcpyAsync(d_rbox, ref_box.data(), 6 * (size_t)ns * sizeof(float), cudaMemcpyHostToDevice, st));
      const bool sah = !(s->flags & PV_BUILD_STATIC_LBVH);
      if (sah) {
        SahOut t;
        sah_build(ref_box, ns, t);
        std::vector<Node> hn(ns > 1 ? ns - 1 : 0);
        for (size_t i = 0; i < hn.size(); ++i) {
          std::memset(&hn[i], 0, sizeof(Node));
          hn[i].d = t.d[i];
        }
        fail(cudaMemcpyAsync(v0, t.order.data(), ns * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        if (!hn.empty()) fail(cudaMemcpyAsync(s->nodes, hn.data(), hn.size() * sizeof(Node), cudaMemcpyHostToDevice, st));
        fail(cudaMemcpyAsync(np, t.node_parent.data(), ns * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        fail(cudaMemcpyAsync(lp, t.leaf_parent.data(), ns * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        fail(cudaStreamSynchronize(st));             // the host vectors go out of scope
      } else {
        k_morton_static<<<blocks(ns, 256), 256, 0, st>>>(d_rbox, ns, f, k0, v0);
        radix_sort(k0, v0, k1, v1, ns, hist, 0, 64, st);
      }
      k_gather_static<<<blocks(ns, 256), 256, 0, st>>>(d_v, d_rtri, d_rbox, v0, d_prim, ns, s->tris, d_lbox);
      if (ns >= 2) {
        if (!sah) k_karras<<<blocks(ns - 1, 256), 256, 0, st>>>(k0, (int)ns, s->nodes, 0, 0, np, lp, nullptr, nullptr);
        fail(cudaMemsetAsync(flags, 0, ns * sizeof(uint32_t), st));
        k_fit<<<blocks(ns, 256), 256, 0, st>>>(s->nodes, np, lp, flags, s->tris, d_lbox, (int)ns);
        s->s_root = 0;
        if (ns <= (uint32_t)kStaticLeafMax) {
          s->s_wroot = leaf_ref(0, ns);
        } else {
          k_collapse<<<1, 1024, 0, st>>>(s->nodes, 0, 0, nullptr, 0, s->cq, s->cq + 2 * s->q_cap, s->q_cap, s->wnodes,
                                         s->wsrc, 0, s->wcount, s->status);
          s->s_wroot = 0;
        }
      } else {
        s->s_root = ~0;
        s->s_wroot = leaf_ref(0, 1);
      }
      fail(cudaGetLastError());
      fail(cudaStreamSynchronize(st));
    }
    cudaFree(d_v); cudaFree(d_prim); cudaFree(d_rtri); cudaFree(d_rbox); cudaFree(d_lbox);
    cudaFree(k0); cudaFree(k1); cudaFree(v0); cudaFree(v1); cudaFree(hist); cudaFree(np); cudaFree(lp); cudaFree(flags);
    if (rc != PV_OK) return rc;
  }

  // ---- dynamic tree
  if (nd == 0) return PV_OK;
  std::vector<float> loc(9 * (size_t)nd);
  std::vector<uint32_t> prim(nd);
  std::vector<uint8_t> slot(nd);
  std::vector<Frame6> frames(s->n_dyn);
  {
    uint32_t w = 0;
    for (uint32_t sl = 0; sl < s->n_dyn; ++sl) {
      DynObj& o = s->h_objs[sl];
      o.tri_begin = w;
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (uint32_t t : s->dyn_tris_of[sl]) {
        std::memcpy(&loc[9 * (size_t)w], h_verts + 9 * (size_t)t, 9 * sizeof(float));
        prim[w] = t;
        slot[w] = (uint8_t)sl;
        for (int k = 0; k < 3; ++k) {
          const float c = (h_verts[9 * (size_t)t + k] + h_verts[9 * (size_t)t + 3 + k] + h_verts[9 * (size_t)t + 6 + k]) * (1.f / 3.f);
          lo[k] = std::min(lo[k], c);
          hi[k] = std::max(hi[k], c);
        }
        ++w;
      }
      o.tri_count = w - o.tri_begin;
      o.root = o.tri_count == 1 ? ~(int32_t)(s->d_tri_off + o.tri_begin) : INT32_MIN;
      o.wroot = INT32_MIN;
      for (int k = 0; k < 3; ++k) {
        frames[sl].lo[k] = lo[k];
        frames[sl].ext[k] = hi[k] - lo[k];
      }
    }
  }
  const uint32_t n_tiles = blocks(nd, kRsTile);
  Frame6* d_frames = nullptr;
  float* tmp_local = nullptr;
  uint32_t* tmp_prim = nullptr;
  fail(cudaMalloc(&d_frames, s->n_dyn * sizeof(Frame6)));
  fail(cudaMalloc(&tmp_local, 9 * (size_t)nd * sizeof(float)));
  fail(cudaMalloc(&tmp_prim, nd * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_local, 9 * (size_t)nd * sizeof(float)));
  fail(cudaMalloc(&s->d_tri_prim, nd * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_tri_slot, nd * sizeof(uint8_t)));
  fail(cudaMalloc(&s->d_leaf_parent, nd * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_node_parent, nd * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_fit_flags, nd * sizeof(uint32_t)));
  fail(cudaMalloc(&s->objs, s->n_dyn * sizeof(DynObj)));
  fail(cudaMalloc(&s->groups, sizeof(MovedGroups)));
  fail(cudaMemset(s->groups, 0, sizeof(MovedGroups)));
  fail(cudaMalloc(&s->w_link, nd * sizeof(uint32_t)));
  fail(cudaMalloc(&s->w_nch, nd * sizeof(uint8_t)));
  fail(cudaMalloc(&s->w_arrive, (nd + 1) * sizeof(uint32_t)));   // + the refit's block counter
  fail(cudaMalloc(&s->t_link, nd * sizeof(uint32_t)));
  fail(cudaMalloc(&s->obox, kMaxDyn * 6 * sizeof(int)));
  fail(cudaMemset(s->w_arrive, 0, (nd + 1) * sizeof(uint32_t)));
  {
    int ob[kMaxDyn * 6];
    for (int i = 0; i < kMaxDyn * 6; ++i) ob[i] = ord_of(i % 6 < 3 ? 3.0e38f : -3.0e38f);
    fail(cudaMemcpy(s->obox, ob, sizeof ob, cudaMemcpyHostToDevice));
  }
  for (int b = 0; b < 2; ++b) {
    fail(cudaMalloc(&s->r_keys[b], nd * sizeof(uint64_t)));
    fail(cudaMalloc(&s->r_vals[b], nd * sizeof(uint32_t)));
  }
  fail(cudaMalloc(&s->r_hist, 256 * (size_t)n_tiles * sizeof(uint32_t)));
  fail(cudaMalloc(&s->r_tris, nd * sizeof(Tri)));
  fail(cudaMalloc(&s->r_local, 9 * (size_t)nd * sizeof(float)));
  fail(cudaMalloc(&s->r_prim, nd * sizeof(uint32_t)));
  if (rc != PV_OK) {
    cudaFree(d_frames); cudaFree(tmp_local); cudaFree(tmp_prim);
    return rc;
  }
  fail(cudaMemcpyAsync(d_frames, frames.data(), s->n_dyn * sizeof(Frame6), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(tmp_local, loc.data(), loc.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(tmp_prim, prim.data(), nd * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(s->d_tri_slot, slot.data(), nd * sizeof(uint8_t), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(s->objs, s->h_objs.data(), s->n_dyn * sizeof(DynObj), cudaMemcpyHostToDevice, st));
  uint64_t *k0 = s->r_keys[0], *k1 = s->r_keys[1];
  uint32_t *v0 = s->r_vals[0], *v1 = s->r_vals[1];
  k_morton_dyn<<<blocks(nd, 256), 256, 0, st>>>(tmp_local, nullptr, s->d_tri_slot, nd, d_frames, s->objs, 0, k0, v0);
  radix_sort(k0, v0, k1, v1, nd, s->r_hist, 0, 64, st);
  k_gather_dyn<<<blocks(nd, 256), 256, 0, st>>>(v0, nd, tmp_local, tmp_prim, nullptr, s->d_local, s->d_tri_prim, nullptr);
  if (nd >= 2)
    k_karras<<<blocks(nd - 1, 256), 256, 0, st>>>(k0, (int)nd, s->nodes, (int)s->d_node_off, (int)s->d_tri_off,
                                                  s->d_node_parent, s->d_leaf_parent, s->d_tri_slot, s->objs);
  fail(cudaGetLastError());
  fail(cudaStreamSynchronize(st));
  cudaFree(d_frames); cudaFree(tmp_local); cudaFree(tmp_prim);
  return rc;
}

// After the first collapse: the pair table of k_refit_wide, from the parent
// links.  Every non-root dynamic wide node contributes one pair per triangle
// of its run, nodes in index order.  The runs are contiguous by construction
// (the triangles are stored in leaf order and each wide node covers one
// binary subtree); if one is not, no table is built and the refit climbs.
// Synchronous.
int build_refit_pairs(pv_scene* s, cudaStream_t st) {
  const uint32_t n = s->n_dyn_tris;
  s->pairs_ok = false;
  if (n == 0 || (s->flags & (PV_BUILD_DYN_REBUILD | PV_BUILD_REFIT_CLIMB)) || kLeafMax != 1) return PV_OK;
  int rc = PV_OK;
  auto fail = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == PV_OK) rc = e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA;
  };
  uint32_t nw = 0;
  fail(cudaStreamSynchronize(st));
  fail(cudaMemcpy(&nw, s->wcount + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (rc != PV_OK) return rc;
  if (nw > n) return PV_OK;
  std::vector<uint32_t> tl(n), wl(std::max<uint32_t>(nw, 1u));
  fail(cudaMemcpy(tl.data(), s->t_link, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (nw) fail(cudaMemcpy(wl.data(), s->w_link, nw * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (rc != PV_OK) return rc;
  // each non-root wide node's run, by its parent slot
  const size_t nl = 4 * (size_t)std::max<uint32_t>(nw, 1u);
  std::vector<uint32_t> lo(nl, 0xFFFFFFFFu), hi(nl, 0u), cnt(nl, 0u);
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t link = tl[i];
    for (int guard = 0; guard < 64 && link != 0xFFFFFFFFu; ++guard) {
      const uint32_t w = link >> 2;
      if (w >= nw) return PV_OK;
      const uint32_t up = wl[w];
      if (up == 0xFFFFFFFFu) break;            // w is an object's root
      if (up >= nl) return PV_OK;
      lo[up] = std::min(lo[up], i);
      hi[up] = std::max(hi[up], i);
      ++cnt[up];
      link = up;
    }
  }
  std::vector<uint32_t> plink, ptri, warps(nl, 0u);
  for (uint32_t w = 0; w < nw; ++w) {
    const uint32_t up = wl[w];
    if (up == 0xFFFFFFFFu || up >= nl) continue;
    if (cnt[up] == 0 || hi[up] - lo[up] + 1u != cnt[up]) return PV_OK;
    const size_t first = plink.size(), last = first + cnt[up] - 1;
    warps[up] = (uint32_t)((last >> 5) - (first >> 5) + 1);
    for (uint32_t i = lo[up]; i <= hi[up]; ++i) {
      plink.push_back(up | (warps[up] == 1u ? kPairOne : 0u));
      ptri.push_back(i);
    }
  }
  const size_t np = plink.size();
  std::vector<int> acc(6 * nl);
  for (size_t k = 0; k < acc.size(); ++k) acc[k] = k % 6 < 3 ? INT_MAX : INT_MIN;
  fail(cudaMalloc(&s->pair_link, std::max<size_t>(np, 1) * sizeof(uint32_t)));
  fail(cudaMalloc(&s->pair_tri, std::max<size_t>(np, 1) * sizeof(uint32_t)));
  fail(cudaMalloc(&s->pair_warps, nl * sizeof(uint32_t)));
  fail(cudaMalloc(&s->pair_acc, acc.size() * sizeof(int)));
  fail(cudaMalloc(&s->pair_count, nl * sizeof(uint32_t)));
  if (rc != PV_OK) return rc;
  if (np) {
    fail(cudaMemcpy(s->pair_link, plink.data(), np * sizeof(uint32_t), cudaMemcpyHostToDevice));
    fail(cudaMemcpy(s->pair_tri, ptri.data(), np * sizeof(uint32_t), cudaMemcpyHostToDevice));
  }
  fail(cudaMemcpy(s->pair_warps, warps.data(), nl * sizeof(uint32_t), cudaMemcpyHostToDevice));
  fail(cudaMemcpy(s->pair_acc, acc.data(), acc.size() * sizeof(int), cudaMemcpyHostToDevice));
  fail(cudaMemcpy(s->pair_count, warps.data(), nl * sizeof(uint32_t), cudaMemcpyHostToDevice));
  if (rc != PV_OK) return rc;
  s->n_pairs = (uint32_t)np;
  s->pairs_ok = true;
  return PV_OK;
}

// Per frame: previous pose kept, moved objects transformed; the dynamic tree
// is refitted, or rebuilt from world-space Morton codes
// (PV_BUILD_DYN_REBUILD); then the top level is rebuilt.
void launch_update_dynamic(pv_scene* s, cudaStream_t st) {
  const uint32_t n = s->n_dyn_tris;
  Tri* dtris = s->tris + s->d_tri_off;
  Node* dnodes = s->nodes + s->d_node_off;
  const bool collapse = s->moved && (!s->top_built || (s->flags & PV_BUILD_DYN_REBUILD));
  if (n) {
    XformParams P;
    std::memset(&P, 0, sizeof P);
    for (uint32_t sl = 0; sl < s->n_dyn; ++sl) std::memcpy(P.xf[sl], &s->h_xf_new[12 * sl], 12 * sizeof(float));
    P.moved = s->moved;
    P.n_dyn = s->n_dyn;
    if (s->top_built && !(s->flags & PV_BUILD_DYN_REBUILD) && kLeafMax == 1) {
      // refit frames: transform + wide refit in one kernel, bookkeeping and top level in another
      if (s->moved) {
        RefitArgs R;
        R.local = s->d_local;
        R.prim = s->d_tri_prim;
        R.tri_slot = s->d_tri_slot;
        R.dtris = dtris;
        R.n = n;
        R.t_link = s->t_link;
        R.w_link = s->w_link;
        R.w_nch = s->w_nch;
        R.w_arrive = s->w_arrive;
        R.wdyn = s->wnodes + s->w_dyn_off;
        R.obox = s->obox;
        TopArgs T;
        T.done = s->w_arrive + n;              // one word past the arrival counters
        T.objs = s->objs;
        T.xf_old = s->xf_old;
        T.xf_new = s->xf_new;
        T.wnodes = s->wnodes;
        T.tris = s->tris;
        T.top_off = (int)s->w_top_off;
        T.static_root = s->s_wroot;
        T.root_out = s->root;
        T.groups = s->groups;
        if (s->pairs_ok) {
          PairArgs Q;
          Q.link = s->pair_link;
          Q.tri = s->pair_tri;
          Q.warps = s->pair_warps;
          Q.acc = s->pair_acc;
          Q.count = s->pair_count;
          Q.n_pairs = s->n_pairs;
          const uint32_t bt = blocks(n, 256);
          k_refit_wide<<<bt + blocks(s->n_pairs, 256), 256, 0, st>>>(P, R, Q, T, bt);
        } else {
          k_refit_climb<<<blocks(n, 256), 256, 0, st>>>(P, R, T);
        }
        return;
      }
      k_frame_top<<<1, 32, 0, st>>>(P, s->objs, s->xf_old, s->xf_new, s->obox, s->wnodes, s->tris, (int)s->w_top_off,
                                    s->s_wroot, s->root, s->groups);
      return;
    }
    k_update_objects<<<s->n_dyn, 256, 0, st>>>(P, s->d_local, s->d_tri_prim, dtris, s->objs, s->xf_old, s->xf_new);
    if (s->moved) {
      if (s->flags & PV_BUILD_DYN_REBUILD) {
        uint64_t *k0 = s->r_keys[0], *k1 = s->r_keys[1];
        uint32_t *v0 = s->r_vals[0], *v1 = s->r_vals[1];
        k_morton_dyn<<<blocks(n, 256), 256, 0, st>>>(nullptr, dtris, s->d_tri_slot, n, nullptr, s->objs, 1, k0, v0);
        radix_sort(k0, v0, k1, v1, n, s->r_hist, 0, 64, st);
        k_gather_dyn<<<blocks(n, 256), 256, 0, st>>>(v0, n, s->d_local, s->d_tri_prim, dtris, s->r_local, s->r_prim, s->r_tris);
        std::swap(s->d_local, s->r_local);
        std::swap(s->d_tri_prim, s->r_prim);
        cudaMemcpyAsync(dtris, s->r_tris, n * sizeof(Tri), cudaMemcpyDeviceToDevice, st);
        if (n >= 2)
          k_karras<<<blocks(n - 1, 256), 256, 0, st>>>(k0, (int)n, s->nodes, (int)s->d_node_off, (int)s->d_tri_off,
                                                       s->d_node_parent, s->d_leaf_parent, s->d_tri_slot, s->objs);
      }
      if (n >= 2) {
        cudaMemsetAsync(s->d_fit_flags, 0, n * sizeof(uint32_t), st);
        k_fit<<<blocks(n, 256), 256, 0, st>>>(dnodes, s->d_node_parent, s->d_leaf_parent, s->d_fit_flags, dtris, nullptr,
                                              (int)n);
      }
      if (collapse) {
        // wide nodes of the dynamic objects (topology from the binary tree), and their parent links
        k_collapse<<<1, 1024, 0, st>>>(s->nodes, (int)s->d_tri_off, 0, s->objs, (int)s->n_dyn, s->cq,
                                       s->cq + 2 * s->q_cap, s->q_cap, s->wnodes, s->wsrc + 4 * (size_t)s->w_dyn_off,
                                       (int)s->w_dyn_off, s->wcount + 1, s->status);
        cudaMemsetAsync(s->w_link, 0xFF, n * sizeof(uint32_t), st);
        cudaMemsetAsync(s->t_link, 0xFF, n * sizeof(uint32_t), st);
        const uint32_t cap = std::max<uint32_t>(s->w_top_off - s->w_dyn_off, 1);
        k_wide_links<<<blocks(cap, 256), 256, 0, st>>>(s->wnodes + s->w_dyn_off, s->wcount + 1, (int)s->w_dyn_off,
                                                        s->d_tri_off, s->w_link, s->w_nch, s->t_link);
      } else if (n > (uint32_t)kLeafMax) {
        // refit: refresh the wide boxes from the binary slots
        const uint32_t cap = s->w_top_off - s->w_dyn_off;
        k_wide_refit<<<blocks(std::max<uint32_t>(cap, 1), 256), 256, 0, st>>>(s->nodes, s->wsrc + 4 * (size_t)s->w_dyn_off,
                                                                             s->wcount + 1, s->wnodes + s->w_dyn_off);
      }
    }
  }
  if (s->moved || !s->top_built) {
    k_build_top<<<1, 32, 0, st>>>(s->wnodes, s->tris, (int)s->w_top_off, s->s_wroot, s->objs, (int)s->n_dyn, s->root,
                                  s->moved, s->groups);
    s->top_built = true;
  }
}

}  // namespace pvh
