// Per-frame update of the dynamic objects' BVH, shared by the single-scene
// kernels (bvh.cu) and the batched ones (batch.cu): rigid transform of the
// moved objects with their tight boxes, bottom-up refit of the binary tree,
// refresh of the wide nodes from it, and the top level over the static root
// and the object roots.
#pragma once
#include <climits>
#include <cstring>

#include "pv_scene.h"

namespace pvk {

__device__ __forceinline__ void store_slot(Node* nd, int side, float3 lo, float3 hi) {
  float* a = reinterpret_cast<float*>(nd);
  if (side == 0) {
    *reinterpret_cast<float4*>(a + 0) = make_float4(lo.x, hi.x, lo.y, hi.y);
    *reinterpret_cast<float2*>(a + 8) = make_float2(lo.z, hi.z);
  } else {
    *reinterpret_cast<float4*>(a + 4) = make_float4(lo.x, hi.x, lo.y, hi.y);
    *reinterpret_cast<float2*>(a + 10) = make_float2(lo.z, hi.z);
  }
}

__device__ __forceinline__ void tri_box(const Tri& T, float3& lo, float3& hi) {
  const float3 v0 = f3(T.v0), v1 = v0 + f3(T.e1), v2 = v0 + f3(T.e2);
  lo = make_float3(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
  hi = make_float3(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
}

__device__ __forceinline__ void pad_box(float3& lo, float3& hi) {
  const float pad = 2.384185791015625e-07f * fmaxf(maxabs3(lo), maxabs3(hi)) + 1e-30f;
  lo = lo - make_float3(pad, pad, pad);
  hi = hi + make_float3(pad, pad, pad);
}

// Bottom-up boxes of one tree (``nodes`` = its first node, local indices):
// leaves from the triangle (or the given leaf box), padded by a relative
// 2^-22 so the FP32 slab test never rejects a box that holds a hit; each
// internal node's box is completed by the second child to arrive.
__device__ __forceinline__ void fit_leaf(Node* nodes, const uint32_t* node_parent, const uint32_t* leaf_parent,
                                         uint32_t* flags, const Tri* tris, const float* leaf_box, int i) {
  float3 lo, hi;
  if (leaf_box) {
    const float* b = leaf_box + 6 * (size_t)i;
    lo = make_float3(b[0], b[1], b[2]);
    hi = make_float3(b[3], b[4], b[5]);
  } else {
    tri_box(tris[i], lo, hi);
  }
  pad_box(lo, hi);
  uint32_t p = leaf_parent[i];
  for (int guard = 0; guard < 200; ++guard) {
    const int node = (int)(p >> 1);
    store_slot(nodes + node, (int)(p & 1u), lo, hi);
    __threadfence();
    if (atomicAdd(&flags[node], 1u) == 0u) return;
    const float* a = reinterpret_cast<const float*>(nodes + node);
    const float4 s0 = __ldcg(reinterpret_cast<const float4*>(a));
    const float4 s1 = __ldcg(reinterpret_cast<const float4*>(a + 4));
    const float4 sz = __ldcg(reinterpret_cast<const float4*>(a + 8));
    lo = make_float3(fminf(s0.x, s1.x), fminf(s0.z, s1.z), fminf(sz.x, sz.z));
    hi = make_float3(fmaxf(s0.y, s1.y), fmaxf(s0.w, s1.w), fmaxf(sz.y, sz.w));
    if (node == 0) return;
    p = node_parent[node];
  }
}

// Order-preserving integer image of a float (monotone over all non-NaN
// values), so that minima and maxima can be taken by integer atomics.
__host__ __device__ __forceinline__ int ord_of(float f) {
#ifdef __CUDA_ARCH__
  const int i = __float_as_int(f);
#else
  int i;
  memcpy(&i, &f, 4);
#endif
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float of_ord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

struct XformParams {
  float xf[kMaxDyn][12];
  uint64_t moved;
  uint32_t n_dyn;
};

// Object-local corners v (9 floats) of one triangle under the 3x4 row-major
// pose m; widens the tight box (lo, hi) by the transformed corners.
__device__ __forceinline__ Tri xform_tri(const float* m, const float* v, uint32_t prim, float* lo, float* hi) {
  float w[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      w[3 * k + r] = fmaf(m[4 * r + 0], v[3 * k + 0], fmaf(m[4 * r + 1], v[3 * k + 1], fmaf(m[4 * r + 2], v[3 * k + 2], m[4 * r + 3])));
      lo[r] = fminf(lo[r], w[3 * k + r]);
      hi[r] = fmaxf(hi[r], w[3 * k + r]);
    }
  Tri T;
  T.v0 = make_float4(w[0], w[1], w[2], __int_as_float((int)prim));
  T.e1 = make_float4(w[3] - w[0], w[4] - w[1], w[5] - w[2], 0.f);
  T.e2 = make_float4(w[6] - w[0], w[7] - w[1], w[8] - w[2], 0.f);
  return T;
}

// Direct refit of the dynamic objects' wide nodes.  One thread per dynamic
// triangle: a moved object's triangle goes to the new pose, its exact box
// joins the object's box (integer atomics), and its padded box is written
// into its slot of the parent wide node (refit_leaf).  The nodes above come
// either from a climb, where the last child to arrive at a node takes the
// union of the node's children up to the parent, and so on to the object's
// root (refit_tri), or from the node's run of triangles, with no dependent
// levels (refit_pair).  Either way the boxes are the same minima and maxima
// of the same padded leaf boxes that the binary refit gathers, so the wide
// nodes come out identical.
struct RefitArgs {
  const float* local;
  const uint32_t* prim;
  const uint8_t* tri_slot;
  Tri* dtris;
  uint32_t n;
  const uint32_t* t_link;
  const uint32_t* w_link;
  const uint8_t* w_nch;
  uint32_t* w_arrive;
  WNode* wdyn;
  int* obox;
};

// Arrival of one child at a wide node: an atomic increment of the node's
// count with release (this thread's slot stores are visible to whoever sees
// the count) and acquire (the slots of the children that arrived before are
// visible to this thread's loads) semantics at GPU scope; returns the count
// before.
__device__ __forceinline__ uint32_t arrive(uint32_t* count) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
  return old;
}

// The first half of a dynamic triangle's refit, called by every thread of
// the block: a moved triangle goes to the new pose (stored), its exact box
// joins the object's box, and its padded box (blo, bhi) is written into its
// slot of the parent wide node.
__device__ __forceinline__ void refit_leaf(const float* xf_slot, bool moved_lane, uint32_t s, const RefitArgs& R,
                                           uint32_t i, float3& blo, float3& bhi) {
  const int lane = threadIdx.x & 31;
  const uint32_t link = moved_lane ? R.t_link[i] : 0xFFFFFFFFu;
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  Tri T;
  if (moved_lane) {
    T = xform_tri(xf_slot, R.local + 9 * (size_t)i, R.prim[i], lo, hi);
    R.dtris[i] = T;
  }
  // The object's exact box: the lanes of one object reduce theirs, one of
  // them adds it to the block's (shared memory), and the block adds its
  // boxes to the objects' (one global atomic per object and bound that the
  // block holds, where one per warp made the objects' few words a queue).
  __shared__ int s_obox[kMaxDyn * 6];
  for (int j = threadIdx.x; j < kMaxDyn * 6; j += blockDim.x) s_obox[j] = j % 6 < 3 ? INT_MAX : INT_MIN;
  __syncthreads();
  const unsigned same = __match_any_sync(0xffffffffu, moved_lane ? (int)s : -1);
  if (moved_lane) {
    const int leader = __ffs(same) - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int l = __reduce_min_sync(same, ord_of(lo[k]));
      const int h = __reduce_max_sync(same, ord_of(hi[k]));
      if (lane == leader) {
        atomicMin(s_obox + 6 * s + k, l);
        atomicMax(s_obox + 6 * s + 3 + k, h);
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kMaxDyn * 6; j += blockDim.x) {
    const int v = s_obox[j];
    if (j % 6 < 3 ? v != INT_MAX : v != INT_MIN) {
      if (j % 6 < 3) atomicMin(R.obox + j, v);
      else atomicMax(R.obox + j, v);
    }
  }
  if (!moved_lane) return;
  tri_box(T, blo, bhi);
  pad_box(blo, bhi);
  if (link == 0xFFFFFFFFu) return;             // a one-triangle object: the triangle is the root
  WNode* nd = R.wdyn + (link >> 2);
  const uint32_t c = link & 3u;
  (&nd->lox.x)[c] = blo.x;
  (&nd->hix.x)[c] = bhi.x;
  (&nd->loy.x)[c] = blo.y;
  (&nd->hiy.x)[c] = bhi.y;
  (&nd->loz.x)[c] = blo.z;
  (&nd->hiz.x)[c] = bhi.z;
}

// The refit by climbing: after refit_leaf, the last child to arrive at a wide
// node takes the union of the node's children up to the parent, and so on to
// the object's root.
__device__ __forceinline__ void refit_tri(const float* xf_slot, bool moved_lane, uint32_t s, const RefitArgs& R,
                                          uint32_t i) {
  float3 blo, bhi;
  refit_leaf(xf_slot, moved_lane, s, R, i, blo, bhi);
  if (!moved_lane) return;
  uint32_t link = R.t_link[i];
  for (int guard = 0; guard < 64 && link != 0xFFFFFFFFu; ++guard) {
    const uint32_t w = link >> 2;
    const uint32_t m = R.w_nch[w];
    if (arrive(R.w_arrive + w) + 1u < m) return;
    R.w_arrive[w] = 0u;                        // every child of this frame has arrived
    blo = make_float3(3.0e38f, 3.0e38f, 3.0e38f);
    bhi = make_float3(-3.0e38f, -3.0e38f, -3.0e38f);
    WNode* nd = R.wdyn + w;
    for (uint32_t q = 0; q < m; ++q) {
      blo.x = fminf(blo.x, __ldcg(&nd->lox.x + q));
      blo.y = fminf(blo.y, __ldcg(&nd->loy.x + q));
      blo.z = fminf(blo.z, __ldcg(&nd->loz.x + q));
      bhi.x = fmaxf(bhi.x, __ldcg(&nd->hix.x + q));
      bhi.y = fmaxf(bhi.y, __ldcg(&nd->hiy.x + q));
      bhi.z = fmaxf(bhi.z, __ldcg(&nd->hiz.x + q));
    }
    link = R.w_link[w];
    if (link == 0xFFFFFFFFu) return;
    WNode* up = R.wdyn + (link >> 2);
    const uint32_t c = link & 3u;
    (&up->lox.x)[c] = blo.x;
    (&up->hix.x)[c] = bhi.x;
    (&up->loy.x)[c] = blo.y;
    (&up->hiy.x)[c] = bhi.y;
    (&up->loz.x)[c] = blo.z;
    (&up->hiz.x)[c] = bhi.z;
  }
}

// The refit without a climb.  The dynamic triangles are stored in the leaf
// order of their tree, so the triangles under a wide node are a contiguous
// run, and the box that the node's parent slot holds (the union of the padded
// triangle boxes below it, which the climb builds level by level) is a
// minimum and a maximum over that run.  The pairs (node, triangle of its run)
// of every non-root dynamic wide node are listed node after node and cut into
// warps of 32, one thread per pair: the thread transforms its triangle as
// refit_leaf does, the lanes of one node reduce their boxes, and the node's
// box is written into its parent slot.  A node whose pairs span several warps
// is combined through integer atomics, and the last warp to arrive writes the
// slot.  No warp waits on another level, and the minima and maxima are exact,
// so the slots come out as the climb makes them.
constexpr uint32_t kPairOne = 0x80000000u;    // flag of a node whose pairs lie inside one warp

struct PairArgs {
  const uint32_t* link;      // [n_pairs] parent slot (wide node << 2 | slot) of the pair's node, with kPairOne
  const uint32_t* tri;       // [n_pairs] local dynamic triangle under the node
  const uint32_t* warps;     // [by parent slot] warps that hold the node's pairs
  int* acc;                  // [by parent slot][6] box over several warps (order-preserving integers; empty
                             // between frames)
  uint32_t* count;           // [by parent slot] warps still to arrive this frame (warps between frames)
  uint32_t n_pairs;
};

// The wide-node box (order-preserving integers r) into parent slot ``link``.
__device__ __forceinline__ void write_slot(const RefitArgs& R, uint32_t link, const int (&r)[6]) {
  WNode* nd = R.wdyn + (link >> 2);
  const uint32_t c = link & 3u;
  (&nd->lox.x)[c] = of_ord(r[0]);
  (&nd->loy.x)[c] = of_ord(r[1]);
  (&nd->loz.x)[c] = of_ord(r[2]);
  (&nd->hix.x)[c] = of_ord(r[3]);
  (&nd->hiy.x)[c] = of_ord(r[4]);
  (&nd->hiz.x)[c] = of_ord(r[5]);
}

// Pair q (every lane of the warp calls it).
__device__ __forceinline__ void refit_pair(const XformParams& P, const RefitArgs& R, const PairArgs& Q, uint32_t q) {
  const int lane = threadIdx.x & 31;
  const bool in = q < Q.n_pairs;
  const uint32_t e = in ? __ldg(Q.link + q) : 0u;
  const uint32_t i = in ? __ldg(Q.tri + q) : 0u;
  const uint32_t s = in ? R.tri_slot[i] : 0u;
  const bool mv = in && ((P.moved >> s) & 1ull);
  int b[6] = {0, 0, 0, 0, 0, 0};
  if (mv) {
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    const Tri T = xform_tri(P.xf[s], R.local + 9 * (size_t)i, 0u, lo, hi);
    float3 blo, bhi;
    tri_box(T, blo, bhi);
    pad_box(blo, bhi);
    b[0] = ord_of(blo.x);
    b[1] = ord_of(blo.y);
    b[2] = ord_of(blo.z);
    b[3] = ord_of(bhi.x);
    b[4] = ord_of(bhi.y);
    b[5] = ord_of(bhi.z);
  }
  const uint32_t link = e & ~kPairOne;
  // a node's pairs are consecutive, so the lanes of one node are one group
  const unsigned grp = __match_any_sync(0xffffffffu, mv ? (int)link : -1);
  if (!mv) return;
  int r[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    r[j] = __reduce_min_sync(grp, b[j]);
    r[3 + j] = __reduce_max_sync(grp, b[3 + j]);
  }
  if (lane != __ffs(grp) - 1) return;
  if (!(e & kPairOne)) {
    int* a = Q.acc + 6 * (size_t)link;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      atomicMin(a + j, r[j]);
      atomicMax(a + 3 + j, r[3 + j]);
    }
    uint32_t left;                             // release: the box atomics above; acquire: the other warps'
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], -1;" : "=r"(left) : "l"(Q.count + link) : "memory");
    if (left != 1u) return;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      r[j] = __ldcg(a + j);
      a[j] = j < 3 ? INT_MAX : INT_MIN;
    }
    Q.count[link] = __ldg(Q.warps + link);
  }
  write_slot(R, link, r);
}

// Per-frame pose bookkeeping of every dynamic slot (what update_object does
// besides transforming): the new pose becomes the old one; a moved object's
// new box is this frame's reduced exact box, whose accumulator is reset.
// Called by all threads of one block.
__device__ __forceinline__ void pose_bookkeeping(const float (*xf)[12], uint64_t moved, uint32_t n_dyn, DynObj* objs,
                                                 float* xf_old, float* xf_new, int* obox) {
  for (uint32_t i = threadIdx.x; i < n_dyn * 12; i += blockDim.x) {
    xf_old[i] = xf_new[i];
    xf_new[i] = xf[i / 12][i % 12];
  }
  for (uint32_t i = threadIdx.x; i < n_dyn * 6; i += blockDim.x) {
    const uint32_t sl = i / 6, k = i % 6;
    objs[sl].box_old[k] = objs[sl].box_new[k];
    if ((moved >> sl) & 1ull) {
      objs[sl].box_new[k] = of_ord(obox[i]);
      obox[i] = ord_of(k < 3 ? 3.0e38f : -3.0e38f);
    }
  }
}

// One block (256 threads) per dynamic slot: keep the previous pose (transform
// and tight box), and for a moved object transform its object-local corners to
// the new pose and reduce the new tight box.
__device__ __forceinline__ void update_object(const float* xf_slot, bool moved, const float* local, const uint32_t* prim,
                                              Tri* tris, DynObj* objs, float* xf_old, float* xf_new, uint32_t s) {
  __shared__ float red[6][256];
  __shared__ float m[12];
  DynObj* o = objs + s;
  if (threadIdx.x < 12) {
    xf_old[12 * s + threadIdx.x] = xf_new[12 * s + threadIdx.x];
    m[threadIdx.x] = xf_slot[threadIdx.x];
  }
  if (threadIdx.x < 6) o->box_old[threadIdx.x] = o->box_new[threadIdx.x];
  __syncthreads();
  if (threadIdx.x < 12) xf_new[12 * s + threadIdx.x] = m[threadIdx.x];
  if (!moved) return;
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  const uint32_t b = o->tri_begin, e = b + o->tri_count;
  for (uint32_t i = b + threadIdx.x; i < e; i += blockDim.x) tris[i] = xform_tri(m, local + 9 * (size_t)i, prim[i], lo, hi);
  for (int k = 0; k < 3; ++k) {
    red[k][threadIdx.x] = lo[k];
    red[3 + k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int k = 0; k < 3; ++k) {
        red[k][threadIdx.x] = fminf(red[k][threadIdx.x], red[k][threadIdx.x + off]);
        red[3 + k][threadIdx.x] = fmaxf(red[3 + k][threadIdx.x], red[3 + k][threadIdx.x + off]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) o->box_new[threadIdx.x] = red[threadIdx.x][0];
}

__device__ __forceinline__ void slot_box(const Node* bnodes, int b, int side, float* box) {
  const float* a = reinterpret_cast<const float*>(bnodes + b) + 4 * side;
  const float* z = reinterpret_cast<const float*>(bnodes + b) + 8 + 2 * side;
  box[0] = __ldcg(a + 0);
  box[3] = __ldcg(a + 1);
  box[1] = __ldcg(a + 2);
  box[4] = __ldcg(a + 3);
  box[2] = __ldcg(z + 0);
  box[5] = __ldcg(z + 1);
}

__device__ __forceinline__ void write_wide(WNode* w, const float (*box)[6], const int* ref, int m) {
  float b[4][6];
  int c[4];
  for (int i = 0; i < 4; ++i) {
    for (int k = 0; k < 3; ++k) {
      b[i][k] = i < m ? box[i][k] : 3.0e38f;
      b[i][3 + k] = i < m ? box[i][3 + k] : -3.0e38f;
    }
    c[i] = i < m ? ref[i] : INT32_MIN;
  }
  w->lox = make_float4(b[0][0], b[1][0], b[2][0], b[3][0]);
  w->hix = make_float4(b[0][3], b[1][3], b[2][3], b[3][3]);
  w->loy = make_float4(b[0][1], b[1][1], b[2][1], b[3][1]);
  w->hiy = make_float4(b[0][4], b[1][4], b[2][4], b[3][4]);
  w->loz = make_float4(b[0][2], b[1][2], b[2][2], b[3][2]);
  w->hiz = make_float4(b[0][5], b[1][5], b[2][5], b[3][5]);
  w->child = make_int4(c[0], c[1], c[2], c[3]);
  w->pad = make_int4(0, 0, 0, 0);
}

// Refresh the boxes of wide node w from the binary slots it was collapsed from.
__device__ __forceinline__ void wide_refit_node(const Node* bnodes, const int* wsrc, WNode* wnodes, uint32_t w) {
  float* lo[3] = {&wnodes[w].lox.x, &wnodes[w].loy.x, &wnodes[w].loz.x};
  float* hi[3] = {&wnodes[w].hix.x, &wnodes[w].hiy.x, &wnodes[w].hiz.x};
  for (int i = 0; i < 4; ++i) {
    const int src = wsrc[4 * w + i];
    if (src < 0) continue;
    float box[6];
    slot_box(bnodes, src >> 1, src & 1, box);
    for (int k = 0; k < 3; ++k) {
      lo[k][i] = box[k];
      hi[k][i] = box[3 + k];
    }
  }
}

// box of a wide reference (node: union of its children; leaf: its triangles)
__device__ __forceinline__ void ref_box(const WNode* wnodes, const Tri* tris, int r, float* b) {
  for (int k = 0; k < 3; ++k) {
    b[k] = 3.0e38f;
    b[3 + k] = -3.0e38f;
  }
  if (r >= 0) {
    const WNode& n = wnodes[r];
    const float lx[4] = {n.lox.x, n.lox.y, n.lox.z, n.lox.w}, hx[4] = {n.hix.x, n.hix.y, n.hix.z, n.hix.w};
    const float ly[4] = {n.loy.x, n.loy.y, n.loy.z, n.loy.w}, hy[4] = {n.hiy.x, n.hiy.y, n.hiy.z, n.hiy.w};
    const float lz[4] = {n.loz.x, n.loz.y, n.loz.z, n.loz.w}, hz[4] = {n.hiz.x, n.hiz.y, n.hiz.z, n.hiz.w};
    for (int c = 0; c < 4; ++c) {
      b[0] = fminf(b[0], lx[c]); b[1] = fminf(b[1], ly[c]); b[2] = fminf(b[2], lz[c]);
      b[3] = fmaxf(b[3], hx[c]); b[4] = fmaxf(b[4], hy[c]); b[5] = fmaxf(b[5], hz[c]);
    }
  } else {
    const uint32_t f = leaf_first(r), c = leaf_count(r);
    for (uint32_t i = 0; i < c; ++i) {
      float3 lo, hi;
      tri_box(tris[f + i], lo, hi);
      pad_box(lo, hi);
      b[0] = fminf(b[0], lo.x); b[1] = fminf(b[1], lo.y); b[2] = fminf(b[2], lo.z);
      b[3] = fmaxf(b[3], hi.x); b[4] = fmaxf(b[4], hi.y); b[5] = fmaxf(b[5], hi.z);
    }
  }
}

// Top level over the static root and the dynamic objects' roots, rebuilt in
// every frame in which objects move: entries sorted along the axis of
// largest centroid spread and cut into four consecutive groups,
// recursively.  The moved objects' groups (MovedGroups) come from the same
// sort over the moved objects' old-and-new boxes, cut into runs of
// kGroupSize.  Both are built by one warp each: the centroid bounds by
// shuffles, the sort by ranks (entry i goes to position #{j: key_j < key_i}
// + #{j < i: key_j = key_i}, the stable ascending order), the top level's
// node ranges by one lane, and the nodes' boxes by a lane per node.

// Stable ascending order of n <= kMaxDyn + 1 boxes by the centroid along the
// axis of largest centroid spread (ties to the first axis).  One warp.
__device__ __forceinline__ void sort_by_centroid(const float (*box)[6], int n, float* key, int* order, int lane) {
  float clo[3] = {3e38f, 3e38f, 3e38f}, chi[3] = {-3e38f, -3e38f, -3e38f};
  for (int i = lane; i < n; i += 32)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float c = 0.5f * (box[i][k] + box[i][3 + k]);
      clo[k] = fminf(clo[k], c);
      chi[k] = fmaxf(chi[k], c);
    }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      clo[k] = fminf(clo[k], __shfl_xor_sync(0xffffffffu, clo[k], o));
      chi[k] = fmaxf(chi[k], __shfl_xor_sync(0xffffffffu, chi[k], o));
    }
  int ax = 0;
  for (int k = 1; k < 3; ++k)
    if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
  for (int i = lane; i < n; i += 32) key[i] = box[i][ax] + box[i][3 + ax];
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const float ki = key[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const float kj = key[j];
      r += (kj < ki) | ((kj == ki) & (j < i));
    }
    order[r] = i;
  }
  __syncwarp();
}

constexpr int kMaxTopNodes = 32;               // internal top-level nodes over at most kMaxDyn + 1 entries

struct TopSmem {
  float box[kMaxDyn + 1][6];                   // entry 0: the static root; 1 + s: slot s
  int ref[kMaxDyn + 1];
  float cbox[kMaxDyn + 1][6];                  // the valid entries, in entry order
  int cref[kMaxDyn + 1];
  float key[kMaxDyn + 1];
  int order[kMaxDyn + 1];
  int nn;                                      // internal nodes, in the order they are numbered
  int node[kMaxTopNodes], ng[kMaxTopNodes];
  int gb[kMaxTopNodes][4], ge[kMaxTopNodes][4], child[kMaxTopNodes][4];
  int sb[kMaxTopNodes], se[kMaxTopNodes], sn[kMaxTopNodes];
};

struct MovedSmem {
  float box[kMaxDyn][6];                       // moved objects' old u new boxes, in slot order
  int slot[kMaxDyn];
  float key[kMaxDyn];
  int order[kMaxDyn];
};

// The top level from the gathered entries of ts (one warp).
__device__ __forceinline__ void top_build_warp(TopSmem& ts, int n_dyn, WNode* wnodes, int top_off, int* root_out,
                                               int lane) {
  int n = 0;                                   // keep the valid entries in order
  for (int e0 = 0; e0 <= n_dyn; e0 += 32) {
    const int e = e0 + lane;
    const bool v = e <= n_dyn && ts.ref[e] != INT32_MIN;
    const unsigned b = __ballot_sync(0xffffffffu, v);
    if (v) {
      const int j = n + __popc(b & ((1u << lane) - 1u));
      ts.cref[j] = ts.ref[e];
#pragma unroll
      for (int k = 0; k < 6; ++k) ts.cbox[j][k] = ts.box[e][k];
    }
    n += __popc(b);
  }
  __syncwarp();
  if (n <= 1) {
    if (lane == 0) *root_out = n == 0 ? INT32_MIN : ts.cref[0];
    return;
  }
  sort_by_centroid(ts.cbox, n, ts.key, ts.order, lane);
  if (lane == 0) {                             // node ranges, numbered as they are pushed
    int sp = 1, next = 1, nn = 0;
    ts.sb[0] = 0;
    ts.se[0] = n;
    ts.sn[0] = top_off;
    while (sp > 0 && nn < kMaxTopNodes) {
      --sp;
      const int b = ts.sb[sp], e = ts.se[sp], node = ts.sn[sp];
      const int size = e - b;
      const int groups = size < 4 ? size : 4;
      ts.node[nn] = node;
      ts.ng[nn] = groups;
      for (int g = 0; g < groups; ++g) {
        const int gb = b + (size * g) / groups, ge = b + (size * (g + 1)) / groups;
        ts.gb[nn][g] = gb;
        ts.ge[nn][g] = ge;
        if (ge - gb == 1) {
          ts.child[nn][g] = ts.cref[ts.order[gb]];
        } else {
          ts.child[nn][g] = top_off + next++;
          ts.sb[sp] = gb;
          ts.se[sp] = ge;
          ts.sn[sp] = ts.child[nn][g];
          ++sp;
        }
      }
      ++nn;
    }
    ts.nn = nn;
    *root_out = top_off;
  }
  __syncwarp();
  for (int k = lane; k < ts.nn; k += 32) {     // each node's group boxes, by one lane
    float cb[4][6];
    int ch[4];
    const int groups = ts.ng[k];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cb[g][c] = 3e38f;
        cb[g][3 + c] = -3e38f;
      }
      ch[g] = INT32_MIN;
      if (g < groups) {
        ch[g] = ts.child[k][g];
        for (int i = ts.gb[k][g]; i < ts.ge[k][g]; ++i) {
          const float* bx = ts.cbox[ts.order[i]];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            cb[g][c] = fminf(cb[g][c], bx[c]);
            cb[g][3 + c] = fmaxf(cb[g][3 + c], bx[3 + c]);
          }
        }
      }
    }
    write_wide(wnodes + ts.node[k], cb, ch, groups);
  }
}

// The moved objects' groups of this frame (one warp).
__device__ __forceinline__ void moved_groups_warp(MovedSmem& ms, const DynObj* objs, int n_dyn, uint64_t moved,
                                                  MovedGroups* g, int lane) {
  const int nd = min(n_dyn, kMaxDyn);
  int n = 0;                                   // the moved slots, in order
  for (int s0 = 0; s0 < nd; s0 += 32) {
    const int s = s0 + lane;
    const bool m = s < nd && ((moved >> s) & 1ull);
    const unsigned b = __ballot_sync(0xffffffffu, m);
    if (m) {
      const int j = n + __popc(b & ((1u << lane) - 1u));
      ms.slot[j] = s;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        ms.box[j][k] = k < 3 ? fminf(objs[s].box_new[k], objs[s].box_old[k])
                             : fmaxf(objs[s].box_new[k], objs[s].box_old[k]);
    }
    n += __popc(b);
  }
  __syncwarp();
  sort_by_centroid(ms.box, n, ms.key, ms.order, lane);
  const int ngr = (n + kGroupSize - 1) / kGroupSize;
  for (int q = lane; q < ngr; q += 32) {
    float b[6] = {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f};
    for (int m = 0; m < kGroupSize; ++m) {
      const int i = q * kGroupSize + m;
      if (i < n) {
        const int o = ms.order[i];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          b[k] = fminf(b[k], ms.box[o][k]);
          b[3 + k] = fmaxf(b[3 + k], ms.box[o][3 + k]);
        }
        g->slot[q][m] = (int8_t)ms.slot[o];
      } else {
        g->slot[q][m] = -1;
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) g->box[q][k] = b[k];
  }
  if (lane == 0) g->n = (uint32_t)ngr;
}

// The top level (and, given a group table, the moved objects' groups):
// every thread of the block gathers the entries' boxes (the dependent loads
// of the roots overlap), then warp 0 builds the top level while warp 1 (warp
// 0 too in a one-warp block) builds the groups.  Called by every thread of
// the block right after pose_bookkeeping: the gather reads nothing that the
// bookkeeping writes, and its barrier orders the bookkeeping's object boxes
// before the groups read them.
__device__ __forceinline__ void build_top_and_groups(WNode* wnodes, const Tri* tris, int top_off, int static_root,
                                                     const DynObj* objs, int n_dyn, int* root_out, uint64_t moved,
                                                     MovedGroups* groups) {
  __shared__ TopSmem ts;
  __shared__ MovedSmem ms;
  for (int e = threadIdx.x; e <= n_dyn; e += blockDim.x) {   // entry 0: the static root; 1 + s: slot s
    const int r = e == 0 ? static_root : objs[e - 1].wroot;
    ts.ref[e] = r;
    if (r != INT32_MIN) ref_box(wnodes, tris, r, ts.box[e]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) top_build_warp(ts, n_dyn, wnodes, top_off, root_out, lane);
  if (groups && warp == (blockDim.x >= 64 ? 1 : 0)) moved_groups_warp(ms, objs, n_dyn, moved, groups, lane);
}

}  // namespace pvk
