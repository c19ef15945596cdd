// Device-side building blocks of the path-verification library (sm_103a).
//
// Layouts
//   Node (64 B): both children's boxes in the parent, so one visit loads one
//   node and tests two boxes:  a = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y),
//   b = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y), c = (c0.lo.z, c0.hi.z, c1.lo.z,
//   c1.hi.z), d = (child0, child1, -, -).  A child index >= 0 is an internal
//   node, ~i (negative) is the leaf holding triangle i.
//   Tri (48 B): v0.xyz + primitive id bits, edge v1-v0, edge v2-v0.
//
// Every loop here is bounded; overflow or cap records a status code and
// returns, never traps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pv.h"

namespace pvk {

constexpr int kStack = 64;            // traversal stack entries (BVH depth bound)
constexpr int kMaxDyn = PV_MAX_DYN_OBJECTS;

struct __align__(16) Node {
  float4 a, b, c;
  int4 d;
};

struct __align__(16) Tri {
  float4 v0;   // w = primitive id (int bits)
  float4 e1;
  float4 e2;
};

// per dynamic object ("slot"), resident on the device
struct DynObj {
  uint32_t user_object;
  uint32_t tri_begin, tri_count;
  int32_t root;              // child-index encoding into the dynamic node array
  float box_new[6];          // tight world box of the current pose (lo xyz, hi xyz)
  float box_old[6];          // tight world box of the previous pose
};

struct LightPose {
  int32_t type;
  float3 pos, n, t, b;       // b = n x t
  float2 size;
  float3 power;
  uint32_t n_paths;
};

// light state passed by value to the kernels
struct FrameLights {
  LightPose cur[PV_MAX_LIGHTS];
  LightPose old[PV_MAX_LIGHTS];
  uint32_t first[PV_MAX_LIGHTS + 1];
  uint32_t n;
  uint32_t moved_mask;       // bit l: light l moved (position, frame or size)
  uint32_t tilted_mask;      // bit l: its normal changed
};

// read-only scene view passed by value to the kernels
struct SceneView {
  const Node* s_nodes;
  const Tri* s_tris;
  int32_t s_root;            // child-index encoding; INT32_MIN = empty
  const Node* d_nodes;
  const Tri* d_tris;
  const DynObj* objs;
  uint32_t n_dyn;
  const uint8_t* prim_slot;  // [n_tris] 255 = static, else dynamic slot
  const uint32_t* prim_dyn;  // [n_tris] index into the dynamic arrays (dynamic prims)
  const float4* prim_alb;    // [n_tris] albedo rgb, w = max (Russian-roulette q)
  const float4* prim_nrm;    // [n_tris] e1 x e2 of the given corners (object-local for dynamic)
  const float* d_local;      // [n_dyn_tris][9] object-local corners, BVH order
  const float* xf_old;       // [kMaxDyn][12] previous pose per slot
  const float* xf_new;       // [kMaxDyn][12] current pose per slot
  uint32_t B;
  float tmin;                // 1e-5 diag
  float close_tol;           // 1e-5 diag
  uint64_t moved;            // bit s: dynamic slot s moved this frame
  uint32_t max_visits;       // traversal visit cap per ray
  int* status;               // sticky device status word
};

// ---------------------------------------------------------------- vectors
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return make_float3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return rsqrtf(dot(a, a)) * a; }
__device__ __forceinline__ float3 normalize_exact(float3 a) {
  float l = sqrtf(dot(a, a));
  return make_float3(a.x / l, a.y / l, a.z / l);
}
__device__ __forceinline__ float maxabs3(float3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }

__device__ __forceinline__ void record_error(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// ---------------------------------------------------------------- random numbers
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds; each
// round multiplies words 0 and 2 by two fixed odd constants, swaps the
// high/low halves across the word pairs with the key xor-ed in, and the key
// is advanced by two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Four 24-bit uniforms keyed by (path, vertex, frame); vertex 0 = emission
// (origin u0,u1; direction u2,u3), vertex k >= 1 = bounce at photon k
// (direction u0,u1; Russian roulette u2).
__device__ __forceinline__ float4 rng4(uint64_t seed, uint32_t path, uint32_t vertex, uint32_t frame) {
  uint4 o = philox4x32_10(make_uint4(path, vertex, frame, 0u), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float s = 5.9604644775390625e-08f;  // 2^-24
  return make_float4((float)(o.x >> 8) * s, (float)(o.y >> 8) * s, (float)(o.z >> 8) * s, (float)(o.w >> 8) * s);
}

// ---------------------------------------------------------------- sampling
// Orthonormal basis about unit n (Duff et al., JCGT 2017), branch on n.z >= 0.
__device__ __forceinline__ void onb(float3 n, float3& b1, float3& b2) {
  const float sg = n.z >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (sg + n.z);
  const float b = n.x * n.y * a;
  b1 = make_float3(1.0f + sg * n.x * n.x * a, sg * b, -sg * n.x);
  b2 = make_float3(b, sg + n.y * n.y * a, -n.y);
}

// cosine-weighted direction (uniform disk point lifted to the hemisphere)
__device__ __forceinline__ float3 cosine_dir(float3 n, float3 b1, float3 b2, float u0, float u1) {
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  const float r = sqrtf(u0);
  const float z = sqrtf(fmaxf(0.0f, 1.0f - u0));
  return normalize_exact((r * c) * b1 + (r * s) * b2 + z * n);
}

__device__ __forceinline__ void emit(const LightPose& L, float4 u, float3& o, float3& d) {
  if (L.type == PV_LIGHT_POINT) {
    o = L.pos;
    const float z = 1.0f - 2.0f * u.z;
    const float r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float s, c;
    sincospif(2.0f * u.w, &s, &c);
    d = normalize_exact(make_float3(r * c, r * s, z));
  } else {
    o = L.pos + ((u.x - 0.5f) * L.size.x) * L.t + ((u.y - 0.5f) * L.size.y) * L.b;
    d = cosine_dir(L.n, L.t, L.b, u.z, u.w);
  }
}

// ---------------------------------------------------------------- ray queries
struct Ray {
  float3 o, d, inv, ooi;   // ooi = -o * inv
  float tmin;
};

__device__ __forceinline__ Ray make_ray(float3 o, float3 d, float tmin) {
  Ray r;
  r.o = o;
  r.d = d;
  const float e = 1e-20f;
  r.inv = make_float3(1.0f / (fabsf(d.x) > e ? d.x : copysignf(e, d.x)),
                      1.0f / (fabsf(d.y) > e ? d.y : copysignf(e, d.y)),
                      1.0f / (fabsf(d.z) > e ? d.z : copysignf(e, d.z)));
  r.ooi = make_float3(-o.x * r.inv.x, -o.y * r.inv.y, -o.z * r.inv.z);
  r.tmin = tmin;
  return r;
}

// Both child boxes of a node against the ray within [tmin, tmax].
__device__ __forceinline__ void box2(const Ray& r, float tmax, const Node& n, bool& h0, bool& h1, float& t0, float& t1) {
  const float ax0 = fmaf(n.a.x, r.inv.x, r.ooi.x), ax1 = fmaf(n.a.y, r.inv.x, r.ooi.x);
  const float ay0 = fmaf(n.a.z, r.inv.y, r.ooi.y), ay1 = fmaf(n.a.w, r.inv.y, r.ooi.y);
  const float az0 = fmaf(n.c.x, r.inv.z, r.ooi.z), az1 = fmaf(n.c.y, r.inv.z, r.ooi.z);
  const float bx0 = fmaf(n.b.x, r.inv.x, r.ooi.x), bx1 = fmaf(n.b.y, r.inv.x, r.ooi.x);
  const float by0 = fmaf(n.b.z, r.inv.y, r.ooi.y), by1 = fmaf(n.b.w, r.inv.y, r.ooi.y);
  const float bz0 = fmaf(n.c.z, r.inv.z, r.ooi.z), bz1 = fmaf(n.c.w, r.inv.z, r.ooi.z);
  t0 = fmaxf(fmaxf(fminf(ax0, ax1), fminf(ay0, ay1)), fmaxf(fminf(az0, az1), r.tmin));
  const float e0 = fminf(fminf(fmaxf(ax0, ax1), fmaxf(ay0, ay1)), fminf(fmaxf(az0, az1), tmax));
  t1 = fmaxf(fmaxf(fminf(bx0, bx1), fminf(by0, by1)), fmaxf(fminf(bz0, bz1), r.tmin));
  const float e1 = fminf(fminf(fmaxf(bx0, bx1), fmaxf(by0, by1)), fminf(fmaxf(bz0, bz1), tmax));
  h0 = t0 <= e0;
  h1 = t1 <= e1;
}

// One box (lo xyz, hi xyz) against the ray within [tmin, tmax]; entry distance.
__device__ __forceinline__ bool box1(const Ray& r, float tmax, const float* bx, float& tenter) {
  const float x0 = fmaf(bx[0], r.inv.x, r.ooi.x), x1 = fmaf(bx[3], r.inv.x, r.ooi.x);
  const float y0 = fmaf(bx[1], r.inv.y, r.ooi.y), y1 = fmaf(bx[4], r.inv.y, r.ooi.y);
  const float z0 = fmaf(bx[2], r.inv.z, r.ooi.z), z1 = fmaf(bx[5], r.inv.z, r.ooi.z);
  tenter = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), r.tmin));
  const float e = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tmax));
  return tenter <= e;
}

// Moller-Trumbore (1997) on the closed triangle, t in (tmin, tmax).
__device__ __forceinline__ bool tri_hit(const Ray& r, const Tri& T, float tmax, float& t) {
  const float3 e1 = f3(T.e1), e2 = f3(T.e2);
  const float3 p = cross(r.d, e2);
  const float det = dot(e1, p);
  if (det == 0.0f) return false;
  const float inv = 1.0f / det;
  const float3 s = r.o - f3(T.v0);
  const float u = dot(s, p) * inv;
  if (!(u >= 0.0f && u <= 1.0f)) return false;
  const float3 q = cross(s, e1);
  const float v = dot(r.d, q) * inv;
  if (!(v >= 0.0f && u + v <= 1.0f)) return false;
  t = dot(e2, q) * inv;
  return t > r.tmin && t < tmax;
}

__device__ __forceinline__ Node load_node(const Node* nodes, int i) {
  const float4* p = reinterpret_cast<const float4*>(nodes + i);
  Node n;
  n.a = __ldg(p);
  n.b = __ldg(p + 1);
  n.c = __ldg(p + 2);
  n.d = __ldg(reinterpret_cast<const int4*>(p + 3));
  return n;
}

__device__ __forceinline__ Tri load_tri(const Tri* tris, int i) {
  const float4* p = reinterpret_cast<const float4*>(tris + i);
  Tri t;
  t.v0 = __ldg(p);
  t.e1 = __ldg(p + 1);
  t.e2 = __ldg(p + 2);
  return t;
}

// Per-thread work counters of the traversal (node visits, triangle tests).
struct Work {
  uint32_t nodes = 0, tris = 0;
};

// Traverse one BVH from ``root``; ANY: stop at the first hit.  ``tbest`` is
// the current closest distance (in/out), ``best`` the hit triangle index.
// Returns false and records an error on stack overflow or visit cap.
template <bool ANY>
__device__ __forceinline__ bool traverse(const Node* nodes, const Tri* tris, int root, const Ray& r, float& tbest,
                                         int& best, int exclude, uint32_t max_visits, int* status, Work& wk) {
  int stack[kStack];
  int sp = 0;
  int node = root;
  uint32_t visits = 0;
  for (;;) {
    if (++visits > max_visits) {
      record_error(status, PV_ERR_ITER_CAP);
      return false;
    }
    if (node >= 0) {
      ++wk.nodes;
      const Node n = load_node(nodes, node);
      bool h0, h1;
      float t0, t1;
      box2(r, tbest, n, h0, h1, t0, t1);
      if (h0 && h1) {
        const bool first0 = t0 <= t1;
        if (sp == kStack) {
          record_error(status, PV_ERR_STACK);
          return false;
        }
        stack[sp++] = first0 ? n.d.y : n.d.x;
        node = first0 ? n.d.x : n.d.y;
        continue;
      }
      if (h0) { node = n.d.x; continue; }
      if (h1) { node = n.d.y; continue; }
    } else {
      const int ti = ~node;
      ++wk.tris;
      const Tri T = load_tri(tris, ti);
      float t;
      if (__float_as_int(T.v0.w) != exclude && tri_hit(r, T, tbest, t)) {
        tbest = t;
        best = ti;
        if (ANY) return true;
      }
    }
    if (sp == 0) return true;
    node = stack[--sp];
  }
}

// Hit record of the two-level query: which array, which triangle.
struct Hit {
  float t;
  int tri;        // index in the static (dyn == false) or dynamic triangle array
  bool dyn;
};

// Closest hit over the static BVH and every dynamic object's BVH at the
// current pose.  ``boxes`` = the dynamic objects' current tight boxes (in
// shared memory), 6 floats each.
__device__ __forceinline__ bool closest_hit(const SceneView& sv, const float* boxes, const Ray& r, int exclude,
                                            Hit& h, Work& wk) {
  float tb = 3.0e38f;
  int best = -1;
  bool dyn = false;
  if (sv.s_root != INT32_MIN) traverse<false>(sv.s_nodes, sv.s_tris, sv.s_root, r, tb, best, exclude, sv.max_visits, sv.status, wk);
  for (uint32_t s = 0; s < sv.n_dyn; ++s) {
    float te;
    if (sv.objs[s].root == INT32_MIN || !box1(r, tb, boxes + 6 * s, te)) continue;
    int b2 = -1;
    traverse<false>(sv.d_nodes, sv.d_tris, sv.objs[s].root, r, tb, b2, exclude, sv.max_visits, sv.status, wk);
    if (b2 >= 0) {
      best = b2;
      dyn = true;
    }
  }
  h.t = tb;
  h.tri = best;
  h.dyn = dyn;
  return best >= 0;
}

// Any hit of the open segment (tmin, tmax) over the static BVH and all
// dynamic objects at the current pose.
__device__ __forceinline__ bool any_hit_all(const SceneView& sv, const float* boxes, const Ray& r, float tmax, int exclude,
                                            Work& wk) {
  float tb = tmax;
  int best = -1;
  if (sv.s_root != INT32_MIN) {
    traverse<true>(sv.s_nodes, sv.s_tris, sv.s_root, r, tb, best, exclude, sv.max_visits, sv.status, wk);
    if (best >= 0) return true;
  }
  for (uint32_t s = 0; s < sv.n_dyn; ++s) {
    float te;
    if (sv.objs[s].root == INT32_MIN || !box1(r, tb, boxes + 6 * s, te)) continue;
    traverse<true>(sv.d_nodes, sv.d_tris, sv.objs[s].root, r, tb, best, exclude, sv.max_visits, sv.status, wk);
    if (best >= 0) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t info_nseg(uint32_t w) { return (w >> PV_INFO_NSEG_SHIFT) & 15u; }
__device__ __forceinline__ uint32_t info_start(uint32_t w) { return (w >> PV_INFO_START_SHIFT) & 15u; }
__device__ __forceinline__ uint32_t info_light(uint32_t w) { return (w >> 20) & 3u; }
__device__ __forceinline__ uint32_t info_make(uint32_t cell, uint32_t nseg, uint32_t start, bool rep, bool reuse) {
  return (cell & PV_INFO_CELL_MASK) | (nseg << PV_INFO_NSEG_SHIFT) | (start << PV_INFO_START_SHIFT) |
         (rep ? PV_INFO_REPLACE : 0u) | (reuse ? PV_INFO_REUSE_LIGHT : 0u);
}

// Warp-aggregated add of ``v`` to a device counter (the calling lanes only).
__device__ __forceinline__ void warp_add(uint32_t* ctr, uint32_t v) {
  if (!ctr) return;
  const unsigned m = __activemask();
  const uint32_t s = __reduce_add_sync(m, v);
  if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && s) atomicAdd(ctr, s);
}

// Block-wide 64-bit sum of per-thread counters, one atomic per block.
__device__ __forceinline__ void block_add64(unsigned long long* ctr, uint32_t v, unsigned long long* sh) {
  unsigned long long s = v;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = s;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long t = l < nw ? sh[l] : 0ull;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0 && t && ctr) atomicAdd(ctr, t);
  }
}

// Block-wide sum of per-thread counters, one atomic per block (all threads
// of the block must call; ``sh`` = 32 words of shared memory).
__device__ __forceinline__ void block_add(uint32_t* ctr, uint32_t v, uint32_t* sh) {
  const uint32_t s = __reduce_add_sync(0xffffffffu, v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = s;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    uint32_t t = l < nw ? sh[l] : 0u;
    t = __reduce_add_sync(0xffffffffu, t);
    if (l == 0 && t && ctr) atomicAdd(ctr, t);
  }
}

}  // namespace pvk

namespace pvk {

// cof(A) n for the 3x3 part A of a row-major 3x4 transform: the normal of a
// triangle transformed by A is cof(A) (e1 x e2).
__device__ __forceinline__ float3 cof_apply(const float* m, float3 n) {
  const float3 c0 = make_float3(m[0], m[4], m[8]);
  const float3 c1 = make_float3(m[1], m[5], m[9]);
  const float3 c2 = make_float3(m[2], m[6], m[10]);
  return n.x * cross(c1, c2) + n.y * cross(c2, c0) + n.z * cross(c0, c1);
}

// Unnormalised geometric normal of a primitive at the old or new pose.
__device__ __forceinline__ float3 prim_normal(const SceneView& sv, int prim, bool old_pose) {
  const float3 n = f3(__ldg(sv.prim_nrm + prim));
  const uint32_t slot = __ldg(sv.prim_slot + prim);
  if (slot == 255u) return n;
  return cof_apply((old_pose ? sv.xf_old : sv.xf_new) + 12 * slot, n);
}

__device__ __forceinline__ bool slot_moved(const SceneView& sv, int prim) {
  if (prim < 0) return false;
  const uint32_t slot = __ldg(sv.prim_slot + prim);
  return slot != 255u && ((sv.moved >> slot) & 1ull);
}

// Eq. 2 per RGB channel: -T E_O <= E_N - E_O <= T E_O (E_O = 0 needs E_N = 0).
__device__ __forceinline__ bool energy_close(float3 EN, float3 EO, float tau) {
  const float en[3] = {EN.x, EN.y, EN.z}, eo[3] = {EO.x, EO.y, EO.z};
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (eo[c] == 0.0f) {
      ok &= en[c] == 0.0f;
    } else {
      const float diff = en[c] - eo[c], lim = tau * eo[c];
      ok &= (-lim <= diff) && (diff <= lim);
    }
  }
  return ok;
}

// Load the dynamic objects' boxes into shared memory: ``cull`` = current
// tight box padded by a relative 2^-20 (ray culling only), ``uni`` = exact
// union of the old and new tight boxes (the Sec. 3.2 box test).
__device__ __forceinline__ void load_boxes(const SceneView& sv, float* cull, float* uni) {
  for (uint32_t i = threadIdx.x; i < sv.n_dyn * 6; i += blockDim.x) {
    const DynObj& o = sv.objs[i / 6];
    const int k = i % 6;
    const float bn = o.box_new[k], bo = o.box_old[k];
    const float lo3 = fmaxf(fmaxf(fabsf(o.box_new[0]), fabsf(o.box_new[1])), fabsf(o.box_new[2]));
    const float hi3 = fmaxf(fmaxf(fabsf(o.box_new[3]), fabsf(o.box_new[4])), fabsf(o.box_new[5]));
    const float pad = 9.5367431640625e-07f * fmaxf(lo3, hi3) + 1e-30f;
    cull[i] = k < 3 ? bn - pad : bn + pad;
    if (uni) uni[i] = k < 3 ? fminf(bn, bo) : fmaxf(bn, bo);
  }
}

}  // namespace pvk
