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

#ifndef PV_STACK
#define PV_STACK 64
#endif
constexpr int kStack = PV_STACK;      // traversal stack entries (BVH depth bound)
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

// Wide (4-child) traversal node, 128 B = one cache line: the four child
// boxes stored per coordinate, then the four child references.  A reference
// >= 0 is a wide node; < 0 is a leaf range ~(first | (count - 1) << 29) of
// 1..4 consecutive triangles.  Unused slots carry an empty box.
struct __align__(128) WNode {
  float4 lox, hix, loy, hiy, loz, hiz;
  int4 child;
  int4 pad;
};

#ifndef PV_LEAF_MAX
#define PV_LEAF_MAX 1
#endif
constexpr int kLeafMax = PV_LEAF_MAX;   // triangles per wide leaf range (dynamic objects: 1 for the direct refit)
// Leaves of the static tree: measured on the city and villa workloads, 2 or 3
// triangles per leaf cut node visits per ray by 3-6 % but added 11-40 % triangle
// tests and did not speed the re-trace up; 4 made it 13-16 % slower.
#ifndef PV_STATIC_LEAF_MAX
#define PV_STATIC_LEAF_MAX 1
#endif
constexpr int kStaticLeafMax = PV_STATIC_LEAF_MAX;   // triangles per leaf range of the static tree (at most 8)

__host__ __device__ __forceinline__ int leaf_ref(uint32_t first, uint32_t count) {
  return ~(int)(first | ((count - 1u) << 29));
}
__host__ __device__ __forceinline__ uint32_t leaf_first(int ref) { return (uint32_t)(~ref) & 0x1FFFFFFFu; }
__host__ __device__ __forceinline__ uint32_t leaf_count(int ref) { return ((uint32_t)(~ref) >> 29) + 1u; }

// per dynamic object ("slot"), resident on the device
struct DynObj {
  uint32_t user_object;
  uint32_t tri_begin, tri_count;
  int32_t root;              // binary subtree root (child-index encoding), INT32_MIN if none
  int32_t wroot;             // wide subtree root reference, INT32_MIN if none
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

// Distribution map of one light (Sec. 3.1): cells over its emission sample
// space (see dm_core.cuh) and its device counts DM_C.
struct DmLight {
  uint32_t res[4];           // cells per dimension: rectangle x, y, theta, phi; point theta, phi
  uint32_t dims;             // 4 rectangle, 2 point, 0 no map
  uint32_t cells;
  uint32_t n_paths;          // N: DM_T spreads N paths over the cells
  uint32_t* dmc;             // DM_C [cells]
};

// The moved objects in spatial groups of up to four, rebuilt with the top
// level each frame in which objects move: sorted along the axis of widest
// centroid spread, cut into consecutive groups.  A group's box is the union
// of its members' old-and-new boxes, so the Sec. 3.2 box test can reject a
// segment against a group before testing its members, with the same result.
#ifndef PV_GROUP_SIZE
#define PV_GROUP_SIZE 4
#endif
constexpr int kGroupSize = PV_GROUP_SIZE;
constexpr int kMaxGroups = (kMaxDyn + kGroupSize - 1) / kGroupSize;
struct MovedGroups {
  uint32_t n;                                  // groups in use
  uint32_t pad;
  float box[kMaxGroups][6];                    // lo xyz, hi xyz
  int8_t slot[kMaxGroups][kGroupSize];         // member slots, -1 past the last
};

// light state passed by value to the kernels
struct FrameLights {
  LightPose cur[PV_MAX_LIGHTS];
  LightPose old[PV_MAX_LIGHTS];
  uint32_t first[PV_MAX_LIGHTS + 1];
  uint32_t n;
  uint32_t moved_mask;       // bit l: light l moved (position, frame or size)
  uint32_t tilted_mask;      // bit l: its normal changed
  DmLight dm[PV_MAX_LIGHTS];
};

// read-only scene view passed by value to the kernels
struct SceneView {
  const WNode* nodes;        // wide nodes [static tree | dynamic objects | top level]
  const Tri* tris;           // [static references | dynamic triangles]
  const int* root;           // device word: root child index of the whole scene (INT32_MIN = empty)
  const DynObj* objs;
  const MovedGroups* groups;   // moved objects in groups (valid in frames where objects moved)
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
  uint32_t n_static_wide;    // wide nodes of the static tree, [0, n_static_wide), in breadth-first order
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
  const float a = -__frcp_rn(sg + n.z);     // = -1 / (sg + n.z), correctly rounded
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
  // __frcp_rn: the correctly rounded 1 / x, i.e. exactly what IEEE division gives
  r.inv = make_float3(__frcp_rn(fabsf(d.x) > e ? d.x : copysignf(e, d.x)),
                      __frcp_rn(fabsf(d.y) > e ? d.y : copysignf(e, d.y)),
                      __frcp_rn(fabsf(d.z) > e ? d.z : copysignf(e, d.z)));
  r.ooi = make_float3(-o.x * r.inv.x, -o.y * r.inv.y, -o.z * r.inv.z);
  r.tmin = tmin;
  return r;
}

// A wide node's child boxes as seen by one ray: along each axis the plane
// the ray meets first ("near": lo for a positive direction component, hi for
// a negative one) and the other ("far"), picked by the load address.
struct WNodeRay {
  float4 nx, fx, ny, fy, nz, fz;
  int4 child;
};

__device__ __forceinline__ WNodeRay load_wnode_ray(const WNode* nodes, int i, const Ray& r) {
  const float4* p = reinterpret_cast<const float4*>(nodes + i);
  const uint32_t sx = __float_as_uint(r.inv.x) >> 31, sy = __float_as_uint(r.inv.y) >> 31;
  const uint32_t sz = __float_as_uint(r.inv.z) >> 31;
  WNodeRay n;
  n.nx = __ldg(p + sx);
  n.fx = __ldg(p + (1u - sx));
  n.ny = __ldg(p + 2u + sy);
  n.fy = __ldg(p + (3u - sy));
  n.nz = __ldg(p + 4u + sz);
  n.fz = __ldg(p + (5u - sz));
  n.child = __ldg(reinterpret_cast<const int4*>(p + 6));
  return n;
}

// The same through a generic pointer: node i comes from ``cache`` (a shared
// copy of wide nodes [0, n_cache)) when i < n_cache, else from ``nodes``.
__device__ __forceinline__ WNodeRay load_wnode_ray_cached(const WNode* nodes, const WNode* cache, int n_cache, int i,
                                                          const Ray& r) {
  const float4* p = reinterpret_cast<const float4*>((unsigned)i < (unsigned)n_cache ? cache + i : nodes + i);
  const uint32_t sx = __float_as_uint(r.inv.x) >> 31, sy = __float_as_uint(r.inv.y) >> 31;
  const uint32_t sz = __float_as_uint(r.inv.z) >> 31;
  WNodeRay n;
  n.nx = p[sx];
  n.fx = p[1u - sx];
  n.ny = p[2u + sy];
  n.fy = p[3u - sy];
  n.nz = p[4u + sz];
  n.fz = p[5u - sz];
  n.child = reinterpret_cast<const int4*>(p)[6];
  return n;
}

// Three-input minimum / maximum: one instruction on sm_100 and later, with the
// NaN rule of fminf / fmaxf (a NaN operand is ignored unless all are NaN).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// The four child boxes of a wide node against the ray within [tmin, tmax]:
// entry distances, hit mask (bit c = child c).  For a box with lo <= hi the
// near plane's distance is exactly the smaller of the two slab distances
// (fmaf is monotone in the plane coordinate), so this is the classic slab
// test without its per-axis min / max; an unused slot (lo > hi) misses.
__device__ __forceinline__ uint32_t box4(const Ray& r, float tmax, const WNodeRay& n, float t[4]) {
  const float nx[4] = {n.nx.x, n.nx.y, n.nx.z, n.nx.w}, fx[4] = {n.fx.x, n.fx.y, n.fx.z, n.fx.w};
  const float ny[4] = {n.ny.x, n.ny.y, n.ny.z, n.ny.w}, fy[4] = {n.fy.x, n.fy.y, n.fy.z, n.fy.w};
  const float nz[4] = {n.nz.x, n.nz.y, n.nz.z, n.nz.w}, fz[4] = {n.fz.x, n.fz.y, n.fz.z, n.fz.w};
  uint32_t mask = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float tn = fmax3(fmaf(nx[c], r.inv.x, r.ooi.x), fmaf(ny[c], r.inv.y, r.ooi.y),
                           fmaxf(fmaf(nz[c], r.inv.z, r.ooi.z), r.tmin));
    const float tf = fmin3(fmaf(fx[c], r.inv.x, r.ooi.x), fmaf(fy[c], r.inv.y, r.ooi.y),
                           fminf(fmaf(fz[c], r.inv.z, r.ooi.z), tmax));
    t[c] = tn;
    mask |= (tn <= tf ? 1u : 0u) << c;
  }
  return mask;
}

// One box (lo xyz, hi xyz) against the ray within [tmin, tmax]; entry distance.
__device__ __forceinline__ bool box1(const Ray& r, float tmax, const float* bx, float& tenter) {
  const float x0 = fmaf(bx[0], r.inv.x, r.ooi.x), x1 = fmaf(bx[3], r.inv.x, r.ooi.x);
  const float y0 = fmaf(bx[1], r.inv.y, r.ooi.y), y1 = fmaf(bx[4], r.inv.y, r.ooi.y);
  const float z0 = fmaf(bx[2], r.inv.z, r.ooi.z), z1 = fmaf(bx[5], r.inv.z, r.ooi.z);
  tenter = fmax3(fminf(x0, x1), fminf(y0, y1), fmaxf(fminf(z0, z1), r.tmin));
  const float e = fmin3(fmaxf(x0, x1), fmaxf(y0, y1), fminf(fmaxf(z0, z1), tmax));
  return tenter <= e;
}

// Moller-Trumbore (1997) on the closed triangle, t in (tmin, tmax].
__device__ __forceinline__ bool tri_hit(const Ray& r, const Tri& T, float tmax, float& t) {
  const float3 e1 = f3(T.e1), e2 = f3(T.e2);
  const float3 p = cross(r.d, e2);
  const float det = dot(e1, p);
  if (det == 0.0f) return false;
  const float inv = __frcp_rn(det);         // correctly rounded, as 1.0f / det
  const float3 s = r.o - f3(T.v0);
  const float u = dot(s, p) * inv;
  if (!(u >= 0.0f && u <= 1.0f)) return false;
  const float3 q = cross(s, e1);
  const float v = dot(r.d, q) * inv;
  if (!(v >= 0.0f && u + v <= 1.0f)) return false;
  t = dot(e2, q) * inv;
  return t > r.tmin && t <= tmax;
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

// Visit a wide node: push the hit children far-to-near, return the nearest
// in ``next`` (INT32_MIN if none was hit).  False on stack overflow.  The
// four (distance, child) pairs are ordered by a five-comparator sorting
// network on registers, misses carrying an infinite distance.
__device__ __forceinline__ void cswap(float& ka, int& va, float& kb, int& vb) {
  const bool s = kb < ka;
  const float k = s ? kb : ka;
  const int v = s ? vb : va;
  kb = s ? ka : kb;
  vb = s ? va : vb;
  ka = k;
  va = v;
}

// Traversal stack of one thread, S entries.  The first SH entries live in
// shared memory, entry i at sh[i * STRIDE] with STRIDE = the block's thread
// count: the lanes of a warp then touch 32 different banks whatever their
// stack depths, where a local-memory stack spreads divergent depths over as
// many cache lines.  Deeper entries live in a local array.  SH = 0 is a
// plain local stack.
template <int S, int SH = 0, int STRIDE = 1>
struct TStack {
  static constexpr int kSize = S;
  int* sh;                                    // this thread's first shared entry
  int loc[S > SH ? S - SH : 1];
  __device__ __forceinline__ int get(int i) const {
    if (SH == 0) return loc[i];
    if (SH >= S) return sh[i * STRIDE];
    return i < SH ? sh[i * STRIDE] : loc[i - SH];
  }
  __device__ __forceinline__ void set(int i, int v) {
    if (SH == 0) {
      loc[i] = v;
    } else if (SH >= S) {
      sh[i * STRIDE] = v;
    } else if (i < SH) {
      sh[i * STRIDE] = v;
    } else {
      loc[i - SH] = v;
    }
  }
};

template <int S = kStack, class Stk>
__device__ __forceinline__ bool visit_wide(const WNodeRay& n, const Ray& r, float tbest, Stk& stk, int& sp, int& next) {
  float t[4];
  const uint32_t mask = box4(r, tbest, n, t);
  const int m = __popc(mask);
  if (m == 0) {
    next = INT32_MIN;
    return true;
  }
  const float inf = __int_as_float(0x7f800000);
  float k0 = (mask & 1u) ? t[0] : inf, k1 = (mask & 2u) ? t[1] : inf;
  float k2 = (mask & 4u) ? t[2] : inf, k3 = (mask & 8u) ? t[3] : inf;
  int v0 = n.child.x, v1 = n.child.y, v2 = n.child.z, v3 = n.child.w;
  cswap(k0, v0, k1, v1);
  cswap(k2, v2, k3, v3);
  cswap(k0, v0, k2, v2);
  cswap(k1, v1, k3, v3);
  cswap(k1, v1, k2, v2);
  if (sp + m - 1 > S) return false;
  if (m >= 4) stk.set(sp++, v3);
  if (m >= 3) stk.set(sp++, v2);
  if (m >= 2) stk.set(sp++, v1);
  next = v0;
  return true;
}

// Test the triangles of a leaf range; true if the closest hit improved.
__device__ __forceinline__ bool visit_leaf(const Tri* tris, int ref, const Ray& r, float& tbest, int& best, int exclude,
                                           Work& wk) {
  const uint32_t first = leaf_first(ref), cnt = leaf_count(ref);
  bool any = false;
  for (uint32_t i = 0; i < cnt; ++i) {
    ++wk.tris;
    const Tri T = load_tri(tris, (int)(first + i));
    float t;
    // closest first, the lower triangle index among equal distances: the answer does not depend on
    // the order in which leaves are visited
    if (__float_as_int(T.v0.w) != exclude && tri_hit(r, T, tbest, t) &&
        (t < tbest || (best >= 0 && (int)(first + i) < best))) {
      tbest = t;
      best = (int)(first + i);
      any = true;
    }
  }
  return any;
}

// Traverse the wide tree from ``root``; ANY: stop at the first hit.
// ``tbest`` is the current closest distance (in/out), ``best`` the hit
// triangle index.  Returns false and records an error on stack overflow or
// visit cap.
template <bool ANY, int S = kStack>
__device__ __forceinline__ bool traverse(const WNode* nodes, const Tri* tris, int root, const Ray& r, float& tbest,
                                         int& best, int exclude, uint32_t max_visits, int* status, Work& wk) {
  TStack<S> stack;
  int sp = 0;
  int node = root;
  uint32_t visits = 0;
  for (;;) {
    if (node != INT32_MIN) {
      if (++visits > max_visits) {
        record_error(status, PV_ERR_ITER_CAP);
        return false;
      }
      if (node >= 0) {
        ++wk.nodes;
        const WNodeRay n = load_wnode_ray(nodes, node, r);
        int next;
        if (!visit_wide<S>(n, r, tbest, stack, sp, next)) {
          record_error(status, PV_ERR_STACK);
          return false;
        }
        if (next != INT32_MIN) {
          node = next;
          continue;
        }
      } else {
        if (visit_leaf(tris, node, r, tbest, best, exclude, wk) && ANY) return true;
      }
    }
    if (sp == 0) return true;
    node = stack.get(--sp);
  }
}

// Hit record of a scene query: distance and triangle index (in sv.tris).
struct Hit {
  float t;
  int tri;
};

// Closest hit over the whole scene (top level, static tree, dynamic objects).
template <int S = kStack>
__device__ __forceinline__ bool closest_hit(const SceneView& sv, int root, const Ray& r, int exclude, Hit& h, Work& wk) {
  float tb = 3.0e38f;
  int best = -1;
  if (root != INT32_MIN) traverse<false, S>(sv.nodes, sv.tris, root, r, tb, best, exclude, sv.max_visits, sv.status, wk);
  h.t = tb;
  h.tri = best;
  return best >= 0;
}

// Any hit of the open segment (tmin, tmax) over the whole scene.
template <int S = kStack>
__device__ __forceinline__ bool any_hit_all(const SceneView& sv, int root, const Ray& r, float tmax, int exclude,
                                            Work& wk) {
  float tb = tmax;
  int best = -1;
  if (root != INT32_MIN) traverse<true, S>(sv.nodes, sv.tris, root, r, tb, best, exclude, sv.max_visits, sv.status, wk);
  return best >= 0;
}

// Resumable traversal state of one ray (used by the persistent kernels).
struct Trav {
  int node, sp, best;
  float tbest;
  uint32_t visits;
};

__device__ __forceinline__ void trav_begin(Trav& t, int root) {
  t.node = root;
  t.sp = 0;
  t.best = -1;
  t.tbest = 3.0e38f;
  t.visits = 0;
}

// One traversal step (one wide node or one leaf range); true once the ray is done.
// ``stk`` holds S entries.  With ``cache`` non-null, wide nodes below
// ``n_cache`` are read from that shared copy.
template <int S = kStack, class Stk>
__device__ __forceinline__ bool trav_step(const SceneView& sv, const Ray& r, Trav& t, Stk& stk, int exclude, Work& wk,
                                          const WNode* cache = nullptr, int n_cache = 0) {
  if (t.node != INT32_MIN) {
    if (++t.visits > sv.max_visits) {
      record_error(sv.status, PV_ERR_ITER_CAP);
      return true;
    }
    if (t.node >= 0) {
      ++wk.nodes;
      const WNodeRay n = cache ? load_wnode_ray_cached(sv.nodes, cache, n_cache, t.node, r)
                               : load_wnode_ray(sv.nodes, t.node, r);
      int next;
      if (!visit_wide<S>(n, r, t.tbest, stk, t.sp, next)) {
        record_error(sv.status, PV_ERR_STACK);
        return true;
      }
      if (next != INT32_MIN) {
        t.node = next;
        return false;
      }
    } else {
      visit_leaf(sv.tris, t.node, r, t.tbest, t.best, exclude, wk);
    }
  }
  if (t.sp == 0) return true;
  t.node = stk.get(--t.sp);
  return false;
}

__device__ __forceinline__ uint32_t info_nseg(uint32_t w) { return (w >> PV_INFO_NSEG_SHIFT) & 15u; }
__device__ __forceinline__ uint32_t info_start(uint32_t w) { return (w >> PV_INFO_START_SHIFT) & 15u; }
__device__ __forceinline__ uint32_t info_light(uint32_t w) { return (w >> 20) & 3u; }
__device__ __forceinline__ uint32_t info_make(uint32_t cell, uint32_t nseg, uint32_t start, bool rep, bool reuse) {
  return (cell & PV_INFO_CELL_MASK) | (nseg << PV_INFO_NSEG_SHIFT) | (start << PV_INFO_START_SHIFT) |
         (rep ? PV_INFO_REPLACE : 0u) | (reuse ? PV_INFO_REUSE_LIGHT : 0u);
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialisation waits in grid_dependency_wait() until the
// kernel before it has completed and its memory operations are visible; for
// an ordinary launch the wait returns at once.  launch_dependents() lets the
// next such kernel be scheduled once every block of this one has issued it.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Warp-aggregated add of ``v`` to a device counter (the calling lanes only).
__device__ __forceinline__ void warp_add(uint32_t* ctr, uint32_t v) {
  if (!ctr) return;
  const unsigned m = __activemask();
  const uint32_t s = __reduce_add_sync(m, v);
  if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && s) atomicAdd(ctr, s);
}

// Block-wide sums of K per-thread counters with one pair of barriers, then one
// atomic per non-zero counter per block (``sh`` = 32*K words of shared memory).
template <int K>
__device__ __forceinline__ void block_add_n(uint32_t* const (&ctr)[K], const uint32_t (&v)[K], uint32_t* sh) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  uint32_t s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = __reduce_add_sync(0xffffffffu, v[k]);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[32 * k + w] = s[k];
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t t = __reduce_add_sync(0xffffffffu, l < nw ? sh[32 * k + l] : 0u);
      if (l == 0 && t && ctr[k]) atomicAdd(ctr[k], t);
    }
  }
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
