// Distribution maps (Sec. 3.1): cells of a light's emission sample space.
//
// A rectangle's uniforms (u0, u1) pick the point on it and (u2, u3) =
// (sin^2 theta, phi / 2 pi) the cosine-weighted direction; a point light's
// (u2, u3) = ((1 - z) / 2, phi / 2 pi) pick the direction on the sphere.  A
// cell is a box of these coordinates, so every cell has the same emission
// probability and DM_T spreads a light's N paths evenly over its n cells:
// DM_T(c) = floor(N (c + 1) / n) - floor(N c / n).  A path's cell is decided in
// float32 with correctly rounded +, -, *, / and sqrt only (explicit
// intrinsics, never contracted), from its stored float32 photon and origin
// and the float32 light pose.
#pragma once
#include "pv_device.cuh"

namespace pvk {

// Fraction of a full turn of the angle of (x, y), in [0, 1): the angle to the
// nearer axis from two half-angle steps atan t = 2 atan(t / (1 + sqrt(1 + t^2)))
// and the Gregory series to t^9 (|t| <= tan(pi/16)).
__device__ __forceinline__ float dm_turn(float x, float y) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = ax > ay ? ax : ay, mn = ax > ay ? ay : ax;
  if (!(mx > 0.0f)) return 0.0f;
  float t = __fdiv_rn(mn, mx);
  t = __fdiv_rn(t, __fadd_rn(1.0f, __fsqrt_rn(__fadd_rn(1.0f, __fmul_rn(t, t)))));
  t = __fdiv_rn(t, __fadd_rn(1.0f, __fsqrt_rn(__fadd_rn(1.0f, __fmul_rn(t, t)))));
  const float q = __fmul_rn(t, t);
  // 1/9, 1/7, 1/5, 1/3, pi/2, pi, 2 pi rounded to float32
  float a = 0x1.c71c72p-4f;
  a = __fsub_rn(0x1.24924ap-3f, __fmul_rn(q, a));
  a = __fsub_rn(0x1.99999ap-3f, __fmul_rn(q, a));
  a = __fsub_rn(0x1.555556p-2f, __fmul_rn(q, a));
  a = __fsub_rn(1.0f, __fmul_rn(q, a));
  a = __fmul_rn(4.0f, __fmul_rn(t, a));
  if (ay > ax) a = __fsub_rn(0x1.921fb6p+0f, a);
  if (x < 0.0f) a = __fsub_rn(0x1.921fb6p+1f, a);
  if (y < 0.0f) a = __fsub_rn(0x1.921fb6p+2f, a);
  const float f = __fdiv_rn(a, 0x1.921fb6p+2f);
  return f < 1.0f ? f : 0.0f;
}

__device__ __forceinline__ float dm_dot(float3 a, float3 b) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), __fmul_rn(a.z, b.z));
}

__device__ __forceinline__ float3 dm_sub(float3 a, float3 b) {
  return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}

__device__ __forceinline__ float3 dm_div(float3 a, float s) {
  return make_float3(__fdiv_rn(a.x, s), __fdiv_rn(a.y, s), __fdiv_rn(a.z, s));
}

// Sample-space coordinates of a path under pose L (the parametrisation
// function of Sec. 3.1): first photon x1 and stored origin o (the rectangle's
// kept direction is re-intersected with its plane); false when the path does
// not come from the light.
__device__ __forceinline__ bool dm_param(const LightPose& L, float3 x1, float3 o, float* u) {
  if (L.type == PV_LIGHT_POINT) {
    const float3 dx = dm_sub(x1, L.pos);
    const float len = __fsqrt_rn(dm_dot(dx, dx));
    if (!(len > 0.0f)) return false;
    const float3 d = dm_div(dx, len);
    u[2] = __fmul_rn(__fsub_rn(1.0f, d.z), 0.5f);
    u[3] = dm_turn(d.x, d.y);
    return u[2] >= 0.0f && u[2] < 1.0f;
  }
  const float3 dv = dm_sub(x1, o);
  const float len = __fsqrt_rn(dm_dot(dv, dv));
  if (!(len > 0.0f)) return false;
  const float3 d = dm_div(dv, len);
  const float nd = dm_dot(L.n, d);
  if (!(nd > 0.0f)) return false;
  const float3 x1c = dm_sub(x1, L.pos);
  const float tp = __fdiv_rn(dm_dot(L.n, x1c), nd);
  if (!(tp > 0.0f)) return false;
  const float3 rel = make_float3(__fsub_rn(x1c.x, __fmul_rn(tp, d.x)), __fsub_rn(x1c.y, __fmul_rn(tp, d.y)),
                                 __fsub_rn(x1c.z, __fmul_rn(tp, d.z)));
  u[0] = __fadd_rn(__fdiv_rn(dm_dot(L.t, rel), L.size.x), 0.5f);
  u[1] = __fadd_rn(__fdiv_rn(dm_dot(L.b, rel), L.size.y), 0.5f);
  const float dx = dm_dot(d, L.t), dy = dm_dot(d, L.b);
  u[2] = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
  u[3] = dm_turn(dx, dy);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!(u[k] >= 0.0f && u[k] < 1.0f)) return false;
  return true;
}

__device__ __forceinline__ uint32_t dm_index(float u, uint32_t n) {
  const uint32_t i = (uint32_t)floorf(__fmul_rn(u, (float)n));
  return i < n ? i : n - 1;
}

// Cell of sample-space coordinates u (row-major over the map's dimensions:
// rectangle x, y, theta, phi = u0..u3; point theta, phi = u2, u3).
__device__ __forceinline__ uint32_t dm_cell_of_u(const DmLight& D, const float* u) {
  if (D.dims == 4)
    return ((dm_index(u[0], D.res[0]) * D.res[1] + dm_index(u[1], D.res[1])) * D.res[2] + dm_index(u[2], D.res[2])) *
               D.res[3] + dm_index(u[3], D.res[3]);
  return dm_index(u[2], D.res[0]) * D.res[1] + dm_index(u[3], D.res[1]);
}

__device__ __forceinline__ uint32_t dm_target(const DmLight& D, uint32_t c) {
  const uint64_t N = D.n_paths, n = D.cells;
  return (uint32_t)(((uint64_t)(c + 1) * N) / n - ((uint64_t)c * N) / n);
}

// Cell of the j-th path of a light in a full trace (floor(N c / n) <= j < floor(N (c + 1) / n)).
__device__ __forceinline__ uint32_t dm_stratified(const DmLight& D, uint32_t j) {
  const uint64_t N = D.n_paths, n = D.cells;
  return (uint32_t)((((uint64_t)j + 1) * n - 1) / N);
}

__device__ __forceinline__ float dm_into(float u, uint32_t i, uint32_t n) {
  return __fdiv_rn(__fadd_rn((float)i, u), (float)n);
}

// Restrict an emission's uniforms to cell c: u_k' = (i_k + u_k) / n_k in float32.
__device__ __forceinline__ void dm_restrict(const DmLight& D, uint32_t c, float4& u) {
  if (D.dims == 4) {
    const uint32_t i3 = c % D.res[3], c2 = c / D.res[3];
    const uint32_t i2 = c2 % D.res[2], c1 = c2 / D.res[2];
    const uint32_t i1 = c1 % D.res[1], i0 = c1 / D.res[1];
    u = make_float4(dm_into(u.x, i0, D.res[0]), dm_into(u.y, i1, D.res[1]), dm_into(u.z, i2, D.res[2]),
                    dm_into(u.w, i3, D.res[3]));
  } else {
    const uint32_t i1 = c % D.res[1], i0 = c / D.res[1];
    u.z = dm_into(u.z, i0, D.res[0]);
    u.w = dm_into(u.w, i1, D.res[1]);
  }
}

// ---- the steps after "compute DM_C" (Sec. 3.1), per path or per cell, shared by
// the single-scene kernels (dm.cu) and the batched ones (batch.cu)

constexpr uint32_t kDmFreshMask = PV_INFO_REPLACE | PV_INFO_REUSE_LIGHT | (15u << PV_INFO_START_SHIFT);

// a fresh emission: replace, start 0, no reuse of the light sample
__device__ __forceinline__ bool dm_is_fresh(uint32_t w) { return (w & kDmFreshMask) == PV_INFO_REPLACE; }

__device__ __forceinline__ uint32_t dm_light_of(const FrameLights& L, uint32_t p) {
  uint32_t l = 0;
  while (l + 1 < L.n && p >= L.first[l + 1]) ++l;
  return l;
}

// light l has a map and moved this frame
__device__ __forceinline__ bool dm_moved(const FrameLights& L, uint32_t l) {
  return L.dm[l].dims != 0 && ((L.moved_mask >> l) & 1u) != 0;
}

// Pass 1 for path p: a kept path of a cell with DM_C > DM_T is pruned with
// probability (DM_C - DM_T) / DM_C (Eq. 1): Philox counter (path, 16,
// frame), pruned iff draw24 * DM_C < (DM_C - DM_T) * 2^24.  It becomes a
// fresh emission that still names its old cell (for pass 2).  Returns 1 if
// pruned.
__device__ __forceinline__ uint32_t dm_prune_path(const FrameLights& L, uint32_t p, uint32_t* info, uint64_t seed,
                                                  uint32_t frame) {
  const uint32_t l = dm_light_of(L, p);
  if (!dm_moved(L, l)) return 0u;
  const uint32_t w = info[p];
  if (dm_is_fresh(w)) return 0u;
  const DmLight& D = L.dm[l];
  const uint32_t c = w & 0xFFFFFu;
  const uint32_t dc = D.dmc[c], dt = dm_target(D, c);
  if (dc <= dt) return 0u;
  const uint4 r = philox4x32_10(make_uint4(p, 16u, frame, 0u), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  if ((uint64_t)(r.x >> 8) * dc >= ((uint64_t)(dc - dt) << 24)) return 0u;
  info[p] = info_make((l << 20) | c, 0, 0, true, false);
  return 1u;
}

// Pass 2 for path p: a pruned path leaves its cell; every fresh emission of a
// light with a moved map is counted free.  Returns the compaction flag
// (PV_INFO_REPLACE for a free path).
__device__ __forceinline__ uint32_t dm_commit_path(const FrameLights& L, uint32_t p, const uint32_t* info,
                                                   uint32_t pruned, uint32_t* free_count) {
  const uint32_t l = dm_light_of(L, p);
  if (!dm_moved(L, l)) return 0u;
  const uint32_t w = info[p];
  if (pruned) atomicSub(L.dm[l].dmc + (w & 0xFFFFFu), 1u);
  if (!dm_is_fresh(w)) return 0u;
  atomicAdd(free_count + l, 1u);
  return PV_INFO_REPLACE;
}

// Deficit of cell c (c == cells: 0, the slot the exclusive scan turns into the total).
__device__ __forceinline__ uint32_t dm_deficit(const DmLight& D, uint32_t c) {
  if (c == D.cells) return 0u;
  const uint32_t t = dm_target(D, c), have = D.dmc[c];
  return have < t ? t - have : 0u;
}

// Largest cell c with pre[c] <= j (pre: exclusive prefix of the deficits, j < pre[cells]).
__device__ __forceinline__ uint32_t dm_deficit_cell(const uint32_t* pre, uint32_t cells, uint32_t j) {
  uint32_t lo = 0, hi = cells;                 // pre[lo] <= j, and j < pre[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= j) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Fill: the j-th of the F free paths of light l takes the cell whose deficit
// range holds j; once the deficits are used up, the rest spread evenly over
// the cells.  Writes the path's info word and counts it in its cell.
__device__ __forceinline__ void dm_fill_path(const DmLight& D, uint32_t l, uint32_t p, uint32_t j, uint32_t F,
                                             const uint32_t* pre, uint32_t* info) {
  const uint32_t total = pre[D.cells];
  const uint32_t c = j < total ? dm_deficit_cell(pre, D.cells, j)
                               : (uint32_t)(((uint64_t)(j - total) * D.cells) / (F - total));
  info[p] = info_make((l << 20) | c, 0, 0, true, false);
  atomicAdd(D.dmc + c, 1u);
}

}  // namespace pvk
