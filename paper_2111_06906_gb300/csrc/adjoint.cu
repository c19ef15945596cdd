// Differentiable deposit model, its adjoint, and budgeted re-trace lists.
//
// The paper has no gradients.  This model ranks the paths to re-trace when a
// ray budget cannot cover every path the Eq. 2 test invalidated.  Each stored
// path keeps its triangles and sampled directions; under parameters theta
//   - the emission follows the light: a point light at p re-aims from p
//     along the stored first segment; a rectangle keeps the stored point
//     (alpha, beta) and direction (ell) in its frame, with the tangent t
//     fixed and the normal n free: o = p + alpha t + beta (n x t) and
//     d0 = ell.x t + ell.y (n x t) + ell.z n;
//   - photon k is re-found on its triangle's plane (unit normal nu_k through
//     the stored photon, translated with its dynamic object) along the stored
//     incoming direction: x_k = x_{k-1} + d nu.(q_k - x_{k-1}) / (nu.d);
//   - energies scale with the light's intensity factor;
//   - photons splat with the uniform cubic B-spline over 4 x 4 texels
//     (C2, texel centres at half-integers, texels outside dropped).
// theta = per light [pos 3, normal 3, scale 1], then per dynamic object in
// slot order [translation 3].  At the current pose the model reproduces the
// stored photons.  The adjoint runs the chain backwards per path:
//   dx_k/dx_{k-1} = I - d nu^T/(nu.d),  dx_k/dq_k = d nu^T/(nu.d),
//   dx_1/do = I - d0 nu^T/(nu.d0),      dx_1/dd0 = tau_1 (I - d0 nu^T/(nu.d0)).
#include <cstring>

#include "pv_scene.h"

using namespace pvk;

namespace {

constexpr int kMaxTheta = 7 * PV_MAX_LIGHTS + 3 * kMaxDyn;

struct ModelArgs {
  uint32_t n, n_lights, n_theta;
  const uint32_t* info;
  const float* origin;
  const float4* pa;
  const float4* pb;
  const float* theta;           // device [n_theta]
  uint32_t W, H;
  float x0, z0, x1, z1;
  float cur_t[kMaxDyn][3];      // current translation of each dynamic slot
};

struct Emission {
  float3 o, d0, t, ell;
  float beta;
  bool rect;
};

__device__ __forceinline__ float3 load3(const float* p) { return make_float3(p[0], p[1], p[2]); }

// Emission of the model path under the light's parameters tl (shared memory).
__device__ __forceinline__ Emission model_emission(const LightPose& Lp, const float* tl, const ModelArgs& A,
                                                   uint32_t p, float3 x10) {
  Emission e;
  const float3 o0 = make_float3(A.origin[p], A.origin[A.n + p], A.origin[2 * (size_t)A.n + p]);
  const float3 d00 = x10 - o0;
  e.t = Lp.t;
  e.rect = Lp.type != PV_LIGHT_POINT;
  if (!e.rect) {
    e.o = load3(tl);
    e.d0 = d00;
    e.beta = 0.f;
    e.ell = make_float3(0.f, 0.f, 0.f);
  } else {
    const float3 rel = o0 - Lp.pos;
    const float alpha = dot(Lp.t, rel);
    e.beta = dot(Lp.b, rel);
    e.ell = make_float3(dot(Lp.t, d00), dot(Lp.b, d00), dot(Lp.n, d00));
    const float3 nl = load3(tl + 3);
    const float3 bl = cross(nl, Lp.t);
    e.o = load3(tl) + alpha * Lp.t + e.beta * bl;
    e.d0 = e.ell.x * Lp.t + e.ell.y * bl + e.ell.z * nl;
  }
  return e;
}

// Unit normal of stored photon v's triangle and its dynamic slot (-1: static).
__device__ __forceinline__ float3 photon_normal(const SceneView& sv, float4 v, int& slot) {
  const int prim = __float_as_int(v.w);
  const uint32_t sl = __ldg(sv.prim_slot + prim);
  slot = sl == 255u ? -1 : (int)sl;
  return normalize(prim_normal(sv, prim, false));
}

// Plane point of stored photon v, moved with its object's translation.
__device__ __forceinline__ float3 photon_point(const ModelArgs& A, const float* s_th, float4 v, int slot) {
  float3 q = f3(v);
  if (slot >= 0) {
    const float* tt = s_th + 7 * A.n_lights + 3 * slot;
    q = q + make_float3(tt[0] - A.cur_t[slot][0], tt[1] - A.cur_t[slot][1], tt[2] - A.cur_t[slot][2]);
  }
  return q;
}

// Uniform cubic B-spline footprint of (x, z): with u = (x - x0) W/(x1 - x0) - 1/2
// (texel-centre coordinate), i0 = floor(u) and f = u - i0, texels i0-1 .. i0+2
// get the cardinal weights (1-f)^3/6, (3f^3 - 6f^2 + 4)/6,
// (-3f^3 + 3f^2 + 3f + 1)/6, f^3/6 (derivatives -(1-f)^2/2, (3f^2 - 4f)/2,
// (-3f^2 + 2f + 1)/2, f^2/2); the 2-D weight is the product over x and z.
struct Spline {
  int i0, j0;                 // texel of tap 0 in x and z
  float wx[4], dx[4], wz[4], dz[4];
  float sx, sz;
};

__device__ __forceinline__ void bspline1(float f, float* w, float* d) {
  const float g = 1.f - f, f2 = f * f, f3 = f2 * f;
  w[0] = g * g * g * (1.f / 6.f);
  w[1] = (3.f * f3 - 6.f * f2 + 4.f) * (1.f / 6.f);
  w[2] = (-3.f * f3 + 3.f * f2 + 3.f * f + 1.f) * (1.f / 6.f);
  w[3] = f3 * (1.f / 6.f);
  d[0] = -0.5f * g * g;
  d[1] = 0.5f * (3.f * f2 - 4.f * f);
  d[2] = 0.5f * (-3.f * f2 + 2.f * f + 1.f);
  d[3] = 0.5f * f2;
}

__device__ __forceinline__ Spline spline(const ModelArgs& A, float x, float z) {
  Spline b;
  b.sx = (float)A.W / (A.x1 - A.x0);
  b.sz = (float)A.H / (A.z1 - A.z0);
  const float u = (x - A.x0) * b.sx - 0.5f, v = (z - A.z0) * b.sz - 0.5f;
  const float fi = floorf(u), fj = floorf(v);
  bspline1(u - fi, b.wx, b.dx);
  bspline1(v - fj, b.wz, b.dz);
  // far outside: keep the indices representable (every tap is dropped)
  b.i0 = (int)fmaxf(fminf(fi, 1e9f), -1e9f) - 1;
  b.j0 = (int)fmaxf(fminf(fj, 1e9f), -1e9f) - 1;
  return b;
}

// Add 12 consecutive floats (one row of four RGB taps) with the widest
// aligned vector atomics (sm_90+ global float2/float4 atomicAdd).  O = floats
// by which p lies past a 16-byte boundary; every index is a constant so v
// stays in registers.
template <int O>
__device__ __forceinline__ void add_row12_at(float* p, const float* v) {
  int i = 0;
  if (O == 1) {
    atomicAdd(p, v[0]);
    atomicAdd(reinterpret_cast<float2*>(p + 1), make_float2(v[1], v[2]));
    i = 3;
  } else if (O == 2) {
    atomicAdd(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
    i = 2;
  } else if (O == 3) {
    atomicAdd(p, v[0]);
    i = 1;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (i + 4 <= 12) {
      atomicAdd(reinterpret_cast<float4*>(p + i), make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
      i += 4;
    }
  if (i + 2 <= 12) {
    atomicAdd(reinterpret_cast<float2*>(p + i), make_float2(v[i], v[i + 1]));
    i += 2;
  }
  if (i < 12) atomicAdd(p + i, v[i]);
}

// p must be 4-byte aligned inside a 16-byte aligned array.
__device__ __forceinline__ void add_row12(float* p, const float* v) {
  switch ((reinterpret_cast<uintptr_t>(p) >> 2) & 3u) {
    case 0: add_row12_at<0>(p, v); break;
    case 1: add_row12_at<1>(p, v); break;
    case 2: add_row12_at<2>(p, v); break;
    default: add_row12_at<3>(p, v); break;
  }
}

__device__ __forceinline__ void stage_theta(const ModelArgs& A, float* s_th) {
  for (uint32_t j = threadIdx.x; j < A.n_theta; j += blockDim.x) s_th[j] = A.theta[j];
}

__global__ void __launch_bounds__(256) k_model_deposit(SceneView sv, FrameLights L, ModelArgs A, float* atlas) {
  __shared__ float s_th[kMaxTheta];
  const bool vec_ok = (reinterpret_cast<uintptr_t>(atlas) & 15u) == 0;
  stage_theta(A, s_th);
  __syncthreads();
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= A.n) return;
  const uint32_t w = A.info[p];
  const uint32_t nseg = min(info_nseg(w), sv.B), l = info_light(w);
  if (nseg == 0) return;
  float4 v = A.pa[p];
  const Emission e = model_emission(L.cur[l], s_th + 7 * l, A, p, f3(v));
  const float sc = s_th[7 * l + 6];
  float3 prev = e.o, dir = e.d0;
  for (uint32_t k = 1; k <= nseg; ++k) {
    int slot;
    const float3 nu = photon_normal(sv, v, slot);
    const float3 q = photon_point(A, s_th, v, slot);
    const float3 x = prev + (dot(nu, q - prev) / dot(nu, dir)) * dir;
    const float3 E = sc * f3(A.pb[(size_t)(k - 1) * A.n + p]);
    const Spline b = spline(A, x.x, x.z);
    const bool row_inside = b.i0 >= 0 && b.i0 + 3 < (int)A.W;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int tj = b.j0 + r;
      if (tj < 0 || tj >= (int)A.H) continue;
      if (row_inside && vec_ok) {
        float rv[12];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float wc = b.wx[c] * b.wz[r];
          rv[3 * c] = E.x * wc;
          rv[3 * c + 1] = E.y * wc;
          rv[3 * c + 2] = E.z * wc;
        }
        add_row12(atlas + 3 * ((size_t)tj * A.W + b.i0), rv);
        continue;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ti = b.i0 + c;
        if (ti < 0 || ti >= (int)A.W) continue;
        float* t = atlas + 3 * ((size_t)tj * A.W + ti);
        const float wc = b.wx[c] * b.wz[r];
        atomicAdd(t + 0, E.x * wc);
        atomicAdd(t + 1, E.y * wc);
        atomicAdd(t + 2, E.z * wc);
      }
    }
    if (k < nseg) {
      const float4 vn = A.pa[(size_t)k * A.n + p];
      dir = f3(vn) - f3(v);                     // stored direction of the next segment
      v = vn;
    }
    prev = x;
  }
}

// Reverse mode, one path per thread: the forward pass keeps the splat
// gradient of each photon position (only x and z are nonzero); the backward
// pass reloads the planes and directions.  dtheta is reduced per block in
// shared memory, then added to the global vector.
__global__ void __launch_bounds__(128) k_adjoint(SceneView sv, FrameLights L, ModelArgs A, const float* G,
                                                 float* dtheta, float* score) {
  __shared__ float s_th[kMaxTheta];
  __shared__ float s_acc[kMaxTheta];
  stage_theta(A, s_th);
  for (uint32_t j = threadIdx.x; j < A.n_theta; j += blockDim.x) s_acc[j] = 0.f;
  __syncthreads();
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  float lc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // this path's light gradient
  int my_l = -1;
  if (p < A.n) {
    const uint32_t w = A.info[p];
    const uint32_t nseg = min(info_nseg(w), sv.B), l = info_light(w);
    float sgE = 0.f;
    if (nseg > 0) {
      my_l = (int)l;
      float2 gpos[PV_MAX_BOUNCES + 1];
      const float4 v1 = A.pa[p];
      const Emission e = model_emission(L.cur[l], s_th + 7 * l, A, p, f3(v1));
      const float sc = s_th[7 * l + 6];
      float3 prev = e.o, dir = e.d0;
      float4 v = v1;
      float gscale = 0.f, tau1 = 0.f;
      for (uint32_t k = 1; k <= nseg; ++k) {
        int slot;
        const float3 nu = photon_normal(sv, v, slot);
        const float3 q = photon_point(A, s_th, v, slot);
        const float tau = dot(nu, q - prev) / dot(nu, dir);
        if (k == 1) tau1 = tau;
        const float3 x = prev + tau * dir;
        const float3 E0 = f3(A.pb[(size_t)(k - 1) * A.n + p]);
        const Spline b = spline(A, x.x, x.z);
        float2 g = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int tj = b.j0 + r;
          if (tj < 0 || tj >= (int)A.H) continue;
          float gr = 0.f, gdx = 0.f, gdz = 0.f;       // row sums of ge weighted by wx, dx
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int ti = b.i0 + c;
            if (ti < 0 || ti >= (int)A.W) continue;
            const float* gg = G + 3 * ((size_t)tj * A.W + ti);
            const float ge = __ldg(gg) * E0.x + __ldg(gg + 1) * E0.y + __ldg(gg + 2) * E0.z;
            gr = fmaf(ge, b.wx[c], gr);
            gdx = fmaf(ge, b.dx[c], gdx);
          }
          gdz = gr * b.dz[r];
          g.x = fmaf(gdx, b.wz[r], g.x);
          g.y += gdz;
          gscale = fmaf(gr, b.wz[r], gscale);
        }
        g.x *= sc * b.sx;
        g.y *= sc * b.sz;
        gpos[k] = g;
        if (k < nseg) {
          const float4 vn = A.pa[(size_t)k * A.n + p];
          dir = f3(vn) - f3(v);
          v = vn;
        }
        prev = x;
      }
      sgE = sc * gscale;
      lc[6] = gscale;
      float3 g = make_float3(0.f, 0.f, 0.f);
      for (uint32_t k = nseg; k >= 1; --k) {
        g.x += gpos[k].x;
        g.z += gpos[k].y;
        const float4 vk = A.pa[(size_t)(k - 1) * A.n + p];
        int slot;
        const float3 nu = photon_normal(sv, vk, slot);
        const float3 d = k == 1 ? e.d0 : f3(vk) - f3(A.pa[(size_t)(k - 2) * A.n + p]);
        const float r = dot(d, g) / dot(nu, d);
        if (slot >= 0) {
          float* a = s_acc + 7 * A.n_lights + 3 * slot;
          atomicAdd(a + 0, nu.x * r);
          atomicAdd(a + 1, nu.y * r);
          atomicAdd(a + 2, nu.z * r);
        }
        g = g - r * nu;
      }
      // light: g is now the gradient with respect to o; d0 receives tau_1 g
      lc[0] = g.x;
      lc[1] = g.y;
      lc[2] = g.z;
      if (e.rect) {
        const float3 gd = tau1 * g;
        const float3 gn = e.beta * cross(e.t, g) + e.ell.y * cross(e.t, gd) + e.ell.z * gd;
        lc[3] = gn.x;
        lc[4] = gn.y;
        lc[5] = gn.z;
      }
    }
    if (score) score[p] = fabsf(sgE);
  }
  // light entries: summed over the warp per light, one shared atomic per entry
  const int lane = threadIdx.x & 31;
  for (uint32_t ll = 0; ll < A.n_lights; ++ll) {
    const bool mine = my_l == (int)ll;
    if (!__any_sync(0xffffffffu, mine)) continue;
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      float v = mine ? lc[c] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && v != 0.f) atomicAdd(&s_acc[7 * ll + c], v);
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < A.n_theta; j += blockDim.x)
    if (s_acc[j] != 0.f) atomicAdd(dtheta + j, s_acc[j]);
}

// Sort keys of the listed paths: high word = complemented score bits (score
// descending); unlisted slots (and ids out of range) sort last.  The radix sort over the high word is
// stable, and the list is ascending, so equal scores keep ascending ids.
__global__ void k_budget_keys(const uint32_t* list, const uint32_t* count, const float* score, uint32_t n,
                              uint64_t* keys, uint32_t* vals) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t id = i < min(*count, n) ? list[i] : 0xffffffffu;
  if (id < n) {
    const float s = score[id];
    const uint32_t bits = s > 0.f ? __float_as_uint(s) : 0u;     // NaN, zero and negatives rank last
    keys[i] = ((uint64_t)(~bits) << 32) | id;
    vals[i] = id;
  } else {
    keys[i] = ~0ull;
    vals[i] = 0xffffffffu;
  }
}

// Mark the first min(budget, count) sorted paths (bit 30, as in the info word).
__global__ void k_budget_mark(const uint32_t* vals, const uint32_t* count, uint32_t budget, uint32_t n,
                              uint32_t* flags) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < budget && i < min(*count, n) && vals[i] < n) flags[vals[i]] = PV_INFO_REPLACE;
}

int model_args(const pv_scene* s, const pv_paths* p, const float* theta, uint32_t width, uint32_t height,
               const float* rect, ModelArgs& A) {
  if (!theta || !rect || width == 0 || height == 0 || width > (1u << 20) || height > (1u << 20)) return PV_ERR_ARG;
  if (!(rect[2] > rect[0]) || !(rect[3] > rect[1])) return PV_ERR_ARG;
  std::memset(&A, 0, sizeof A);
  A.n = p->n;
  A.n_lights = s->n_lights;
  A.n_theta = 7 * s->n_lights + 3 * s->n_dyn;
  A.info = p->info;
  A.origin = p->origin;
  A.pa = reinterpret_cast<const float4*>(p->pa);
  A.pb = reinterpret_cast<const float4*>(p->pb);
  A.theta = theta;
  A.W = width;
  A.H = height;
  A.x0 = rect[0];
  A.z0 = rect[1];
  A.x1 = rect[2];
  A.z1 = rect[3];
  for (uint32_t sl = 0; sl < s->n_dyn; ++sl)
    for (int k = 0; k < 3; ++k) A.cur_t[sl][k] = s->h_xf_new[12 * sl + 4 * k + 3];
  return PV_OK;
}

}  // namespace

extern "C" int pv_theta_size(const pv_scene* s) {
  if (!s) return PV_ERR_ARG;
  return (int)(7 * s->n_lights + 3 * s->n_dyn);
}

extern "C" int pv_theta_current(const pv_scene* s, float* h_theta) {
  if (!s || !h_theta) return PV_ERR_ARG;
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    for (int k = 0; k < 3; ++k) {
      h_theta[7 * l + k] = s->lights_new[l].pos[k];
      h_theta[7 * l + 3 + k] = s->lights_new[l].normal[k];
    }
    h_theta[7 * l + 6] = 1.0f;
  }
  for (uint32_t sl = 0; sl < s->n_dyn; ++sl)
    for (int k = 0; k < 3; ++k) h_theta[7 * s->n_lights + 3 * sl + k] = s->h_xf_new[12 * sl + 4 * k + 3];
  return PV_OK;
}

extern "C" int pv_model_deposit(pv_scene* s, const pv_paths* paths, const float* d_theta, float* d_atlas,
                                uint32_t width, uint32_t height, const float* rect, void* stream) {
  int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!d_atlas) return PV_ERR_ARG;
  ModelArgs A;
  if ((rc = model_args(s, paths, d_theta, width, height, rect, A)) != PV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (paths->n)
    k_model_deposit<<<(paths->n + 255) / 256, 256, 0, st>>>(pvh::view(s), pvh::frame_lights(s), A, d_atlas);
  return pvh::cuda_status(cudaGetLastError());
}

extern "C" int pv_adjoint_deposit(pv_scene* s, const pv_paths* paths, const float* d_theta, const float* d_grad_atlas,
                                  uint32_t width, uint32_t height, const float* rect, float* d_dtheta, float* d_score,
                                  void* stream) {
  int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!d_grad_atlas || !d_dtheta) return PV_ERR_ARG;
  ModelArgs A;
  if ((rc = model_args(s, paths, d_theta, width, height, rect, A)) != PV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (paths->n)
    k_adjoint<<<(paths->n + 127) / 128, 128, 0, st>>>(pvh::view(s), pvh::frame_lights(s), A, d_grad_atlas, d_dtheta,
                                                      d_score);
  return pvh::cuda_status(cudaGetLastError());
}

extern "C" int pv_budget_list(pv_scene* s, const uint32_t* d_list, const uint32_t* d_count, const float* d_score,
                              uint32_t budget, uint32_t* d_out, uint32_t* d_out_count, void* stream) {
  if (!s || !d_list || !d_count || !d_score || !d_out || !d_out_count) return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  const uint32_t n = s->n_paths_total;
  if (n == 0) return pvh::cuda_status(cudaMemsetAsync(d_out_count, 0, sizeof(uint32_t), st));
  uint64_t *k0 = s->b_keys[0], *k1 = s->b_keys[1];
  uint32_t *v0 = s->b_vals[0], *v1 = s->b_vals[1];
  k_budget_keys<<<(n + 255) / 256, 256, 0, st>>>(d_list, d_count, d_score, n, k0, v0);
  pvh::radix_sort(k0, v0, k1, v1, n, s->b_hist, 32, 64, st);
  PV_CHECK(cudaMemsetAsync(s->ws_mask, 0, (size_t)n * sizeof(uint32_t), st));
  const uint32_t m = budget < n ? budget : n;
  if (m) k_budget_mark<<<(m + 255) / 256, 256, 0, st>>>(v0, d_count, m, n, s->ws_mask);
  pvh::launch_compact(s, s->ws_mask, n, d_out, d_out_count, nullptr, st);
  return pvh::cuda_status(cudaGetLastError());
}
