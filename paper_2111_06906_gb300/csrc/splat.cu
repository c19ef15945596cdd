// Screen-space photon splat: the renderer's "splat/gather" step of Fig. 2.
// The paper only cites its splatting method, so this is a plain radius
// kernel.  k_gbuffer casts one primary ray per pixel through the scene's BVH
// (visible point, normal facing the camera, primitive); k_splat takes one path
// per thread and, for each stored photon x with energy E arriving on the
// visible side of a pixel's point p, adds rho/pi E 2 (1 - s^2) / (pi r^2),
// s = |p - x| / r < 1, over the pixels inside the screen footprint of the
// photon's kernel cube (its eight corners projected: the footprint of every
// point within r of x lies inside their hull).
#include <cmath>

#include "pv_scene.h"

using namespace pvk;

namespace {

struct Cam {
  float3 pos, f, r, u;       // centre, forward, right, up (unit)
  float tx, ty;              // tan of the half field of view, horizontal and vertical
  uint32_t W, H;
  float znear;               // photons whose kernel cube reaches closer are skipped
};

struct GPixel {              // 32 bytes per pixel
  float4 p;                  // visible point, w = primitive id bits (-1: background)
  float4 n;                  // normal facing the camera
};

__global__ void __launch_bounds__(256) k_gbuffer(SceneView sv, Cam c, GPixel* g) {
  const uint32_t px = blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= c.W * c.H) return;
  const uint32_t i = px % c.W, j = px / c.W;
  const float x = (2.0f * ((float)i + 0.5f) / (float)c.W - 1.0f) * c.tx;
  const float y = (1.0f - 2.0f * ((float)j + 0.5f) / (float)c.H) * c.ty;
  const float3 d = normalize(c.f + x * c.r + y * c.u);
  const Ray r = make_ray(c.pos, d, 0.0f);
  Hit h;
  Work wk;
  GPixel o;
  o.p = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
  o.n = make_float4(0.f, 0.f, 0.f, 0.f);
  const int root = *sv.root;
  if (closest_hit(sv, root, r, -1, h, wk)) {
    const Tri T = load_tri(sv.tris, h.tri);
    const float3 p = make_float3(fmaf(h.t, d.x, c.pos.x), fmaf(h.t, d.y, c.pos.y), fmaf(h.t, d.z, c.pos.z));
    float3 nn = normalize(cross(f3(T.e1), f3(T.e2)));
    if (dot(nn, d) > 0.0f) nn = -1.0f * nn;
    o.p = make_float4(p.x, p.y, p.z, T.v0.w);
    o.n = make_float4(nn.x, nn.y, nn.z, 0.f);
  }
  g[px] = o;
}

// Continuous pixel coordinates of q (pixel centres at integers); false behind the near plane.
__device__ __forceinline__ bool project(const Cam& c, float3 q, float& pi, float& pj) {
  const float3 v = q - c.pos;
  const float z = dot(v, c.f);
  if (!(z > c.znear)) return false;
  pi = (dot(v, c.r) / (z * c.tx) + 1.0f) * 0.5f * (float)c.W - 0.5f;
  pj = (1.0f - dot(v, c.u) / (z * c.ty)) * 0.5f * (float)c.H - 0.5f;
  return true;
}

__global__ void __launch_bounds__(256) k_splat(SceneView sv, Cam c, uint32_t n, const uint32_t* info, const float* origin,
                                              const float4* pa, const float4* pb, float radius, const GPixel* g,
                                              float* image) {
  const float r2 = radius * radius;
  const float norm = 2.0f / (3.14159265f * r2) / 3.14159265f;   // kernel normalisation times 1/pi (Lambertian)
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t L = min(info_nseg(info[p]), sv.B);
    float3 prev = make_float3(origin[p], origin[n + p], origin[2 * (size_t)n + p]);
    for (uint32_t k = 0; k < L; ++k) {
      const float4 xv = pa[(size_t)k * n + p];
      const float4 ev = pb[(size_t)k * n + p];
      const float3 x = f3(xv), din = x - prev;
      prev = x;
      float i0 = 3e38f, i1 = -3e38f, j0 = 3e38f, j1 = -3e38f;
      bool front = true;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float3 cor = make_float3(x.x + ((q & 1) ? radius : -radius), x.y + ((q & 2) ? radius : -radius),
                                       x.z + ((q & 4) ? radius : -radius));
        float pi, pj;
        if (!project(c, cor, pi, pj)) front = false;
        i0 = fminf(i0, pi);
        i1 = fmaxf(i1, pi);
        j0 = fminf(j0, pj);
        j1 = fmaxf(j1, pj);
      }
      if (!front) continue;
      // clamp in float before converting (a corner may project far off screen)
      const int ia = (int)fmaxf(floorf(i0) - 1.0f, 0.0f), ib = (int)fminf(ceilf(i1) + 1.0f, (float)c.W - 1.0f);
      const int ja = (int)fmaxf(floorf(j0) - 1.0f, 0.0f), jb = (int)fminf(ceilf(j1) + 1.0f, (float)c.H - 1.0f);
      for (int j = ja; j <= jb; ++j)
        for (int i = ia; i <= ib; ++i) {
          const GPixel gp = g[(size_t)j * c.W + i];
          const int prim = __float_as_int(gp.p.w);
          if (prim < 0) continue;
          const float3 dp = f3(gp.p) - x;
          const float s2 = dot(dp, dp) / r2;
          if (!(s2 < 1.0f) || !(dot(f3(gp.n), din) < 0.0f)) continue;
          const float4 alb = __ldg(sv.prim_alb + prim);
          const float w = norm * (1.0f - s2);
          float* px = image + 3 * ((size_t)j * c.W + i);
          atomicAdd(px + 0, alb.x * ev.x * w);
          atomicAdd(px + 1, alb.y * ev.y * w);
          atomicAdd(px + 2, alb.z * ev.z * w);
        }
    }
  }
}

Cam make_cam(const pv_scene* s, const pv_camera* cam) {
  double pos[3], tg[3], up[3], f[3], r[3], u[3];
  for (int k = 0; k < 3; ++k) {
    pos[k] = cam->pos[k];
    tg[k] = cam->target[k];
    up[k] = cam->up[k];
    f[k] = tg[k] - pos[k];
  }
  auto nrm = [](double* v) {
    const double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) v[k] /= l;
  };
  nrm(f);
  r[0] = f[1] * up[2] - f[2] * up[1];
  r[1] = f[2] * up[0] - f[0] * up[2];
  r[2] = f[0] * up[1] - f[1] * up[0];
  nrm(r);
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  const double ty = std::tan(0.5 * (double)cam->fov_y);
  Cam c;
  c.pos = make_float3((float)pos[0], (float)pos[1], (float)pos[2]);
  c.f = make_float3((float)f[0], (float)f[1], (float)f[2]);
  c.r = make_float3((float)r[0], (float)r[1], (float)r[2]);
  c.u = make_float3((float)u[0], (float)u[1], (float)u[2]);
  c.ty = (float)ty;
  c.tx = (float)(ty * (double)cam->width / (double)cam->height);
  c.W = cam->width;
  c.H = cam->height;
  c.znear = 1e-3f * s->diag;
  return c;
}

bool camera_ok(const pv_camera* c) {
  if (!c || c->width == 0 || c->height == 0 || c->width > 16384 || c->height > 16384) return false;
  if (!(c->fov_y > 0.0f && c->fov_y < 3.1f)) return false;
  const double f[3] = {(double)c->target[0] - c->pos[0], (double)c->target[1] - c->pos[1],
                       (double)c->target[2] - c->pos[2]};
  const double cr[3] = {f[1] * c->up[2] - f[2] * c->up[1], f[2] * c->up[0] - f[0] * c->up[2],
                        f[0] * c->up[1] - f[1] * c->up[0]};
  return f[0] * f[0] + f[1] * f[1] + f[2] * f[2] > 0.0 && cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2] > 0.0;
}

}  // namespace

extern "C" size_t pv_splat_workspace_bytes(uint32_t width, uint32_t height) {
  return (size_t)width * height * sizeof(GPixel);
}

extern "C" int pv_splat(pv_scene* s, const pv_paths* paths, const pv_camera* cam, float radius, float* d_image,
                        void* d_work, size_t work_bytes, void* stream) {
  const int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!camera_ok(cam) || !d_image || !d_work || !(radius > 0.0f)) return PV_ERR_ARG;
  if (work_bytes < pv_splat_workspace_bytes(cam->width, cam->height) || (reinterpret_cast<uintptr_t>(d_work) & 15u))
    return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  const Cam c = make_cam(s, cam);
  const size_t npx = (size_t)cam->width * cam->height;
  PV_CHECK(cudaMemsetAsync(d_image, 0, npx * 3 * sizeof(float), st));
  GPixel* g = static_cast<GPixel*>(d_work);
  const pvk::SceneView sv = pvh::view(s);
  k_gbuffer<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(sv, c, g);
  if (paths->n) {
    const uint32_t blocks = std::min<uint32_t>((paths->n + 255) / 256, 16u * (uint32_t)s->num_sms);
    k_splat<<<blocks, 256, 0, st>>>(sv, c, paths->n, paths->info, paths->origin,
                                   reinterpret_cast<const float4*>(paths->pa), reinterpret_cast<const float4*>(paths->pb),
                                   radius, g, d_image);
  }
  return pvh::cuda_status(cudaGetLastError());
}
