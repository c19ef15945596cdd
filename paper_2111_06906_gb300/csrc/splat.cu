// Screen-space photon splat: the renderer's "splat/gather" step of Fig. 2.
// The paper only cites its splatting method, so this is a plain radius
// kernel, evaluated as a gather.  k_gbuffer casts one primary ray per pixel
// through the scene's BVH (visible point, normal facing the camera,
// primitive).  k_grid_fill hashes every stored photon into a grid of cells
// of edge r (count, scan of the buckets, place), skipping photons whose
// kernel cube reaches the near plane.  k_gather then gives each pixel the
// photons of the 27 cells around its visible point p: every photon x with
// energy E arriving on the visible side and s = |p - x| / r < 1 adds
// rho/pi E 2 (1 - s^2) / (pi r^2).  Each pixel is written once, without
// atomics, and the work per pixel is bounded by the photons near it, not by
// how many pixels a photon's footprint covers.
#include <algorithm>
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

// A photon takes part when every corner of its kernel cube lies beyond the
// near plane (its screen footprint is then bounded).
__device__ __forceinline__ bool in_front(const Cam& c, float3 x, float radius) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float3 cor = make_float3(x.x + ((q & 1) ? radius : -radius), x.y + ((q & 2) ? radius : -radius),
                                   x.z + ((q & 4) ? radius : -radius));
    if (!(dot(cor - c.pos, c.f) > c.znear)) return false;
  }
  return true;
}

// Photon grid: cells of edge ``radius``, hashed into a power-of-two number of
// buckets; a photon within ``radius`` of a point lies in one of the 27 cells
// around the point's cell.
struct Grid {
  float inv_r;                 // 1 / radius
  uint32_t mask;               // buckets - 1
};

__device__ __forceinline__ int3 grid_cell(const Grid& g, float3 x) {
  const float lim = 1.0e9f;
  return make_int3((int)fminf(fmaxf(floorf(x.x * g.inv_r), -lim), lim), (int)fminf(fmaxf(floorf(x.y * g.inv_r), -lim), lim),
                   (int)fminf(fmaxf(floorf(x.z * g.inv_r), -lim), lim));
}

__device__ __forceinline__ uint32_t grid_bucket(const Grid& g, int3 c) {
  return (((uint32_t)c.x * 73856093u) ^ ((uint32_t)c.y * 19349663u) ^ ((uint32_t)c.z * 83492791u)) & g.mask;
}

struct PhotonRec {           // 32 bytes
  float4 x;                  // position, w = path index * 16 + row (int bits)
  float4 e;                  // incident energy
};

// pass 0: count the photons per bucket; pass 1: place them (heads: exclusive
// prefix of the counts on entry, each bucket's end on exit).
template <int kPass>
__global__ void __launch_bounds__(256) k_grid_fill(Cam c, Grid g, float radius, uint32_t n, uint32_t B,
                                                   const uint32_t* info, const float4* pa, const float4* pb,
                                                   uint32_t* heads, PhotonRec* rec) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t L = min(info_nseg(info[p]), B);
    for (uint32_t k = 0; k < L; ++k) {
      const float4 xv = pa[(size_t)k * n + p];
      const float3 x = f3(xv);
      if (!in_front(c, x, radius)) continue;
      const uint32_t b = grid_bucket(g, grid_cell(g, x));
      if (kPass == 0) {
        atomicAdd(heads + b, 1u);
      } else {
        const uint32_t slot = atomicAdd(heads + b, 1u);
        PhotonRec r;
        r.x = make_float4(x.x, x.y, x.z, __int_as_float((int)(p * 16u + k)));
        r.e = pb[(size_t)k * n + p];
        rec[slot] = r;
      }
    }
  }
}

// Exclusive scan of m = tiles * 4096 counters: tile sums, their scan, then
// each tile's own scan plus its offset.
__global__ void __launch_bounds__(1024) k_tile_sums(const uint32_t* v, uint32_t* sums) {
  __shared__ uint32_t w[32];
  const uint4 x = reinterpret_cast<const uint4*>(v)[(size_t)blockIdx.x * 1024 + threadIdx.x];
  uint32_t t = __reduce_add_sync(0xffffffffu, x.x + x.y + x.z + x.w);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    t = __reduce_add_sync(0xffffffffu, w[threadIdx.x]);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_tile_scan(uint32_t* v, const uint32_t* offs) {
  __shared__ uint32_t w[32];
  uint4* p = reinterpret_cast<uint4*>(v) + (size_t)blockIdx.x * 1024 + threadIdx.x;
  const uint4 x = *p;
  const uint32_t own = x.x + x.y + x.z + x.w;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) w[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = w[lane], si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    w[lane] = si - s;
  }
  __syncthreads();
  const uint32_t base = offs[blockIdx.x] + w[wid] + incl - own;
  *p = make_uint4(base, base + x.x, base + x.x + x.y, base + x.x + x.y + x.z);
}

// One pixel per thread: the photons of the 27 cells around its visible point.
__global__ void __launch_bounds__(256) k_gather(SceneView sv, Cam c, Grid g, float radius, uint32_t n,
                                                const float* origin, const float4* pa, const GPixel* gb,
                                                const uint32_t* heads, const PhotonRec* rec, float* image) {
  const uint32_t px = blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= c.W * c.H) return;
  const GPixel gp = gb[px];
  const int prim = __float_as_int(gp.p.w);
  float3 acc = make_float3(0.f, 0.f, 0.f);
  if (prim >= 0) {
    const float3 P = f3(gp.p), nrm = f3(gp.n);
    const float r2 = radius * radius;
    const int3 cp = grid_cell(g, P);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int3 cc = make_int3(cp.x + dx, cp.y + dy, cp.z + dz);
          const uint32_t b = grid_bucket(g, cc);
          const uint32_t beg = b ? heads[b - 1] : 0u, end = heads[b];
          for (uint32_t i = beg; i < end; ++i) {
            const float4 xv = __ldg(&rec[i].x);
            const float3 x = f3(xv);
            const float3 d = P - x;
            const float s2 = dot(d, d) / r2;
            if (!(s2 < 1.0f)) continue;
            const int3 xc = grid_cell(g, x);         // each photon once: only from its own cell
            if (xc.x != cc.x || xc.y != cc.y || xc.z != cc.z) continue;
            const uint32_t id = (uint32_t)__float_as_int(xv.w), p = id >> 4, k = id & 15u;
            const float3 prev = k == 0 ? make_float3(origin[p], origin[n + p], origin[2 * (size_t)n + p])
                                       : f3(__ldg(pa + (size_t)(k - 1) * n + p));
            if (!(dot(nrm, x - prev) < 0.0f)) continue;   // arrives on the visible side
            const float4 e = __ldg(&rec[i].e);
            const float w = 1.0f - s2;
            acc = make_float3(fmaf(e.x, w, acc.x), fmaf(e.y, w, acc.y), fmaf(e.z, w, acc.z));
          }
        }
  }
  const float norm = 2.0f / (3.14159265f * radius * radius) / 3.14159265f;   // kernel normalisation and 1/pi
  float* o = image + 3 * (size_t)px;
  if (prim >= 0) {
    const float4 alb = __ldg(sv.prim_alb + prim);
    o[0] = alb.x * acc.x * norm;
    o[1] = alb.y * acc.y * norm;
    o[2] = alb.z * acc.z * norm;
  } else {
    o[0] = o[1] = o[2] = 0.0f;
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

namespace {

// Workspace layout: G-buffer, bucket heads, tile sums, photon records.
struct SplatLayout {
  size_t gbuf, heads, sums, rec, bytes;
  uint32_t buckets, tiles;
  SplatLayout(uint64_t photons, uint32_t width, uint32_t height) {
    buckets = 4096;                                 // a power of two >= the photons, at least one scan tile
    while (buckets < photons && buckets < (1u << 30)) buckets <<= 1;
    tiles = buckets / 4096;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    gbuf = 0;
    heads = up(gbuf + (size_t)width * height * sizeof(GPixel));
    sums = up(heads + (size_t)buckets * sizeof(uint32_t));
    rec = up(sums + (size_t)(tiles + 1) * sizeof(uint32_t));
    bytes = up(rec + (size_t)photons * sizeof(PhotonRec));
  }
};

}  // namespace

extern "C" size_t pv_splat_workspace_bytes(const pv_scene* s, uint32_t width, uint32_t height) {
  if (!s) return 0;
  return SplatLayout((uint64_t)s->n_paths_total * s->B, width, height).bytes;
}

extern "C" int pv_splat(pv_scene* s, const pv_paths* paths, const pv_camera* cam, float radius, float* d_image,
                        void* d_work, size_t work_bytes, void* stream) {
  const int rc = pvh::check_paths(s, paths);
  if (rc != PV_OK) return rc;
  if (!camera_ok(cam) || !d_image || !d_work || !(radius > 0.0f)) return PV_ERR_ARG;
  if (paths->n > (1u << 27)) return PV_ERR_LIMIT;            // a photon is named by path * 16 + row
  const SplatLayout lay((uint64_t)paths->n * paths->max_bounces, cam->width, cam->height);
  if (work_bytes < lay.bytes || (reinterpret_cast<uintptr_t>(d_work) & 255u)) return PV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  const Cam c = make_cam(s, cam);
  const size_t npx = (size_t)cam->width * cam->height;
  char* w = static_cast<char*>(d_work);
  GPixel* gbuf = reinterpret_cast<GPixel*>(w + lay.gbuf);
  uint32_t* heads = reinterpret_cast<uint32_t*>(w + lay.heads);
  uint32_t* sums = reinterpret_cast<uint32_t*>(w + lay.sums);
  PhotonRec* rec = reinterpret_cast<PhotonRec*>(w + lay.rec);
  const pvk::SceneView sv = pvh::view(s);
  k_gbuffer<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(sv, c, gbuf);
  Grid g;
  g.inv_r = 1.0f / radius;
  g.mask = lay.buckets - 1;
  PV_CHECK(cudaMemsetAsync(heads, 0, (size_t)lay.buckets * sizeof(uint32_t), st));
  const uint32_t n = paths->n;
  const float4* pa = reinterpret_cast<const float4*>(paths->pa);
  const float4* pb = reinterpret_cast<const float4*>(paths->pb);
  if (n) {
    const uint32_t blocks = std::min<uint32_t>((n + 255) / 256, 16u * (uint32_t)s->num_sms);
    k_grid_fill<0><<<blocks, 256, 0, st>>>(c, g, radius, n, s->B, paths->info, pa, pb, heads, rec);
    k_tile_sums<<<lay.tiles, 1024, 0, st>>>(heads, sums);
    pvh::exclusive_scan(sums, lay.tiles, st);
    k_tile_scan<<<lay.tiles, 1024, 0, st>>>(heads, sums);
    k_grid_fill<1><<<blocks, 256, 0, st>>>(c, g, radius, n, s->B, paths->info, pa, pb, heads, rec);
  }
  k_gather<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(sv, c, g, radius, n, paths->origin, pa, gbuf, heads, rec,
                                                          d_image);
  return pvh::cuda_status(cudaGetLastError());
}
