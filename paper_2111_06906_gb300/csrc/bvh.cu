// Morton-code LBVH construction, refit and per-frame rebuild.
//
// Build: 63-bit Morton keys of triangle centroids (21 bits per axis), a
// stable LSD radix sort (8-bit digits, per-warp stable ranks), the binary
// radix tree of Karras ("Maximizing parallelism in the construction of BVHs,
// octrees and k-d trees", HPG 2012) with index tie-break for equal keys, and
// a bottom-up box pass where the second child to arrive at a node builds the
// union.  The dynamic objects share one tree keyed by (slot, 57-bit Morton of
// the object-local centroid): slots occupy the top key bits, so every
// object's triangles form one subtree whose root is recorded per slot.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pv_scene.h"

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

// keys for the static triangles: centroid Morton code over the scene frame
__global__ void k_morton_static(const float* verts, uint32_t n, Frame6 f, uint64_t* keys, uint32_t* vals) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* v = verts + 9 * (size_t)i;
  const float3 c = make_float3((v[0] + v[3] + v[6]) * (1.f / 3.f), (v[1] + v[4] + v[7]) * (1.f / 3.f),
                               (v[2] + v[5] + v[8]) * (1.f / 3.f));
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
// and children; parent links for the bottom-up pass; per-object roots.
__global__ void k_karras(const uint64_t* keys, int n, Node* nodes, uint32_t* node_parent, uint32_t* leaf_parent,
                         const uint8_t* tri_slot, DynObj* objs) {
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
  const int left = first == gamma ? ~gamma : gamma;
  const int right = last == gamma + 1 ? ~(gamma + 1) : gamma + 1;
  nodes[i].d = make_int4(left, right, first, last);
  if (left < 0) leaf_parent[gamma] = ((uint32_t)i << 1); else node_parent[gamma] = ((uint32_t)i << 1);
  if (right < 0) leaf_parent[gamma + 1] = ((uint32_t)i << 1) | 1u; else node_parent[gamma + 1] = ((uint32_t)i << 1) | 1u;
  if (tri_slot) {
    const uint32_t sl = tri_slot[first];
    if (objs[sl].tri_begin == (uint32_t)first && objs[sl].tri_begin + objs[sl].tri_count - 1 == (uint32_t)last)
      objs[sl].root = i;
  }
}

__global__ void k_gather_static(const float* verts, const uint32_t* order, const uint32_t* prim_of, uint32_t n, Tri* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t src = order[i];
  const float* v = verts + 9 * (size_t)src;
  Tri T;
  T.v0 = make_float4(v[0], v[1], v[2], __int_as_float((int)prim_of[src]));
  T.e1 = make_float4(v[3] - v[0], v[4] - v[1], v[5] - v[2], 0.f);
  T.e2 = make_float4(v[6] - v[0], v[7] - v[1], v[8] - v[2], 0.f);
  out[i] = T;
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

// Bottom-up boxes: leaves from triangles (padded by a relative 2^-22 so the
// FP32 slab test never rejects a box that holds a hit), then each internal
// node's box is completed by the second child to arrive.
__global__ void k_fit(Node* nodes, const uint32_t* node_parent, const uint32_t* leaf_parent, uint32_t* flags,
                      const Tri* tris, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || n < 2) return;
  const Tri T = tris[i];
  const float3 v0 = f3(T.v0), v1 = v0 + f3(T.e1), v2 = v0 + f3(T.e2);
  float3 lo = make_float3(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
  float3 hi = make_float3(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
  const float pad = 2.384185791015625e-07f * fmaxf(maxabs3(lo), maxabs3(hi)) + 1e-30f;
  lo = lo - make_float3(pad, pad, pad);
  hi = hi + make_float3(pad, pad, pad);
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

// ------------------------------------------------------------------ per-frame update
struct XformParams {
  float xf[kMaxDyn][12];
  uint64_t moved;
  uint32_t n_dyn;
};

// One block per dynamic slot: keep the previous pose (transform and tight
// box), and for a moved object transform its object-local corners to the new
// pose and reduce the new tight box.
__global__ void __launch_bounds__(256) k_update_objects(XformParams P, const float* local, const uint32_t* prim,
                                                          Tri* tris, DynObj* objs, float* xf_old, float* xf_new) {
  const uint32_t s = blockIdx.x;
  __shared__ float red[6][256];
  __shared__ float m[12];
  DynObj* o = objs + s;
  if (threadIdx.x < 12) {
    xf_old[12 * s + threadIdx.x] = xf_new[12 * s + threadIdx.x];
    m[threadIdx.x] = P.xf[s][threadIdx.x];
  }
  if (threadIdx.x < 6) o->box_old[threadIdx.x] = o->box_new[threadIdx.x];
  __syncthreads();
  if (threadIdx.x < 12) xf_new[12 * s + threadIdx.x] = m[threadIdx.x];
  if (!((P.moved >> s) & 1ull)) return;
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  const uint32_t b = o->tri_begin, e = b + o->tri_count;
  for (uint32_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const float* v = local + 9 * (size_t)i;
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
    T.v0 = make_float4(w[0], w[1], w[2], __int_as_float((int)prim[i]));
    T.e1 = make_float4(w[3] - w[0], w[4] - w[1], w[5] - w[2], 0.f);
    T.e2 = make_float4(w[6] - w[0], w[7] - w[1], w[8] - w[2], 0.f);
    tris[i] = T;
  }
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

}  // namespace pvk

using namespace pvk;

namespace pvh {

static void radix_sort(uint64_t*& k0, uint32_t*& v0, uint64_t*& k1, uint32_t*& v1, uint32_t n, uint32_t* hist,
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

static inline uint32_t blocks(uint32_t n, uint32_t t) { return (n + t - 1) / t; }

int build_static_bvh(pv_scene* s, const float* h_verts, const std::vector<uint32_t>& static_prims, cudaStream_t st) {
  const uint32_t n = (uint32_t)static_prims.size();
  s->n_static = n;
  if (n == 0) {
    s->s_root = INT32_MIN;
    return PV_OK;
  }
  std::vector<float> sv(9 * (size_t)n);
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = 0; i < n; ++i) {
    const float* v = h_verts + 9 * (size_t)static_prims[i];
    std::memcpy(&sv[9 * (size_t)i], v, 9 * sizeof(float));
    for (int k = 0; k < 3; ++k) {
      const float c = (v[k] + v[3 + k] + v[6 + k]) * (1.f / 3.f);
      lo[k] = std::min(lo[k], c);
      hi[k] = std::max(hi[k], c);
    }
  }
  Frame6 f;
  for (int k = 0; k < 3; ++k) {
    f.lo[k] = lo[k];
    f.ext[k] = hi[k] - lo[k];
  }
  float* d_v = nullptr;
  uint32_t* d_prim = nullptr;
  uint64_t *k0 = nullptr, *k1 = nullptr;
  uint32_t *v0 = nullptr, *v1 = nullptr, *hist = nullptr, *np = nullptr, *lp = nullptr, *flags = nullptr;
  const uint32_t n_tiles = blocks(n, kRsTile);
  int rc = PV_OK;
  auto fail = [&](cudaError_t e) { if (e != cudaSuccess && rc == PV_OK) rc = e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA; };
  fail(cudaMalloc(&d_v, sv.size() * sizeof(float)));
  fail(cudaMalloc(&d_prim, n * sizeof(uint32_t)));
  fail(cudaMalloc(&k0, n * sizeof(uint64_t)));
  fail(cudaMalloc(&k1, n * sizeof(uint64_t)));
  fail(cudaMalloc(&v0, n * sizeof(uint32_t)));
  fail(cudaMalloc(&v1, n * sizeof(uint32_t)));
  fail(cudaMalloc(&hist, 256 * (size_t)n_tiles * sizeof(uint32_t)));
  fail(cudaMalloc(&np, n * sizeof(uint32_t)));
  fail(cudaMalloc(&lp, n * sizeof(uint32_t)));
  fail(cudaMalloc(&flags, n * sizeof(uint32_t)));
  fail(cudaMalloc(&s->s_tris, n * sizeof(Tri)));
  fail(cudaMalloc(&s->s_nodes, std::max<uint32_t>(n - 1, 1) * sizeof(Node)));
  if (rc == PV_OK) {
    fail(cudaMemcpyAsync(d_v, sv.data(), sv.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    fail(cudaMemcpyAsync(d_prim, static_prims.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    k_morton_static<<<blocks(n, 256), 256, 0, st>>>(d_v, n, f, k0, v0);
    radix_sort(k0, v0, k1, v1, n, hist, 0, 64, st);
    k_gather_static<<<blocks(n, 256), 256, 0, st>>>(d_v, v0, d_prim, n, s->s_tris);
    if (n >= 2) {
      k_karras<<<blocks(n - 1, 256), 256, 0, st>>>(k0, (int)n, s->s_nodes, np, lp, nullptr, nullptr);
      fail(cudaMemsetAsync(flags, 0, n * sizeof(uint32_t), st));
      k_fit<<<blocks(n, 256), 256, 0, st>>>(s->s_nodes, np, lp, flags, s->s_tris, (int)n);
      s->s_root = 0;
    } else {
      s->s_root = ~0;
    }
    fail(cudaGetLastError());
    fail(cudaStreamSynchronize(st));
  }
  cudaFree(d_v); cudaFree(d_prim); cudaFree(k0); cudaFree(k1); cudaFree(v0); cudaFree(v1);
  cudaFree(hist); cudaFree(np); cudaFree(lp); cudaFree(flags);
  return rc;
}

// Dynamic objects: one tree over all dynamic triangles; keeps the parent
// links and the sort scratch for refits and rebuilds.
int build_dynamic_bvh(pv_scene* s, const float* h_verts, cudaStream_t st) {
  const uint32_t n = s->n_dyn_tris;
  if (n == 0) return PV_OK;
  // group the dynamic triangles by slot (object order), local corners
  std::vector<float> loc(9 * (size_t)n);
  std::vector<uint32_t> prim(n);
  std::vector<uint8_t> slot(n);
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
      o.root = o.tri_count == 1 ? ~(int32_t)o.tri_begin : INT32_MIN;
      for (int k = 0; k < 3; ++k) {
        frames[sl].lo[k] = lo[k];
        frames[sl].ext[k] = hi[k] - lo[k];
      }
    }
  }
  int rc = PV_OK;
  auto fail = [&](cudaError_t e) { if (e != cudaSuccess && rc == PV_OK) rc = e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA; };
  const uint32_t n_tiles = blocks(n, kRsTile);
  Frame6* d_frames = nullptr;
  float* tmp_local = nullptr;
  uint32_t* tmp_prim = nullptr;
  fail(cudaMalloc(&d_frames, s->n_dyn * sizeof(Frame6)));
  fail(cudaMalloc(&tmp_local, 9 * (size_t)n * sizeof(float)));
  fail(cudaMalloc(&tmp_prim, n * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_local, 9 * (size_t)n * sizeof(float)));
  fail(cudaMalloc(&s->d_tri_prim, n * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_tri_slot, n * sizeof(uint8_t)));
  fail(cudaMalloc(&s->d_tris, n * sizeof(Tri)));
  fail(cudaMalloc(&s->d_nodes, std::max<uint32_t>(n - 1, 1) * sizeof(Node)));
  fail(cudaMalloc(&s->d_leaf_parent, n * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_node_parent, n * sizeof(uint32_t)));
  fail(cudaMalloc(&s->d_fit_flags, n * sizeof(uint32_t)));
  fail(cudaMalloc(&s->objs, s->n_dyn * sizeof(DynObj)));
  for (int b = 0; b < 2; ++b) {
    fail(cudaMalloc(&s->r_keys[b], n * sizeof(uint64_t)));
    fail(cudaMalloc(&s->r_vals[b], n * sizeof(uint32_t)));
  }
  fail(cudaMalloc(&s->r_hist, 256 * (size_t)n_tiles * sizeof(uint32_t)));
  fail(cudaMalloc(&s->r_tris, n * sizeof(Tri)));
  fail(cudaMalloc(&s->r_local, 9 * (size_t)n * sizeof(float)));
  fail(cudaMalloc(&s->r_prim, n * sizeof(uint32_t)));
  if (rc != PV_OK) {
    cudaFree(d_frames); cudaFree(tmp_local); cudaFree(tmp_prim);
    return rc;
  }
  fail(cudaMemcpyAsync(d_frames, frames.data(), s->n_dyn * sizeof(Frame6), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(tmp_local, loc.data(), loc.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(tmp_prim, prim.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(s->d_tri_slot, slot.data(), n * sizeof(uint8_t), cudaMemcpyHostToDevice, st));
  fail(cudaMemcpyAsync(s->objs, s->h_objs.data(), s->n_dyn * sizeof(DynObj), cudaMemcpyHostToDevice, st));
  uint64_t *k0 = s->r_keys[0], *k1 = s->r_keys[1];
  uint32_t *v0 = s->r_vals[0], *v1 = s->r_vals[1];
  k_morton_dyn<<<blocks(n, 256), 256, 0, st>>>(tmp_local, nullptr, s->d_tri_slot, n, d_frames, s->objs, 0, k0, v0);
  radix_sort(k0, v0, k1, v1, n, s->r_hist, 0, 64, st);
  k_gather_dyn<<<blocks(n, 256), 256, 0, st>>>(v0, n, tmp_local, tmp_prim, nullptr, s->d_local, s->d_tri_prim, nullptr);
  if (n >= 2) k_karras<<<blocks(n - 1, 256), 256, 0, st>>>(k0, (int)n, s->d_nodes, s->d_node_parent, s->d_leaf_parent, s->d_tri_slot, s->objs);
  fail(cudaGetLastError());
  fail(cudaStreamSynchronize(st));
  cudaFree(d_frames); cudaFree(tmp_local); cudaFree(tmp_prim);
  return rc;
}

// Per frame: previous pose kept, moved objects transformed; the tree is
// refitted, or rebuilt from world-space Morton codes (PV_BUILD_DYN_REBUILD).
void launch_update_dynamic(pv_scene* s, cudaStream_t st) {
  const uint32_t n = s->n_dyn_tris;
  if (n == 0) return;
  XformParams P;
  std::memset(&P, 0, sizeof P);
  for (uint32_t sl = 0; sl < s->n_dyn; ++sl) std::memcpy(P.xf[sl], &s->h_xf_new[12 * sl], 12 * sizeof(float));
  P.moved = s->moved;
  P.n_dyn = s->n_dyn;
  k_update_objects<<<s->n_dyn, 256, 0, st>>>(P, s->d_local, s->d_tri_prim, s->d_tris, s->objs, s->xf_old, s->xf_new);
  if (!s->moved) return;
  if (s->flags & PV_BUILD_DYN_REBUILD) {
    uint64_t *k0 = s->r_keys[0], *k1 = s->r_keys[1];
    uint32_t *v0 = s->r_vals[0], *v1 = s->r_vals[1];
    k_morton_dyn<<<blocks(n, 256), 256, 0, st>>>(nullptr, s->d_tris, s->d_tri_slot, n, nullptr, s->objs, 1, k0, v0);
    radix_sort(k0, v0, k1, v1, n, s->r_hist, 0, 64, st);
    k_gather_dyn<<<blocks(n, 256), 256, 0, st>>>(v0, n, s->d_local, s->d_tri_prim, s->d_tris, s->r_local, s->r_prim, s->r_tris);
    std::swap(s->d_local, s->r_local);
    std::swap(s->d_tri_prim, s->r_prim);
    std::swap(s->d_tris, s->r_tris);
    if (n >= 2) k_karras<<<blocks(n - 1, 256), 256, 0, st>>>(k0, (int)n, s->d_nodes, s->d_node_parent, s->d_leaf_parent, s->d_tri_slot, s->objs);
  }
  if (n >= 2) {
    cudaMemsetAsync(s->d_fit_flags, 0, n * sizeof(uint32_t), st);
    k_fit<<<blocks(n, 256), 256, 0, st>>>(s->d_nodes, s->d_node_parent, s->d_leaf_parent, s->d_fit_flags, s->d_tris, (int)n);
  }
}

}  // namespace pvh
