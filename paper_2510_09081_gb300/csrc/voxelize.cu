// A1 / A5: the two voxelization passes of the voxelize-(cull-)scan-voxelize
// list build (Sec. 3.1, 3.3).
//
// Both passes enumerate the same candidate voxels per segment -- the
// slab-by-slab traversal of Alg. 1 along the major axis a0 of d = v1 - v0, each
// slab visiting a 2D box of minor-axis voxels around the segment -- and keep a
// voxel iff the segment lies within the list radius of the voxel's closed box.
// The minor half-extent of a slab uses the exact half-width of the tube's
// cross-section in a major-axis plane, rl * sqrt(1 + (d_ai / d_a0)^2), which is
// never below Eq. 1's projected radius. Every slab's box is indexed with the
// same width bound (the slab's extent along a minor axis is at most
// |d_ai / d_a0| + 2 * half-extent), so candidate q of a segment decodes in O(1).
//
// Work layout: each lane loads one segment (coalesced) and sets up its walk;
// the warp then takes its 32 segments one at a time and splits the current
// segment's candidates over the lanes, so segments of different lengths do not
// leave lanes idle. The fp32 filter decides almost every candidate; pairs it
// cannot decide go to a queue that a separate kernel decides exactly (keeping
// the 128-bit integer path out of the hot kernels' registers).
//
// Pass 1 adds (occupancy code << 16) | 1 to the voxel's packed word with one
// 32-bit atomic (Sec. 3.1); pass 2 appends the segment id to the lists of
// voxels that received a list (Sec. 3.3), after skipping segments whose box
// touches no listed brick.
#include "launch.h"

namespace vrt {

constexpr float kWalkEps = 1e-3f;
constexpr unsigned FULLW = 0xffffffffu;

struct Walk {
  float3 a, b;
  float am, a1, a2, s1, s2, rho1, rho2, lo_m, hi_m;
  int m, c0, W1, W2;
  uint32_t n;  // candidates: slabs * W1 * W2
};

__device__ __forceinline__ void walk_setup(float3 a, float3 b, const GridDev& g, Walk& w) {
  const float rl = g.rl;
  const int n = g.n;
  const float3 d = b - a;
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  const int m = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  const int k1 = m == 0 ? 1 : 0, k2 = m == 2 ? 1 : 2;
  w.a = a;
  w.b = b;
  w.m = m;
  w.am = cmp3(a, m);
  const float dm = cmp3(b, m) - w.am;
  w.s1 = dm != 0.0f ? cmp3(d, k1) / dm : 0.0f;
  w.s2 = dm != 0.0f ? cmp3(d, k2) / dm : 0.0f;
  w.rho1 = rl * sqrtf(fmaf(w.s1, w.s1, 1.0f)) + kWalkEps;
  w.rho2 = rl * sqrtf(fmaf(w.s2, w.s2, 1.0f)) + kWalkEps;
  w.lo_m = fminf(w.am, w.am + dm) - rl;
  w.hi_m = fmaxf(w.am, w.am + dm) + rl;
  w.a1 = cmp3(a, k1);
  w.a2 = cmp3(a, k2);
  w.c0 = max(0, (int)floorf(w.lo_m - kWalkEps));
  const int c1 = min(n - 1, (int)floorf(w.hi_m + kWalkEps));
  // a range of length L touches at most floor(L) + 2 unit cells
  w.W1 = (int)floorf(fabsf(w.s1) + 2.0f * w.rho1) + 2;
  w.W2 = (int)floorf(fabsf(w.s2) + 2.0f * w.rho2) + 2;
  w.n = c1 >= w.c0 ? (uint32_t)(c1 - w.c0 + 1) * (uint32_t)(w.W1 * w.W2) : 0u;
}

__device__ __forceinline__ Walk shfl_walk(const Walk& w, int src) {
  Walk r;
  r.a = make_float3(__shfl_sync(FULLW, w.a.x, src), __shfl_sync(FULLW, w.a.y, src),
                    __shfl_sync(FULLW, w.a.z, src));
  r.b = make_float3(__shfl_sync(FULLW, w.b.x, src), __shfl_sync(FULLW, w.b.y, src),
                    __shfl_sync(FULLW, w.b.z, src));
  r.am = __shfl_sync(FULLW, w.am, src);
  r.a1 = __shfl_sync(FULLW, w.a1, src);
  r.a2 = __shfl_sync(FULLW, w.a2, src);
  r.s1 = __shfl_sync(FULLW, w.s1, src);
  r.s2 = __shfl_sync(FULLW, w.s2, src);
  r.rho1 = __shfl_sync(FULLW, w.rho1, src);
  r.rho2 = __shfl_sync(FULLW, w.rho2, src);
  r.lo_m = __shfl_sync(FULLW, w.lo_m, src);
  r.hi_m = __shfl_sync(FULLW, w.hi_m, src);
  r.m = __shfl_sync(FULLW, w.m, src);
  r.c0 = __shfl_sync(FULLW, w.c0, src);
  r.W1 = __shfl_sync(FULLW, w.W1, src);
  r.W2 = __shfl_sync(FULLW, w.W2, src);
  r.n = __shfl_sync(FULLW, w.n, src);
  return r;
}

// Candidate q of walk w: its voxel, or false when q falls outside its slab's box.
__device__ __forceinline__ bool walk_decode(const Walk& w, int n, uint32_t q, int& x, int& y,
                                            int& z) {
  const uint32_t w12 = (uint32_t)(w.W1 * w.W2);
  const uint32_t slab = q / w12;
  const uint32_t rem = q - slab * w12;
  const int dj = (int)(rem / (uint32_t)w.W2);
  const int dl = (int)rem - dj * w.W2;
  const int c = w.c0 + (int)slab;
  const float x0 = fmaxf((float)c, w.lo_m), x1 = fminf((float)(c + 1), w.hi_m);
  const float p1a = fmaf(x0 - w.am, w.s1, w.a1), p1b = fmaf(x1 - w.am, w.s1, w.a1);
  const float p2a = fmaf(x0 - w.am, w.s2, w.a2), p2b = fmaf(x1 - w.am, w.s2, w.a2);
  const int j0 = max(0, (int)floorf(fminf(p1a, p1b) - w.rho1));
  const int j1 = min(n - 1, (int)floorf(fmaxf(p1a, p1b) + w.rho1));
  const int l0 = max(0, (int)floorf(fminf(p2a, p2b) - w.rho2));
  const int l1 = min(n - 1, (int)floorf(fmaxf(p2a, p2b) + w.rho2));
  const int j = j0 + dj, l = l0 + dl;
  if (j > j1 || l > l1) return false;
  const int m = w.m;
  x = m == 0 ? c : j;
  y = m == 1 ? c : (m == 0 ? j : l);
  z = m == 2 ? c : l;
  return true;
}

__device__ __forceinline__ void queue_exact(const GridDev& g, uint32_t seg, int x, int y, int z) {
  const uint32_t q = atomicAdd(&g.st->xq_cnt, 1u);
  if (q < g.xq_cap) g.xq[q] = make_uint2(seg, pack_voxel(x, y, z));
  else set_err(g.st, kErrOverflow);
}

__device__ __forceinline__ void flush_counters(DevStatus* st, unsigned long long F,
                                               unsigned long long q, unsigned long long ex) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F += __shfl_down_sync(FULLW, F, o);
    q += __shfl_down_sync(FULLW, q, o);
    ex += __shfl_down_sync(FULLW, ex, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (F) atomicAdd(&st->F, F);
    if (q) atomicAdd(&st->sum_q, q);
    if (ex) atomicAdd(&st->exact_decisions, ex);
  }
}

__device__ __forceinline__ void add_fragment(const GridDev& g, float3 a, float3 b, float3 n0,
                                             float3 n1, bool en0, bool en1, int x, int y, int z,
                                             unsigned long long& F, unsigned long long& sq) {
  const float3 o = make_float3((float)x, (float)y, (float)z);
  const float occ = capsule_occupancy(make_float3(0.5f, 0.5f, 0.5f), a - o, b - o, n0, n1, en0,
                                      en1, g.r_clamp, g.corr);
  const uint32_t q = (uint32_t)floorf(fmaf(g.occ_scale, occ, 0.5f));
  atomicAdd(&g.word[brick_index(x, y, z, g.log2nb)], (q << 16) | 1u);
  F += 1;
  sq += q;
}

__global__ void __launch_bounds__(256) k_pass1(const float4* __restrict__ pos,
                                               const float4* __restrict__ nrm, long long V,
                                               GridDev g) {
  const int lane = threadIdx.x & 31;
  const long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
  const long long i = base + lane;
  Walk w;
  w.n = 0;
  float3 n0 = make_float3(0.f, 0.f, 0.f), n1 = n0;
  uint32_t en = 0;
  if (i + 1 < V) {
    const float4 p0 = pos[i];
    const uint32_t f0 = __float_as_uint(p0.w);
    if (!(f0 & kLast)) {
      const float4 p1 = pos[i + 1];
      walk_setup(f3(p0), f3(p1), g, w);
      n0 = f3(nrm[i]);
      n1 = f3(nrm[i + 1]);
      en = ((f0 & kClipOn) ? 1u : 0u) | ((__float_as_uint(p1.w) & kClipOn) ? 2u : 0u);
    }
  }
  unsigned long long F = 0, sq = 0, ex = 0;
  for (int j = 0; j < 32; ++j) {
    if (__shfl_sync(FULLW, w.n, j) == 0) continue;
    const Walk wj = shfl_walk(w, j);
    const float3 n0j = make_float3(__shfl_sync(FULLW, n0.x, j), __shfl_sync(FULLW, n0.y, j),
                                   __shfl_sync(FULLW, n0.z, j));
    const float3 n1j = make_float3(__shfl_sync(FULLW, n1.x, j), __shfl_sync(FULLW, n1.y, j),
                                   __shfl_sync(FULLW, n1.z, j));
    const uint32_t enj = __shfl_sync(FULLW, en, j);
    for (uint32_t q = lane; q < wj.n; q += 32) {
      int x, y, z;
      if (!walk_decode(wj, g.n, q, x, y, z)) continue;
      const int dec = g.force_exact ? -1 : seg_filter_at(wj.a, wj.b, x, y, z, g.rl);
      if (dec == 0) continue;
      if (dec < 0) {
        queue_exact(g, (uint32_t)(base + j), x, y, z);
        ++ex;
        continue;
      }
      add_fragment(g, wj.a, wj.b, n0j, n1j, enj & 1u, enj & 2u, x, y, z, F, sq);
    }
  }
  flush_counters(g.st, F, sq, ex);
}

// Exact decisions of pass 1's undecided pairs.
__global__ void __launch_bounds__(256) k_exact1(const float4* __restrict__ pos,
                                                const float4* __restrict__ nrm, GridDev g) {
  const uint32_t cnt = min(g.st->xq_cnt, g.xq_cap);
  unsigned long long F = 0, sq = 0;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const uint2 it = g.xq[e];
    int x, y, z;
    unpack_voxel(it.y, x, y, z);
    const float4 p0 = pos[it.x], p1 = pos[it.x + 1];
    if (!seg_exact_at(f3(p0), f3(p1), x, y, z, g.RL)) continue;
    add_fragment(g, f3(p0), f3(p1), f3(nrm[it.x]), f3(nrm[it.x + 1]),
                 __float_as_uint(p0.w) & kClipOn, __float_as_uint(p1.w) & kClipOn, x, y, z, F, sq);
  }
  unsigned long long z0 = 0;
  flush_counters(g.st, F, sq, z0);
}

__device__ __forceinline__ bool bit_set(const uint32_t* bits, uint32_t i) {
  return (bits[i >> 5] >> (i & 31)) & 1u;
}

// Does the box [lo, hi] (voxel coords, clamped) touch a brick whose bit is set?
__device__ __forceinline__ bool any_brick(const uint32_t* bits, int log2nb, int x0, int y0, int z0,
                                          int x1, int y1, int z1) {
  for (int bz = z0 >> 2; bz <= (z1 >> 2); ++bz)
    for (int by = y0 >> 2; by <= (y1 >> 2); ++by)
      for (int bx = x0 >> 2; bx <= (x1 >> 2); ++bx) {
        const uint32_t b = ((uint32_t)bz << (2 * log2nb)) | ((uint32_t)by << log2nb) | (uint32_t)bx;
        if (bit_set(bits, b)) return true;
      }
  return false;
}

__device__ __forceinline__ void list_append(const GridDev& g, uint32_t idx, uint32_t seg,
                                            unsigned long long& listed) {
  const uint32_t slot = atomicAdd(&g.cur[idx], 1u);
  if (slot < g.list_cap) {
    g.lists[slot] = seg;
    ++listed;
  } else {
    set_err(g.st, kErrOverflow);
  }
}

__device__ __forceinline__ void flush_listed(DevStatus* st, unsigned long long listed,
                                             unsigned long long ex) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    listed += __shfl_down_sync(FULLW, listed, o);
    ex += __shfl_down_sync(FULLW, ex, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (listed) atomicAdd(&st->listed, listed);
    if (ex) atomicAdd(&st->exact_decisions, ex);
  }
}

// mode 0: every occupied voxel has a list; 1: voxels marked by the cull;
// 2: repair -- only voxels whose `need` bit is set (bricks from `needb`).
__global__ void __launch_bounds__(256) k_pass2(const float4* __restrict__ pos, long long V, GridDev g,
                                               int mode, const uint32_t* __restrict__ need,
                                               const uint32_t* __restrict__ needb,
                                               const uint32_t* __restrict__ pending) {
  if (mode == 2 && *pending == 0) return;
  const int lane = threadIdx.x & 31;
  const uint32_t* sel = mode == 2 ? need : g.vis;
  const uint32_t* bb = mode == 1 ? g.visb : needb;
  const long long stride = (long long)gridDim.x * (blockDim.x >> 5) * 32;
  unsigned long long ex = 0, listed = 0;
  for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
       base + 1 < V; base += stride) {
    const long long i = base + lane;
    Walk w;
    w.n = 0;
    if (i + 1 < V) {
      const float4 p0 = pos[i];
      if (!(__float_as_uint(p0.w) & kLast)) {
        const float3 a = f3(p0), b = f3(pos[i + 1]);
        bool keep = true;
        if (mode != 0) {
          const int n = g.n;
          const int x0 = max(0, (int)floorf(fminf(a.x, b.x) - g.rl - kWalkEps));
          const int y0 = max(0, (int)floorf(fminf(a.y, b.y) - g.rl - kWalkEps));
          const int z0 = max(0, (int)floorf(fminf(a.z, b.z) - g.rl - kWalkEps));
          const int x1 = min(n - 1, (int)floorf(fmaxf(a.x, b.x) + g.rl + kWalkEps));
          const int y1 = min(n - 1, (int)floorf(fmaxf(a.y, b.y) + g.rl + kWalkEps));
          const int z1 = min(n - 1, (int)floorf(fmaxf(a.z, b.z) + g.rl + kWalkEps));
          keep = x0 <= x1 && y0 <= y1 && z0 <= z1 && any_brick(bb, g.log2nb, x0, y0, z0, x1, y1, z1);
        }
        if (keep) walk_setup(a, b, g, w);
      }
    }
    for (int j = 0; j < 32; ++j) {
      if (__shfl_sync(FULLW, w.n, j) == 0) continue;
      const Walk wj = shfl_walk(w, j);
      for (uint32_t q = lane; q < wj.n; q += 32) {
        int x, y, z;
        if (!walk_decode(wj, g.n, q, x, y, z)) continue;
        const uint32_t idx = brick_index(x, y, z, g.log2nb);
        if (!bit_set(sel, idx)) continue;
        const int dec = g.force_exact ? -1 : seg_filter_at(wj.a, wj.b, x, y, z, g.rl);
        if (dec == 0) continue;
        if (dec < 0) {
          queue_exact(g, (uint32_t)(base + j), x, y, z);
          ++ex;
          continue;
        }
        list_append(g, idx, (uint32_t)(base + j), listed);
      }
    }
  }
  flush_listed(g.st, listed, ex);
}

// Exact decisions of pass 2's undecided pairs (already restricted to voxels
// that get lists).
__global__ void __launch_bounds__(256) k_exact2(const float4* __restrict__ pos, GridDev g) {
  const uint32_t cnt = min(g.st->xq_cnt, g.xq_cap);
  unsigned long long listed = 0, z0 = 0;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const uint2 it = g.xq[e];
    int x, y, z;
    unpack_voxel(it.y, x, y, z);
    if (!seg_exact_at(f3(pos[it.x]), f3(pos[it.x + 1]), x, y, z, g.RL)) continue;
    list_append(g, brick_index(x, y, z, g.log2nb), it.x, listed);
  }
  flush_listed(g.st, listed, z0);
}

int launch_pass1(const float4* pos, const float4* nrm, long long V, const GridDev& g,
                 cudaStream_t s) {
  if (V < 2) return 0;
  const int T = 256;
  k_pass1<<<(unsigned)((V - 1 + T - 1) / T), T, 0, s>>>(pos, nrm, V, g);
  k_exact1<<<152 * 4, T, 0, s>>>(pos, nrm, g);
  return 2;
}

int launch_pass2(const float4* pos, long long V, const GridDev& g, int mode, const uint32_t* need,
                 const uint32_t* needb, const uint32_t* pending, cudaStream_t s) {
  if (V < 2) return 0;
  const int T = 256;
  long long blocks = (V - 1 + T - 1) / T;
  if (mode == 2 && blocks > 152 * 8) blocks = 152 * 8;  // repair: grid-stride, cheap when idle
  k_pass2<<<(unsigned)blocks, T, 0, s>>>(pos, V, g, mode, need, needb, pending);
  k_exact2<<<152 * 4, T, 0, s>>>(pos, g);
  return 2;
}

}  // namespace vrt
