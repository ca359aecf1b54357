// A1 / A5: the two voxelization passes of the voxelize-(cull-)scan-voxelize
// list build (Sec. 3.1, 3.3).
//
// Both passes walk the same candidate voxels per segment -- the slab-by-slab
// traversal of Alg. 1 along the major axis of d = v1 - v0, each slab visiting
// the 2D box of minor-axis voxels around the segment -- and keep a voxel iff
// the segment lies within the list radius of the voxel's closed box (decided
// exactly). The minor half-extent of a slab uses the exact half-width of the
// tube's cross-section in a major-axis plane, rl * sqrt(1 + (d_ai / d_a0)^2),
// which is never below Eq. 1's projected radius.
//
// Pass 1 adds (occupancy code << 16) | 1 to the voxel's packed word with one
// 32-bit atomic (Sec. 3.1); pass 2 appends the segment id to the lists of
// voxels that received a list (Sec. 3.3), after skipping segments whose box
// touches no listed brick.
#include "launch.h"

namespace vrt {

constexpr float kWalkEps = 1e-3f;

__device__ __forceinline__ void swap_axes(int m, int& k1, int& k2) {
  k1 = m == 0 ? 1 : 0;
  k2 = m == 2 ? 1 : 2;
}

// Calls visit(x, y, z) for every voxel of [0, n)^3 within rl of segment [a, b].
template <class Visit>
__device__ __forceinline__ void walk_segment(float3 a, float3 b, const GridDev& g,
                                             unsigned long long& n_exact, Visit&& visit) {
  const float rl = g.rl;
  const int n = g.n;
  const float3 d = b - a;
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  const int m = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  int k1, k2;
  swap_axes(m, k1, k2);
  const float am = cmp3(a, m), bm = cmp3(b, m);
  const float dm = bm - am;
  const float s1 = dm != 0.0f ? cmp3(d, k1) / dm : 0.0f;
  const float s2 = dm != 0.0f ? cmp3(d, k2) / dm : 0.0f;
  const float rho1 = rl * sqrtf(fmaf(s1, s1, 1.0f)) + kWalkEps;
  const float rho2 = rl * sqrtf(fmaf(s2, s2, 1.0f)) + kWalkEps;
  const float lo_m = fminf(am, bm) - rl, hi_m = fmaxf(am, bm) + rl;
  const int c0 = max(0, (int)floorf(lo_m - kWalkEps));
  const int c1 = min(n - 1, (int)floorf(hi_m + kWalkEps));
  const float a1 = cmp3(a, k1), a2 = cmp3(a, k2);
  for (int c = c0; c <= c1; ++c) {
    const float x0 = fmaxf((float)c, lo_m), x1 = fminf((float)(c + 1), hi_m);
    const float p1a = fmaf(x0 - am, s1, a1), p1b = fmaf(x1 - am, s1, a1);
    const float p2a = fmaf(x0 - am, s2, a2), p2b = fmaf(x1 - am, s2, a2);
    const int j0 = max(0, (int)floorf(fminf(p1a, p1b) - rho1));
    const int j1 = min(n - 1, (int)floorf(fmaxf(p1a, p1b) + rho1));
    const int l0 = max(0, (int)floorf(fminf(p2a, p2b) - rho2));
    const int l1 = min(n - 1, (int)floorf(fmaxf(p2a, p2b) + rho2));
    for (int j = j0; j <= j1; ++j)
      for (int l = l0; l <= l1; ++l) {
        int v[3];
        v[m] = c;
        v[k1] = j;
        v[k2] = l;
        if (seg_in_voxel(a, b, v[0], v[1], v[2], rl, g.RL, g.force_exact, &n_exact))
          visit(v[0], v[1], v[2]);
      }
  }
}

__device__ __forceinline__ void flush_counters(DevStatus* st, unsigned long long F,
                                               unsigned long long q, unsigned long long ex) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F += __shfl_down_sync(0xffffffffu, F, o);
    q += __shfl_down_sync(0xffffffffu, q, o);
    ex += __shfl_down_sync(0xffffffffu, ex, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (F) atomicAdd(&st->F, F);
    if (q) atomicAdd(&st->sum_q, q);
    if (ex) atomicAdd(&st->exact_decisions, ex);
  }
}

__global__ void __launch_bounds__(256) k_pass1(const float4* __restrict__ pos,
                                               const float4* __restrict__ nrm, long long V,
                                               GridDev g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long F = 0, sq = 0, ex = 0;
  if (i + 1 < V) {
    const float4 p0 = pos[i];
    const uint32_t f0 = __float_as_uint(p0.w);
    if (!(f0 & kLast)) {
      const float4 p1 = pos[i + 1];
      const uint32_t f1 = __float_as_uint(p1.w);
      const float3 a = f3(p0), b = f3(p1);
      const float3 n0 = f3(nrm[i]), n1 = f3(nrm[i + 1]);
      const bool en0 = f0 & kClipOn, en1 = f1 & kClipOn;
      walk_segment(a, b, g, ex, [&](int x, int y, int z) {
        const float3 o = make_float3((float)x, (float)y, (float)z);
        const float occ = capsule_occupancy(make_float3(0.5f, 0.5f, 0.5f), a - o, b - o, n0, n1,
                                            en0, en1, g.r_clamp, g.corr);
        const uint32_t q = (uint32_t)floorf(fmaf(g.occ_scale, occ, 0.5f));
        atomicAdd(&g.word[brick_index(x, y, z, g.log2nb)], (q << 16) | 1u);
        F += 1;
        sq += q;
      });
    }
  }
  flush_counters(g.st, F, sq, ex);
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

__global__ void __launch_bounds__(256) k_pass2(const float4* __restrict__ pos, long long V, GridDev g,
                                               int mode, const uint32_t* __restrict__ need,
                                               const uint32_t* __restrict__ needb,
                                               const uint32_t* __restrict__ pending) {
  if (mode == 2 && *pending == 0) return;
  unsigned long long ex = 0, listed = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < V;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 p0 = pos[i];
    if (__float_as_uint(p0.w) & kLast) continue;
    const float4 p1 = pos[i + 1];
    const float3 a = f3(p0), b = f3(p1);
    if (mode != 0) {
      const uint32_t* bb = mode == 1 ? g.visb : needb;
      const int n = g.n;
      const int x0 = max(0, (int)floorf(fminf(a.x, b.x) - g.rl - kWalkEps));
      const int y0 = max(0, (int)floorf(fminf(a.y, b.y) - g.rl - kWalkEps));
      const int z0 = max(0, (int)floorf(fminf(a.z, b.z) - g.rl - kWalkEps));
      const int x1 = min(n - 1, (int)floorf(fmaxf(a.x, b.x) + g.rl + kWalkEps));
      const int y1 = min(n - 1, (int)floorf(fmaxf(a.y, b.y) + g.rl + kWalkEps));
      const int z1 = min(n - 1, (int)floorf(fmaxf(a.z, b.z) + g.rl + kWalkEps));
      if (x0 > x1 || y0 > y1 || z0 > z1) continue;
      if (!any_brick(bb, g.log2nb, x0, y0, z0, x1, y1, z1)) continue;
    }
    const uint32_t* sel = mode == 2 ? need : g.vis;
    walk_segment(a, b, g, ex, [&](int x, int y, int z) {
      const uint32_t idx = brick_index(x, y, z, g.log2nb);
      if (!bit_set(sel, idx)) return;
      const uint32_t slot = atomicAdd(&g.cur[idx], 1u);
      if (slot < g.list_cap) {
        g.lists[slot] = (uint32_t)i;
        ++listed;
      } else {
        set_err(g.st, kErrOverflow);
      }
    });
  }
  unsigned long long z = 0;
  flush_counters(g.st, z, z, ex);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) listed += __shfl_down_sync(0xffffffffu, listed, o);
  if ((threadIdx.x & 31) == 0 && listed) atomicAdd(&g.st->listed, listed);
}

int launch_pass1(const float4* pos, const float4* nrm, long long V, const GridDev& g,
                  cudaStream_t s) {
  if (V < 2) return 0;
  const int T = 256;
  k_pass1<<<(unsigned)((V - 1 + T - 1) / T), T, 0, s>>>(pos, nrm, V, g);
  return 1;
}

int launch_pass2(const float4* pos, long long V, const GridDev& g, int mode, const uint32_t* need,
                  const uint32_t* needb, const uint32_t* pending, cudaStream_t s) {
  if (V < 2) return 0;
  const int T = 256;
  long long blocks = (V - 1 + T - 1) / T;
  if (mode == 2 && blocks > 152 * 8) blocks = 152 * 8;  // repair: grid-stride, cheap when idle
  k_pass2<<<(unsigned)blocks, T, 0, s>>>(pos, V, g, mode, need, needb, pending);
  return 1;
}

}  // namespace vrt
