// Empty-space skipping for the trace and the cull march: for every 4^3 brick,
// the Chebyshev distance (in bricks, capped at kBrickDistMax) to the nearest
// brick that holds an occupied voxel (count > 0); 0 marks such a brick. A ray
// in a brick at distance k >= 1 can cross the whole cube of bricks within
// k - 1 of it in one step, since none of them holds a voxel with segments.
//
// Built after pass 1 in three separable passes: the L-infinity distance to a
// set factors over the axes, d(b) = min_k max(|k|, d_xy(b + k e_z)), and
// likewise for d_xy from d_x and d_x from the occupancy.
#include "launch.h"

namespace vrt {

// One thread per brick: 0 when any of its 64 voxels has a count, else the cap.
__global__ void __launch_bounds__(256) k_brick_occ(GridDev g, uint8_t* __restrict__ out) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nb = 1u << (3 * g.log2nb);
  if (b >= nb) return;
  const uint4* w = reinterpret_cast<const uint4*>(g.word + ((size_t)b << 6));
  uint32_t any = 0;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const uint4 v = __ldg(&w[q]);
    any |= (v.x | v.y | v.z | v.w) & 0xffffu;
  }
  out[b] = any ? 0 : (uint8_t)kBrickDistMax;
}

// out(b) = min over |i| <= kBrickDistMax (inside the grid) of max(|i|, in(b + i e)),
// along axis `axis` (0 x, 1 y, 2 z).
__global__ void __launch_bounds__(256) k_brick_dist(int log2nb, int axis,
                                                    const uint8_t* __restrict__ in,
                                                    uint8_t* __restrict__ out) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nb = 1u << (3 * log2nb);
  if (b >= nb) return;
  const int side = 1 << log2nb;
  const int shift = axis * log2nb;
  const int c = (int)((b >> shift) & (uint32_t)(side - 1));
  const uint32_t base = b - ((uint32_t)c << shift);
  int d = __ldg(&in[b]);
  for (int i = 1; i < d; ++i) {
    if (c - i >= 0) d = min(d, max(i, (int)__ldg(&in[base + ((uint32_t)(c - i) << shift)])));
    if (c + i < side) d = min(d, max(i, (int)__ldg(&in[base + ((uint32_t)(c + i) << shift)])));
  }
  out[b] = (uint8_t)d;
}

int launch_brick_dist_passes(int log2nb, uint8_t* tmp, uint8_t* dist, cudaStream_t s) {
  const uint32_t nb = 1u << (3 * log2nb);
  const int T = 256;
  const unsigned blocks = (nb + T - 1) / T;
  k_brick_dist<<<blocks, T, 0, s>>>(log2nb, 0, tmp, dist);
  k_brick_dist<<<blocks, T, 0, s>>>(log2nb, 1, dist, tmp);
  k_brick_dist<<<blocks, T, 0, s>>>(log2nb, 2, tmp, dist);
  return 3;
}

int launch_brick_dist(const GridDev& g, uint8_t* tmp, uint8_t* dist, cudaStream_t s) {
  const uint32_t nb = 1u << (3 * g.log2nb);
  const int T = 256;
  k_brick_occ<<<(nb + T - 1) / T, T, 0, s>>>(g, tmp);
  return 1 + launch_brick_dist_passes(g.log2nb, tmp, dist, s);
}

}  // namespace vrt
