// A2: the averaging occupancy pyramid used by cone-traced ambient occlusion
// (Sec. 3.1 "averaging mipmap", Sec. 3.4 cones). Level 0 is
// min(1, occupancy code sum / occ_scale) per voxel, level l+1 the mean of the
// 8 children; each level is stored x-fastest (canonical) so the trace's
// trilinear samples are plain strided loads.
#include "launch.h"

namespace vrt {

// Level 0 and 1 together: one thread per level-1 texel reads its 2x2x2 block
// of packed words (two bricks' worth of rows) and writes 8 level-0 values and
// their mean.
__global__ void __launch_bounds__(256) k_mip01(GridDev g, float* __restrict__ l0,
                                               float* __restrict__ l1) {
  const int m = g.n >> 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)m * m * m) return;
  const int x = (int)(t % m), y = (int)((t / m) % m), z = (int)(t / ((long long)m * m));
  const float inv = 1.0f / g.occ_scale;
  float s = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int X = 2 * x, Y = 2 * y + dy, Z = 2 * z + dz;
      const uint32_t w0 = g.word[brick_index(X, Y, Z, g.log2nb)];
      const uint32_t w1 = g.word[brick_index(X + 1, Y, Z, g.log2nb)];
      const float o0 = fminf(1.0f, (float)(w0 >> 16) * inv);
      const float o1 = fminf(1.0f, (float)(w1 >> 16) * inv);
      *reinterpret_cast<float2*>(&l0[((long long)Z * g.n + Y) * g.n + X]) = make_float2(o0, o1);
      s += o0 + o1;
    }
  l1[t] = s * 0.125f;
}

__global__ void __launch_bounds__(256) k_mip_down(const float* __restrict__ src, float* __restrict__ dst,
                                                  int m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)m * m * m) return;
  const int x = (int)(t % m), y = (int)((t / m) % m), z = (int)(t / ((long long)m * m));
  const int mp = 2 * m;
  float s = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const float2 v = *reinterpret_cast<const float2*>(
          &src[((long long)(2 * z + dz) * mp + (2 * y + dy)) * mp + 2 * x]);
      s += v.x + v.y;
    }
  dst[t] = s * 0.125f;
}

int launch_mips(const GridDev& g, float* mips, const long long* lev_off, int n_levels,
                 cudaStream_t s) {
  const int T = 256;
  long long m = g.n >> 1;
  long long cnt = m * m * m;
  int launches = 1;
  k_mip01<<<(unsigned)((cnt + T - 1) / T), T, 0, s>>>(g, mips + lev_off[0], mips + lev_off[1]);
  for (int l = 2; l < n_levels; ++l) {
    m = g.n >> l;
    cnt = m * m * m;
    k_mip_down<<<(unsigned)((cnt + T - 1) / T), T, 0, s>>>(mips + lev_off[l - 1], mips + lev_off[l],
                                                           (int)m);
    ++launches;
  }
  return launches;
}

}  // namespace vrt
