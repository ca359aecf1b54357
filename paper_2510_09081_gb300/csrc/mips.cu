// A2: the averaging occupancy pyramid used by cone-traced ambient occlusion
// (an averaging mipmap, Sec. 3.1; sampled by the cones of Sec. 3.4). Level 0 is
// min(1, occupancy code sum / occ_scale) per voxel, level l+1 the mean of the
// 8 children; each level is stored x-fastest (canonical) so the trace's
// trilinear samples are plain strided loads. Texels are fp32, fp16 or bf16.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "launch.h"

namespace vrt {

// Storage of a texel: fp32, or fp16 / bf16 rounded to nearest from the fp32 value
// (each level is averaged in fp32 from its stored children, then rounded once).
__device__ __forceinline__ void store_texel(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_texel(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void store_texel(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ float load_texel(const float* p) { return *p; }
__device__ __forceinline__ float load_texel(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float load_texel(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Level 0 and 1 together: one thread per level-1 texel reads its 2x2x2 block
// of packed words (two bricks' worth of rows), writes 8 level-0 values and
// the mean of the 8 as stored (so that every level averages its stored
// children).
template <class T>
__global__ void __launch_bounds__(256) k_mip01(GridDev g, T* __restrict__ l0, T* __restrict__ l1) {
  const int m = g.n >> 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)m * m * m) return;
  const int x = (int)(t % m), y = (int)((t / m) % m), z = (int)(t / ((long long)m * m));
  const float inv = 1.0f / g.occ_scale;
  float s = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int X = 2 * x + dx, Y = 2 * y + dy, Z = 2 * z + dz;
        const uint32_t w = g.word[brick_index(X, Y, Z, g.log2nb)];
        T* p = &l0[((long long)Z * g.n + Y) * g.n + X];
        store_texel(p, fminf(1.0f, (float)(w >> 16) * inv));
        s += load_texel(p);
      }
  store_texel(&l1[t], s * 0.125f);
}

template <class T>
__global__ void __launch_bounds__(256) k_mip_down(const T* __restrict__ src, T* __restrict__ dst, int m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)m * m * m) return;
  const int x = (int)(t % m), y = (int)((t / m) % m), z = (int)(t / ((long long)m * m));
  const int mp = 2 * m;
  float s = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const T* row = &src[((long long)(2 * z + dz) * mp + (2 * y + dy)) * mp + 2 * x];
      s += load_texel(row) + load_texel(row + 1);
    }
  store_texel(&dst[t], s * 0.125f);
}

template <class T>
int launch_mips_t(const GridDev& g, T* mips, const long long* lev_off, int n_levels, cudaStream_t s) {
  const int T_ = 256;
  long long m = g.n >> 1;
  long long cnt = m * m * m;
  int launches = 1;
  k_mip01<T><<<(unsigned)((cnt + T_ - 1) / T_), T_, 0, s>>>(g, mips + lev_off[0], mips + lev_off[1]);
  for (int l = 2; l < n_levels; ++l) {
    m = g.n >> l;
    cnt = m * m * m;
    k_mip_down<T><<<(unsigned)((cnt + T_ - 1) / T_), T_, 0, s>>>(mips + lev_off[l - 1], mips + lev_off[l],
                                                                 (int)m);
    ++launches;
  }
  return launches;
}

int launch_mips(const GridDev& g, void* mips, int fmt, const long long* lev_off, int n_levels,
                cudaStream_t s) {
  if (fmt == kMipsF16) return launch_mips_t(g, (__half*)mips, lev_off, n_levels, s);
  if (fmt == kMipsBF16) return launch_mips_t(g, (__nv_bfloat16*)mips, lev_off, n_levels, s);
  return launch_mips_t(g, (float*)mips, lev_off, n_levels, s);
}

}  // namespace vrt
