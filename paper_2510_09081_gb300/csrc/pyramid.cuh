// Sampling of the occupancy pyramid and cone-traced ambient occlusion (Sec. 3.4),
// shared by the trace (AO per hit) and the voxel-space shading kernels. The
// functions take any argument struct with the pyramid's fields: g.n, mips,
// mips_fmt, lev_off[], n_levels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vrt_internal.cuh"

namespace vrt {

constexpr float kConeTan = 1.1180340f;    // tan(half angle), cos(half angle) = 2/3
constexpr int kConeSteps = 4;             // samples per cone: t = 1, 2.118, 4.486, 9.502 (<= 16)

// Texel i of a pyramid level stored in format fmt, widened to fp32.
__device__ __forceinline__ float texel(const void* lev, int fmt, int m, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)m || (unsigned)y >= (unsigned)m || (unsigned)z >= (unsigned)m)
    return 0.0f;
  const long long i = ((long long)z * m + y) * m + x;
  if (fmt == kMipsF16) return __half2float(__ldg((const __half*)lev + i));
  if (fmt == kMipsBF16) return __bfloat162float(__ldg((const __nv_bfloat16*)lev + i));
  return __ldg((const float*)lev + i);
}

__device__ __forceinline__ float trilinear(const void* lev, int fmt, int m, float scale, float3 q) {
  const float ux = q.x * scale - 0.5f, uy = q.y * scale - 0.5f, uz = q.z * scale - 0.5f;
  const float fx0 = floorf(ux), fy0 = floorf(uy), fz0 = floorf(uz);
  const int x = (int)fx0, y = (int)fy0, z = (int)fz0;
  const float fx = ux - fx0, fy = uy - fy0, fz = uz - fz0;
  float acc = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dz ? fz : 1.0f - fz);
        acc = fmaf(w, texel(lev, fmt, m, x + dx, y + dy, z + dz), acc);
      }
  return acc;
}

// One cone sample: cone c (axis c/2, sign by parity), step k; returns 1 - s.
template <class Args>
__device__ float cone_sample_clear(const Args& A, float3 P, int c, int k) {
  float t = 1.0f;
  for (int q = 0; q < k; ++q) t += 0.5f * fmaxf(1.0f, 2.0f * t * kConeTan);
  if (t > 16.0f) return 1.0f;
  const float dia = fmaxf(1.0f, 2.0f * t * kConeTan);
  const int maxl = A.n_levels - 1;
  const float lam = fminf(log2f(dia), (float)maxl);
  const int l0 = (int)floorf(lam);
  const float fl = lam - (float)l0;
  const float sg = (c & 1) ? -1.0f : 1.0f;
  float3 q = P;
  const int ax = c >> 1;
  if (ax == 0) q.x += sg * t; else if (ax == 1) q.y += sg * t; else q.z += sg * t;
  const int tb = A.mips_fmt == kMipsF32 ? 4 : 2;  // bytes per texel
  const char* base = (const char*)A.mips;
  float s = trilinear(base + tb * A.lev_off[l0], A.mips_fmt, A.g.n >> l0, 1.0f / (float)(1 << l0), q);
  if (fl > 0.0f && l0 + 1 <= maxl)
    s = (1.0f - fl) * s + fl * trilinear(base + tb * A.lev_off[l0 + 1], A.mips_fmt, A.g.n >> (l0 + 1),
                                         1.0f / (float)(2 << l0), q);
  return 1.0f - s;
}

// AO at P by one lane: mean over cones of prod_k (1 - s_k).
template <class Args>
__device__ __noinline__ float ao_lane(const Args& A, float3 P) {
  float sum = 0.0f;
  for (int c = 0; c < 6; ++c) {
    float p = 1.0f;
    for (int k = 0; k < kConeSteps; ++k) p *= cone_sample_clear(A, P, c, k);
    sum += p;
  }
  return sum * (1.0f / 6.0f);
}

// AO at P (same P in every lane) by the whole warp: lane 4c + k takes sample k
// of cone c.
template <class Args>
__device__ __noinline__ float ao_warp(const Args& A, float3 P) {
  const int lane = threadIdx.x & 31;
  float v = lane < 6 * kConeSteps ? cone_sample_clear(A, P, lane / kConeSteps, lane % kConeSteps) : 1.0f;
  v *= __shfl_xor_sync(0xffffffffu, v, 1);
  v *= __shfl_xor_sync(0xffffffffu, v, 2);   // product over the cone's 4 samples
  float s = (lane < 6 * kConeSteps && (lane & 3) == 0) ? v : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s * (1.0f / 6.0f);
}

}  // namespace vrt
