// Voxel-space shading (Sec. 3.4, Shading).
//
// The paper evaluates global illumination once per voxel before ray tracing,
// so that a ray-capsule hit costs one texture sample: cone-traced ambient
// occlusion (cones spread over the whole sphere, sampling the occupancy
// pyramid) and a directional shadow traced from the voxel centre toward the
// light, for voxels marked visible. Here the value stored for voxel v is
//   AO(c_v) * (1/2 + 1/2 * S(c_v)),
// AO the six-cone occlusion of the per-hit path evaluated at the centre c_v,
// S the transmittance of the ray c_v + k L, k = 1, 2, ..., through the base
// level of the pyramid (trilinear at texel centres, A <- A + (1 - A) s,
// S = 1 - A), ended where a sample's texels all lie outside the grid. The
// trace samples the field trilinearly at each hit, which reads the centres of
// the hit voxel and of its neighbours, so the field is computed for every
// voxel within one step of a listed voxel (and, in each culling-repair round,
// next to the voxels that round lists).
//
// Empty space: a shadow sample whose texels all lie in bricks the brick
// distance field proves empty is exactly zero and leaves A unchanged, so the
// march steps over the run of such samples (an integer number of steps, the
// sample positions stay those of the plain march). The march stops early once
// S < 1e-4, which moves the stored value by less than 5e-5.
#include "launch.h"
#include "pyramid.cuh"

namespace vrt {

namespace {

constexpr float kShadowStop = 1e-4f;  // transmittance below which the march ends

__device__ __forceinline__ bool listed_at(const GridDev& g, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)g.n || (unsigned)y >= (unsigned)g.n || (unsigned)z >= (unsigned)g.n)
    return false;
  const uint32_t i = brick_index(x, y, z, g.log2nb);
  return (__ldg(&g.word[i]) & 0xffffu) && ((__ldg(&g.vis[i >> 5]) >> (i & 31)) & 1u);
}

// Transmittance from P toward the light through the base occupancy level.
__device__ float shadow_clear(const ShadeArgs& A, float3 P) {
  const int n = A.g.n;
  const float lo = -0.5f, hi = (float)n + 0.5f;
  const float3 L = make_float3(A.lx, A.ly, A.lz);
  float acc = 0.0f;  // accumulated occlusion
  float t = 1.0f;    // integer steps: exact in fp32
  // each iteration advances t by at least 1, and the ray leaves the box
  // [lo, hi]^3 within sqrt(3) (n + 1) + 1 steps
  const int max_it = 2 * n + 8;
  for (int it = 0; it < max_it; ++it) {
    const float3 q = make_float3(fmaf(t, L.x, P.x), fmaf(t, L.y, P.y), fmaf(t, L.z, P.z));
    if (!(q.x >= lo && q.x <= hi && q.y >= lo && q.y <= hi && q.z >= lo && q.z <= hi)) break;
    const int vx = min(max((int)floorf(q.x), 0), n - 1);
    const int vy = min(max((int)floorf(q.y), 0), n - 1);
    const int vz = min(max((int)floorf(q.z), 0), n - 1);
    const uint32_t b = ((uint32_t)(vz >> 2) << (2 * A.g.log2nb)) | ((uint32_t)(vy >> 2) << A.g.log2nb) |
                       (uint32_t)(vx >> 2);
    const int kd = __ldg(&A.g.bdist[b]);
    if (kd >= 2) {
      // bricks within kd - 1 of this one are empty: the voxels [b0, b0 + w)
      // per axis. A sample reads texels floor(q - 1/2) and one more, all in
      // that range while q lies in [b0 + 1/2, b0 + w - 1/2).
      const int ext = 4 * (kd - 1), w = 4 + 2 * ext;
      const float bx = (float)((vx & ~3) - ext), by = (float)((vy & ~3) - ext),
                  bz = (float)((vz & ~3) - ext);
      float te = __int_as_float(0x7f800000);
      if (L.x != 0.0f) te = fminf(te, ((L.x > 0.0f ? bx + (float)w - 0.5f : bx + 0.5f) - P.x) / L.x);
      if (L.y != 0.0f) te = fminf(te, ((L.y > 0.0f ? by + (float)w - 0.5f : by + 0.5f) - P.y) / L.y);
      if (L.z != 0.0f) te = fminf(te, ((L.z > 0.0f ? bz + (float)w - 0.5f : bz + 0.5f) - P.z) / L.z);
      // samples up to te - 0.01 lie inside (margin for the rounding of te);
      // the current one does by the test above
      t = fmaxf(t + 1.0f, floorf(te - 0.01f) + 1.0f);
      continue;
    }
    const float s = trilinear(A.mips, A.mips_fmt, n, 1.0f, q);
    acc = fmaf(1.0f - acc, s, acc);
    if (1.0f - acc < kShadowStop) break;
    t += 1.0f;
  }
  return 1.0f - acc;
}

__device__ float voxel_shade(const ShadeArgs& A, int x, int y, int z) {
  const float3 P = make_float3((float)x + 0.5f, (float)y + 0.5f, (float)z + 0.5f);
  const float ao = A.ao ? ao_lane(A, P) : 1.0f;
  return ao * fmaf(0.5f, shadow_clear(A, P), 0.5f);
}

// One block per brick: the brick's voxels that have a listed voxel among
// their 26 neighbours (or are listed) get a value; the mask records which.
__global__ void __launch_bounds__(64) k_shade(ShadeArgs A) {
  const int lb = A.g.log2nb;
  const uint32_t mb = (1u << lb) - 1u;
  const uint32_t b = blockIdx.x;
  const int t = threadIdx.x;
  // a brick at distance >= 2 from every occupied brick has no listed voxel
  // within one step of any of its voxels
  if (__ldg(&A.g.bdist[b]) >= 2) {
    if (t < 2) A.mask[2 * b + t] = 0u;
    return;
  }
  const int bx = 4 * (int)(b & mb), by = 4 * (int)((b >> lb) & mb), bz = 4 * (int)(b >> (2 * lb));
  __shared__ uint8_t s_l[216];  // listed flags of the brick and a one-voxel halo (6^3)
  for (int i = t; i < 216; i += 64)
    s_l[i] = listed_at(A.g, bx - 1 + i % 6, by - 1 + (i / 6) % 6, bz - 1 + i / 36) ? 1 : 0;
  __syncthreads();
  const int lx = t & 3, ly = (t >> 2) & 3, lz = t >> 4;  // brick_index's in-brick order
  bool need = false;
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) need |= s_l[(lz + dz) * 36 + (ly + dy) * 6 + lx + dx] != 0;
  const uint32_t ball = __ballot_sync(0xffffffffu, need);
  if ((t & 31) == 0) A.mask[2 * b + (t >> 5)] = ball;
  if (need) A.shade[(b << 6) | (uint32_t)t] = voxel_shade(A, bx + lx, by + ly, bz + lz);
}

// Repair round: the neighbours of each newly listed voxel not shaded yet; the
// thread that sets a voxel's mask bit computes its value.
__global__ void k_shade_repair(ShadeArgs A) {
  const uint32_t nq = min(*A.vq_cnt, A.vq_cap);
  const int n = A.g.n;
  const unsigned long long tot = (unsigned long long)nq * 27ull;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < tot;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t v = A.vq[i / 27];
    const int d = (int)(i % 27);
    int x, y, z;
    brick_coords(v, A.g.log2nb, x, y, z);
    x += d % 3 - 1;
    y += (d / 3) % 3 - 1;
    z += d / 9 - 1;
    if ((unsigned)x >= (unsigned)n || (unsigned)y >= (unsigned)n || (unsigned)z >= (unsigned)n) continue;
    const uint32_t u = brick_index(x, y, z, A.g.log2nb), bit = 1u << (u & 31);
    if (A.mask[u >> 5] & bit) continue;
    if (atomicOr(&A.mask[u >> 5], bit) & bit) continue;
    A.shade[u] = voxel_shade(A, x, y, z);
  }
}

}  // namespace

int launch_shade(const ShadeArgs& a, cudaStream_t s) {
  const unsigned n_bricks = 1u << (3 * a.g.log2nb);
  k_shade<<<n_bricks, 64, 0, s>>>(a);
  return 1;
}

int launch_shade_repair(const ShadeArgs& a, cudaStream_t s) {
  k_shade_repair<<<152, 256, 0, s>>>(a);
  return 1;
}

}  // namespace vrt
