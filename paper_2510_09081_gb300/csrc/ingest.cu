// A0 ingest: snap vertices to multiples of 2^-14 voxel, attach polyline flags
// and compute clip-plane normals as central-difference tangents (Sec. 3.1,
// clipped capsules after Gross & Gumhold), disabled at polyline ends.
#include "launch.h"

namespace vrt {

__device__ __forceinline__ float snap(float x, bool& bad) {
  if (!(x >= kCoordMin && x < kCoordMax)) {  // also catches NaN
    bad = true;
    x = fminf(fmaxf(x, kCoordMin), kCoordMax - 1.0f);
    if (x != x) x = 0.0f;
  }
  return rintf(x * kUnits) * (1.0f / kUnits);
}

// Vertices [lo, hi): the ones uploaded or updated since the last ingest and
// their polyline neighbours (whose clip normals they enter).
__global__ void __launch_bounds__(256) k_ingest(const float* __restrict__ raw,
                                                const uint8_t* __restrict__ flags, long long lo,
                                                long long hi, float4* __restrict__ pos,
                                                float4* __restrict__ nrm, DevStatus* st) {
  const long long i = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi) return;
  bool bad = false;
  const float x = snap(raw[3 * i], bad), y = snap(raw[3 * i + 1], bad), z = snap(raw[3 * i + 2], bad);
  uint32_t fl = flags[i];
  float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!(fl & (kFirst | kLast))) {
    bool b2 = false;
    const float tx = snap(raw[3 * i + 3], b2) - snap(raw[3 * i - 3], b2);
    const float ty = snap(raw[3 * i + 4], b2) - snap(raw[3 * i - 2], b2);
    const float tz = snap(raw[3 * i + 5], b2) - snap(raw[3 * i - 1], b2);
    const float l2 = tx * tx + ty * ty + tz * tz;
    if (l2 > 0.0f) {
      const float l = sqrtf(l2);
      n = make_float4(tx / l, ty / l, tz / l, 0.f);
      fl |= kClipOn;
    }
  }
  if (bad) set_err(st, kErrRange);
  pos[i] = make_float4(x, y, z, __uint_as_float(fl));
  nrm[i] = n;
}

int launch_ingest(const float* raw, const uint8_t* flags, long long lo, long long hi, float4* pos,
                  float4* nrm, DevStatus* st, cudaStream_t s) {
  if (hi <= lo) return 0;
  const int T = 256;
  k_ingest<<<(unsigned)((hi - lo + T - 1) / T), T, 0, s>>>(raw, flags, lo, hi, pos, nrm, st);
  return 1;
}

// Spatial key of a polyline: the 12-bit Morton code of the 16^3 cell of the
// grid holding vertex mid[p] (any coordinate outside the grid, or not finite,
// is clamped into it; the key only orders work).
__global__ void k_poly_keys(const float* __restrict__ raw, const uint32_t* __restrict__ mid,
                            uint32_t P, float cells_per_voxel, uint16_t* __restrict__ key) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const uint32_t v = mid[p];
  uint32_t k = 0;
  for (int a = 0; a < 3; ++a) {
    const float c = raw[3 * (size_t)v + a] * cells_per_voxel;
    const uint32_t q = c >= 0.0f ? (uint32_t)fminf(c, 15.0f) : 0u;  // NaN -> 0
#pragma unroll
    for (int b = 0; b < 4; ++b) k |= ((q >> b) & 1u) << (3 * b + a);
  }
  key[p] = (uint16_t)k;
}

int launch_poly_keys(const float* raw, const uint32_t* mid, uint32_t P, int n, uint16_t* key,
                     cudaStream_t s) {
  if (P == 0) return 0;
  k_poly_keys<<<(P + 255) / 256, 256, 0, s>>>(raw, mid, P, 16.0f / (float)n, key);
  return 1;
}

}  // namespace vrt
