// A3: voxel-based view culling (Sec. 3.2).
//
// Occupancy is eroded by taking the minimum over each voxel and its six
// neighbours (outside the grid counts as empty), which makes the estimate of
// what blocks the view conservative. Every occupied voxel inside the view
// frustum then marches from its centre toward the camera through the eroded
// occupancy. The march turns occupancy into optical depth: tubes of radius r
// filling a volume fraction e are crossed 2 e / (pi r) times per unit length,
// and each crossing lets 1 - alpha through (an opaque crossing counts as one
// unit), so depth += kappa * e * (path length in the voxel) with
// kappa = 1/2 * 2 / (pi r) * (-ln(1 - alpha) or 1); the factor 1/2 covers the
// occupancy estimate's excess over the true tube volume (about 4/3 for thin
// tubes under the PWAA clamp). A voxel is marked visible unless
// the depth in front of it exceeds ln(1e4) + 3, past the depth where a ray
// stops. The march uses the eroded occupancy at two levels of its pyramid:
// voxels for the first few voxel lengths, then 4^3 bricks (their mean); it
// crosses, in one step, cubes of bricks without eroded occupancy (they add no
// depth), using a distance field over such bricks built after the erosion. The marks decide which voxels get lists; voxels a ray later needs but
// that were left unmarked are listed by the trace's repair rounds, so the
// marks only affect speed.
#include <cmath>

#include "launch.h"

namespace vrt {

constexpr float kCullDepth = 9.2103404f + 3.0f;  // ln(1e4) + 3

__device__ __forceinline__ uint32_t occ8(const GridDev& g, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)g.n || (unsigned)y >= (unsigned)g.n || (unsigned)z >= (unsigned)g.n)
    return 0u;
  const uint32_t q = __ldg(&g.word[brick_index(x, y, z, g.log2nb)]) >> 16;
  return min(255u, (uint32_t)((float)q * (255.0f / g.occ_scale)));
}

// Erosion, and per brick whether any voxel keeps eroded occupancy (0) or none
// does (kBrickDistMax), the seed of the march's skipping field, and the mean
// eroded occupancy. A thread takes one x-row of a brick (four consecutive
// words, one 16-byte load), so 16 threads cover a brick and a warp two; the
// rows next to it in y and z are four consecutive words too. The thread also
// clears its row's bits of the cull marks, and queues the row's voxels that
// hold segments for the march (one atomic per warp) when occq is given.
__device__ __forceinline__ uint32_t occ8w(const GridDev& g, uint32_t w) {
  return min(255u, (uint32_t)((float)(w >> 16) * (255.0f / g.occ_scale)));
}

__device__ __forceinline__ uint4 row_words(const GridDev& g, int x, int y, int z) {
  if ((unsigned)y >= (unsigned)g.n || (unsigned)z >= (unsigned)g.n) return make_uint4(0u, 0u, 0u, 0u);
  return __ldg(reinterpret_cast<const uint4*>(g.word) + (brick_index(x, y, z, g.log2nb) >> 2));
}

__global__ void __launch_bounds__(256) k_erode(GridDev g, uint8_t* __restrict__ eroded,
                                               uint8_t* __restrict__ ebrick,
                                               float* __restrict__ emean,
                                               uint32_t* __restrict__ occq,
                                               unsigned long long occq_cap) {
  const uint32_t row = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nrow = ((uint32_t)g.n * g.n * g.n) >> 2;  // a multiple of 32 (n >= 16)
  const int lane = threadIdx.x & 31;
  if (row >= nrow) return;  // whole warps
  const uint32_t idx0 = row << 2;
  int x, y, z;
  brick_coords(idx0, g.log2nb, x, y, z);  // x: a multiple of 4
  const uint4 w = __ldg(reinterpret_cast<const uint4*>(g.word) + row);
  const uint32_t o[4] = {occ8w(g, w.x), occ8w(g, w.y), occ8w(g, w.z), occ8w(g, w.w)};
  uint32_t e[4] = {o[0], o[1], o[2], o[3]};
  if (o[0] | o[1] | o[2] | o[3]) {
    // x neighbours: the row's own voxels, and one word of each neighbouring brick
    const uint32_t xm = x > 0 ? occ8w(g, __ldg(&g.word[brick_index(x - 1, y, z, g.log2nb)])) : 0u;
    const uint32_t xp = x + 4 < g.n ? occ8w(g, __ldg(&g.word[brick_index(x + 4, y, z, g.log2nb)])) : 0u;
    const uint4 ym = row_words(g, x, y - 1, z), yp = row_words(g, x, y + 1, z);
    const uint4 zm = row_words(g, x, y, z - 1), zp = row_words(g, x, y, z + 1);
    const uint32_t wy0[4] = {ym.x, ym.y, ym.z, ym.w}, wy1[4] = {yp.x, yp.y, yp.z, yp.w};
    const uint32_t wz0[4] = {zm.x, zm.y, zm.z, zm.w}, wz1[4] = {zp.x, zp.y, zp.z, zp.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!e[k]) continue;
      uint32_t v = min(e[k], k > 0 ? o[k - 1] : xm);
      v = min(v, k < 3 ? o[k + 1] : xp);
      v = min(v, min(occ8w(g, wy0[k]), occ8w(g, wy1[k])));
      v = min(v, min(occ8w(g, wz0[k]), occ8w(g, wz1[k])));
      e[k] = v;
    }
  }
  reinterpret_cast<uchar4*>(eroded)[row] =
      make_uchar4((uint8_t)e[0], (uint8_t)e[1], (uint8_t)e[2], (uint8_t)e[3]);
  if ((row & 7u) == 0) g.vis[idx0 >> 5] = 0u;  // marks: set by the march
  // the brick's 16 rows are lanes 0-15 or 16-31
  uint32_t esum = e[0] + e[1] + e[2] + e[3];
#pragma unroll
  for (int off = 8; off > 0; off >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, off);
  if ((lane & 15) == 0) {
    const uint32_t b = row >> 4;
    ebrick[b] = esum ? 0 : (uint8_t)kBrickDistMax;
    emean[b] = (float)esum * (1.0f / (255.0f * 64.0f));
  }
  if (occq) {
    const uint32_t om = ((w.x & 0xffffu) ? 1u : 0u) | ((w.y & 0xffffu) ? 2u : 0u) |
                        ((w.z & 0xffffu) ? 4u : 0u) | ((w.w & 0xffffu) ? 8u : 0u);
    const uint32_t nq = __popc(om);
    uint32_t incl = nq;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0;
    if (lane == 0 && total) base = atomicAdd(&g.st->occq_cnt, total);
    base = __shfl_sync(0xffffffffu, base, 0);
    unsigned long long k = (unsigned long long)base + (incl - nq);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((om >> j) & 1u) {
        if (k < occq_cap) occq[k] = idx0 + (uint32_t)j;
        ++k;
      }
  }
}

struct CullCam {
  float3 eye, f, nr, nl, nt, nb;  // perspective: inward side-plane normals
  float3 rt, up;                  // orthographic: half extents along right / up
  float hw, hh, lr, ll, lt, lb;   // |n| * sqrt(3)/2 margins
  float kappa;                    // optical depth per unit length at full occupancy
  float depth_max;                // estimated depth beyond which a voxel is culled
  int ortho;
};

// Voxel steps of the march before it continues brick by brick.
constexpr float kCullNear = 6.0f;

// Whether occupied voxel idx keeps its list: inside the view frustum, and the
// estimated optical depth between it and the camera stays below cc.depth_max.
__device__ bool voxel_visible(const GridDev& g, const CullCam& cc, const uint8_t* __restrict__ eroded,
                              const uint8_t* __restrict__ cdist, const float* __restrict__ emean,
                              uint32_t idx) {
  bool visible = false;
  {
    int x, y, z;
    brick_coords(idx, g.log2nb, x, y, z);
    const float3 c = make_float3(x + 0.5f, y + 0.5f, z + 0.5f);
    const float3 v = c - cc.eye;
    const float h = 0.8660254f;
    bool inside;
    float3 dir;
    float tmax;
    if (cc.ortho) {
      inside = dot3(v, cc.f) >= -h && fabsf(dot3(v, cc.rt)) <= cc.hw + h &&
               fabsf(dot3(v, cc.up)) <= cc.hh + h;
      dir = make_float3(-cc.f.x, -cc.f.y, -cc.f.z);
      tmax = __int_as_float(0x7f800000);
    } else {
      inside = dot3(v, cc.f) >= -h && dot3(v, cc.nr) >= -cc.lr && dot3(v, cc.nl) >= -cc.ll &&
               dot3(v, cc.nt) >= -cc.lt && dot3(v, cc.nb) >= -cc.lb;
      const float dist = sqrtf(dot3(v, v));
      dir = dist > 0.0f ? (-1.0f / dist) * v : make_float3(0.f, 0.f, 1.f);
      tmax = dist;
    }
    if (inside) {
      // March from the centre toward the camera through the eroded occupancy
      // pyramid: voxel by voxel for the first kCullNear voxel lengths, then
      // brick by brick with each 4^3 brick's mean, crossing cubes of bricks
      // without eroded occupancy (which add no depth) in one step.
      const int n = g.n, nb = n >> 2;
      int px = x, py = y, pz = z;
      const int sx = dir.x > 0.0f ? 1 : (dir.x < 0.0f ? -1 : 0);
      const int sy = dir.y > 0.0f ? 1 : (dir.y < 0.0f ? -1 : 0);
      const int sz = dir.z > 0.0f ? 1 : (dir.z < 0.0f ? -1 : 0);
      const float ix = dir.x != 0.0f ? 1.0f / dir.x : 0.0f;
      const float iy = dir.y != 0.0f ? 1.0f / dir.y : 0.0f;
      const float iz = dir.z != 0.0f ? 1.0f / dir.z : 0.0f;
      // parameter where the march leaves [lo, hi] along one axis
      auto leave = [](int s, int lo, int hi, float o, float inv) {
        return s != 0 ? ((float)(s > 0 ? hi : lo) - o) * inv : __int_as_float(0x7f800000);
      };
      float depth = 0.0f, tcur = 0.0f;
      bool counted = false;  // the voxel itself adds nothing to the depth in front of it
      bool done = false;
      visible = true;
      // near: voxels
      for (int it = 0; it < 3 * n + 16 && !done; ++it) {
        const float tx = leave(sx, px, px + 1, c.x, ix);
        const float ty = leave(sy, py, py + 1, c.y, iy);
        const float tz = leave(sz, pz, pz + 1, c.z, iz);
        const float te = fminf(tx, fminf(ty, tz));
        if (counted) {
          const float e = (float)__ldg(&eroded[brick_index(px, py, pz, g.log2nb)]) * (1.0f / 255.0f);
          depth = fmaf(cc.kappa * e, fminf(te, tmax) - tcur, depth);
          if (depth > cc.depth_max) { visible = false; done = true; break; }
        }
        counted = true;
        if (te >= tmax) { done = true; break; }
        if (te == tx) px += sx; else if (te == ty) py += sy; else pz += sz;
        if ((unsigned)px >= (unsigned)n || (unsigned)py >= (unsigned)n || (unsigned)pz >= (unsigned)n) {
          done = true;
          break;
        }
        tcur = te;
        if (tcur >= kCullNear) break;  // on to bricks, at voxel p from tcur
      }
      // far: bricks (brick coordinates bx, by, bz; the march is in brick b from tcur)
      int bx = px >> 2, by = py >> 2, bz = pz >> 2;
      for (int it = 0; it < 3 * nb + 16 && !done; ++it) {
        const uint32_t bidx = ((uint32_t)bz << (2 * g.log2nb)) | ((uint32_t)by << g.log2nb) | (uint32_t)bx;
        const int kd = __ldg(&cdist[bidx]);
        if (kd > 0) {
          // cross the cube of bricks within kd - 1 of this one (voxel box [lo, lo + w))
          const int ext = kd - 1;
          const int lx = 4 * (bx - ext), ly = 4 * (by - ext), lz = 4 * (bz - ext), w = 4 * (2 * ext + 1);
          const float ux = leave(sx, lx, lx + w, c.x, ix);
          const float uy = leave(sy, ly, ly + w, c.y, iy);
          const float uz = leave(sz, lz, lz + w, c.z, iz);
          const float tb = fminf(ux, fminf(uy, uz));
          if (tb >= tmax) break;
          const int qx = min(min(bx + ext, nb - 1), max(max(bx - ext, 0), (int)floorf(fmaf(tb, dir.x, c.x) * 0.25f)));
          const int qy = min(min(by + ext, nb - 1), max(max(by - ext, 0), (int)floorf(fmaf(tb, dir.y, c.y) * 0.25f)));
          const int qz = min(min(bz + ext, nb - 1), max(max(bz - ext, 0), (int)floorf(fmaf(tb, dir.z, c.z) * 0.25f)));
          if (tb == ux) { bx = sx > 0 ? bx + ext + 1 : bx - ext - 1; by = qy; bz = qz; }
          else if (tb == uy) { by = sy > 0 ? by + ext + 1 : by - ext - 1; bx = qx; bz = qz; }
          else { bz = sz > 0 ? bz + ext + 1 : bz - ext - 1; bx = qx; by = qy; }
          if ((unsigned)bx >= (unsigned)nb || (unsigned)by >= (unsigned)nb || (unsigned)bz >= (unsigned)nb) break;
          tcur = tb;
          continue;
        }
        const float tx = leave(sx, 4 * bx, 4 * bx + 4, c.x, ix);
        const float ty = leave(sy, 4 * by, 4 * by + 4, c.y, iy);
        const float tz = leave(sz, 4 * bz, 4 * bz + 4, c.z, iz);
        const float te = fminf(tx, fminf(ty, tz));
        depth = fmaf(cc.kappa * __ldg(&emean[bidx]), fminf(te, tmax) - tcur, depth);
        if (depth > cc.depth_max) { visible = false; break; }
        if (te >= tmax) break;
        if (te == tx) bx += sx; else if (te == ty) by += sy; else bz += sz;
        if ((unsigned)bx >= (unsigned)nb || (unsigned)by >= (unsigned)nb || (unsigned)bz >= (unsigned)nb) break;
        tcur = te;
      }
    }
  }
  return visible;
}

// One thread per voxel; the warp writes its 32 marks.
__global__ void __launch_bounds__(256) k_visible(GridDev g, CullCam cc,
                                                 const uint8_t* __restrict__ eroded,
                                                 const uint8_t* __restrict__ cdist,
                                                 const float* __restrict__ emean) {
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nvox = (uint32_t)g.n * g.n * g.n;
  const bool visible = idx < nvox && (__ldg(&g.word[idx]) & 0xffffu) &&
                       voxel_visible(g, cc, eroded, cdist, emean, idx);
  const uint32_t m = __ballot_sync(0xffffffffu, visible);
  if ((threadIdx.x & 31) == 0 && idx < nvox) g.vis[idx >> 5] = m;
}

// One thread per queued occupied voxel (the erosion cleared the marks): every
// lane of a warp marches, where one thread per voxel leaves the lanes of empty
// voxels idle (ABC pathlines at 512^3 occupy a third of the grid).
__global__ void __launch_bounds__(256) k_visible_queued(GridDev g, CullCam cc,
                                                        const uint8_t* __restrict__ eroded,
                                                        const uint8_t* __restrict__ cdist,
                                                        const float* __restrict__ emean,
                                                        const uint32_t* __restrict__ occq,
                                                        unsigned long long occq_cap) {
  const unsigned long long cnt = min((unsigned long long)g.st->occq_cnt, occq_cap);
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < cnt;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t idx = __ldg(&occq[q]);
    if (voxel_visible(g, cc, eroded, cdist, emean, idx)) atomicOr(&g.vis[idx >> 5], 1u << (idx & 31));
  }
}

namespace {
struct D3 { double x, y, z; };
D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
D3 add(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
D3 mul(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
D3 crs(D3 a, D3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double len(D3 a) { return std::sqrt(a.x * a.x + a.y * a.y + a.z * a.z); }
D3 nrmz(D3 a) { return mul(1.0 / len(a), a); }
float3 tof(D3 a) { return make_float3((float)a.x, (float)a.y, (float)a.z); }
}  // namespace

int launch_cull(const GridDev& g, const HostCamera& cam, float alpha, uint8_t* eroded,
                uint8_t* btmp, uint8_t* cdist, float* emean, float depth_max, uint32_t* occq,
                unsigned long long occq_cap, cudaStream_t s) {
  const D3 eye = {cam.eye[0], cam.eye[1], cam.eye[2]};
  const D3 tgt = {cam.target[0], cam.target[1], cam.target[2]};
  const D3 upw = {cam.up[0], cam.up[1], cam.up[2]};
  const D3 f = nrmz(sub(tgt, eye));
  const D3 rt = nrmz(crs(f, upw));
  const D3 up = crs(rt, f);
  const double aspect = (double)cam.width / (double)cam.height;
  const double h = 0.8660254037844386;
  CullCam cc;
  cc.ortho = cam.ortho;
  cc.depth_max = depth_max > 0.0f ? depth_max : kCullDepth;
  // x 1/2: sampled PWAA occupancy integrates to about 4/3 of the tubes' true
  // volume, and the estimate must stay below the depth a ray really sees
  cc.kappa = (float)(0.5 * 2.0 / (3.14159265358979323846 * g.r) *
                     (alpha < 1.0f ? -std::log(1.0 - (double)alpha) : 1.0));
  cc.eye = tof(eye);
  cc.f = tof(f);
  cc.rt = tof(rt);
  cc.up = tof(up);
  cc.hh = (float)(0.5 * cam.ortho_h);
  cc.hw = (float)(0.5 * cam.ortho_h * aspect);
  const double th = std::tan(cam.fovy_deg * 3.14159265358979323846 / 360.0);
  const D3 nr = sub(mul(th * aspect, f), rt), nl = add(mul(th * aspect, f), rt);
  const D3 nt = sub(mul(th, f), up), nb = add(mul(th, f), up);
  cc.nr = tof(nr); cc.nl = tof(nl); cc.nt = tof(nt); cc.nb = tof(nb);
  // a little slack on top of the bounding sphere keeps the test conservative
  cc.lr = (float)(len(nr) * h + 1e-3); cc.ll = (float)(len(nl) * h + 1e-3);
  cc.lt = (float)(len(nt) * h + 1e-3); cc.lb = (float)(len(nb) * h + 1e-3);
  const uint32_t nvox = (uint32_t)g.n * g.n * g.n;
  const int T = 256;
  // the queue holds every voxel at most once, so it never overflows when it
  // has room for the whole grid; otherwise each voxel's thread tests its own
  const bool queued = occq && occq_cap >= nvox;
  k_erode<<<(nvox / 4 + T - 1) / T, T, 0, s>>>(g, eroded, btmp, emean, queued ? occq : nullptr,
                                               occq_cap);
  const int passes = launch_brick_dist_passes(g.log2nb, btmp, cdist, s);
  if (queued) k_visible_queued<<<152 * 8, T, 0, s>>>(g, cc, eroded, cdist, emean, occq, occq_cap);
  else k_visible<<<(nvox + T - 1) / T, T, 0, s>>>(g, cc, eroded, cdist, emean);
  return 2 + passes;
}

}  // namespace vrt
