// A6: voxel ray tracing (Sec. 3.5).
//
// One thread per pixel; a warp covers an 8x4 pixel tile so its rays cross
// the same voxels and lists. Each ray is clipped to the grid box and stepped
// by 3D-DDA (Amanatides & Woo); bricks with no occupied voxel are crossed in
// one step (empty-space skipping). In each voxel every listed segment's first
// entry into its capsule is computed; an entry counts only if it lies in this
// voxel's parameter interval [t_enter, t_exit) -- the intervals partition the
// ray, so each hit is counted once and hits come out voxel by voxel in depth
// order -- and both clip planes keep it.
//  - opaque (K = 1): nearest entry in the first voxel that has one, then stop;
//  - transparent (K > 1): the K nearest entries of the voxel are kept sorted
//    in registers as 64-bit keys (depth bits << 32 | segment id), composited
//    front to back; a voxel holding more than K entries is scanned again for
//    keys beyond the last composited one (ground-truth order). The ray stops
//    once transmittance drops below 1e-4.
// Shading: colour = |unit tangent| (tangent colouring) times cone-traced
// ambient occlusion when enabled (six cones over the occupancy pyramid).
//
// Culling validation: a ray that reaches a voxel holding segments but no list
// queues the voxel (deduplicated by a bitmap), marches on as if the voxel were
// empty -- until it has queued max_queue voxels -- and finally queues its pixel
// instead of writing it; the repair round lists the queued voxels and traces
// the pixel again, so the image never depends on the culling heuristic. With
// no limit, the march queues every culled voxel before the point where it
// ends; the voxels' hits could only end the ray sooner, so the next trace
// of that pixel needs nothing more.
#include "launch.h"

namespace vrt {

__device__ __forceinline__ bool bit_at(const uint32_t* bits, uint32_t i) {
  return (bits[i >> 5] >> (i & 31)) & 1u;
}

// ------------------------------------------------ ambient occlusion (Sec 3.4)
__device__ __forceinline__ float texel(const float* lev, int m, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)m || (unsigned)y >= (unsigned)m || (unsigned)z >= (unsigned)m)
    return 0.0f;
  return __ldg(&lev[((long long)z * m + y) * m + x]);
}

__device__ __forceinline__ float trilinear(const float* lev, int m, float scale, float3 q) {
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
        acc = fmaf(w, texel(lev, m, x + dx, y + dy, z + dz), acc);
      }
  return acc;
}

__device__ float ambient_occlusion(const TraceArgs& A, float3 P) {
  const float tan_half = 1.1180340f;  // cos(half angle) = 2/3: six cones tile the sphere
  const int maxl = A.n_levels - 1;
  float sumA = 0.0f;
  for (int cone = 0; cone < 6; ++cone) {
    const float sg = (cone & 1) ? -1.0f : 1.0f;
    const int ax = cone >> 1;
    float occl = 0.0f, t = 1.0f;
    while (t <= 16.0f) {
      const float dia = fmaxf(1.0f, 2.0f * t * tan_half);
      float lam = fminf(log2f(dia), (float)maxl);
      const int l0 = (int)floorf(lam);
      const float fl = lam - (float)l0;
      float3 q = P;
      if (ax == 0) q.x += sg * t; else if (ax == 1) q.y += sg * t; else q.z += sg * t;
      float s = trilinear(A.mips + A.lev_off[l0], A.g.n >> l0, 1.0f / (float)(1 << l0), q);
      if (fl > 0.0f && l0 + 1 <= maxl)
        s = (1.0f - fl) * s +
            fl * trilinear(A.mips + A.lev_off[l0 + 1], A.g.n >> (l0 + 1), 1.0f / (float)(2 << l0), q);
      occl = occl + (1.0f - occl) * s;
      t += dia * 0.5f;
    }
    sumA += occl;
  }
  return 1.0f - sumA * (1.0f / 6.0f);
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ bool clip_keeps(const TraceArgs& A, float3 P, float4 p0, float4 p1,
                                           uint32_t id) {
  if (__float_as_uint(p0.w) & kClipOn) {
    const float3 n0 = f3(__ldg(&A.nrm[id]));
    if (dot3(P - f3(p0), n0) < 0.0f) return false;
  }
  if (__float_as_uint(p1.w) & kClipOn) {
    const float3 n1 = f3(__ldg(&A.nrm[id + 1]));
    if (dot3(P - f3(p1), n1) > 0.0f) return false;
  }
  return true;
}

struct RayState {
  float3 o, d;
  float C[3];
  float T;
  int first_id;
  float first_t;
};

__device__ __forceinline__ void shade(const TraceArgs& A, RayState& R, uint32_t id, float t) {
  const float3 a = f3(__ldg(&A.pos[id])), b = f3(__ldg(&A.pos[id + 1]));
  const float3 dv = b - a;
  const float l2 = dot3(dv, dv);
  float3 c = make_float3(1.0f, 1.0f, 1.0f);
  if (l2 > 0.0f) {
    const float il = 1.0f / sqrtf(l2);
    c = make_float3(fabsf(dv.x) * il, fabsf(dv.y) * il, fabsf(dv.z) * il);
  }
  if (A.ao) {
    const float ao = ambient_occlusion(A, R.o + t * R.d);
    c = ao * c;
  }
  const float w = R.T * A.alpha;
  R.C[0] = fmaf(w, c.x, R.C[0]);
  R.C[1] = fmaf(w, c.y, R.C[1]);
  R.C[2] = fmaf(w, c.z, R.C[2]);
  R.T *= (1.0f - A.alpha);
  if (R.first_id < 0) {
    R.first_id = (int)id;
    R.first_t = t;
  }
}

// Process one voxel's list over [t0, t1). Returns true when the ray is done.
template <int K>
__device__ __forceinline__ bool process_voxel(const TraceArgs& A, RayState& R, uint32_t beg,
                                              uint32_t end, float t0, float t1) {
  const float r2 = A.g.r * A.g.r;
  if (K == 1) {
    float bt = __int_as_float(0x7f800000);
    uint32_t bid = 0xffffffffu;
    for (uint32_t s = beg; s < end; ++s) {
      const uint32_t id = __ldg(&A.g.lists[s]);
      if (id + 1 >= A.n_vert) { set_err(A.g.st, kErrBounds); continue; }
      const float4 p0 = __ldg(&A.pos[id]), p1 = __ldg(&A.pos[id + 1]);
      const float t = capsule_entry(R.o, R.d, f3(p0), f3(p1), r2);
      if (t >= t0 && t < t1 && (t < bt || (t == bt && id < bid)) &&
          clip_keeps(A, R.o + t * R.d, p0, p1, id)) {
        bt = t;
        bid = id;
      }
    }
    if (bid != 0xffffffffu) {
      shade(A, R, bid, bt);
      return true;
    }
    return false;
  } else {
    unsigned long long last = 0ull;
    bool more = true;
    while (more) {
      unsigned long long key[K];
#pragma unroll
      for (int q = 0; q < K; ++q) key[q] = ~0ull;
      uint32_t nacc = 0;
      for (uint32_t s = beg; s < end; ++s) {
        const uint32_t id = __ldg(&A.g.lists[s]);
        if (id + 1 >= A.n_vert) { set_err(A.g.st, kErrBounds); continue; }
        const float4 p0 = __ldg(&A.pos[id]), p1 = __ldg(&A.pos[id + 1]);
        const float t = capsule_entry(R.o, R.d, f3(p0), f3(p1), r2);
        if (!(t >= t0 && t < t1)) continue;
        const unsigned long long k = ((unsigned long long)__float_as_uint(t) << 32) | id;
        if (k <= last) continue;
        if (!clip_keeps(A, R.o + t * R.d, p0, p1, id)) continue;
        ++nacc;
        if (k < key[K - 1]) {
          key[K - 1] = k;
#pragma unroll
          for (int q = K - 1; q > 0; --q) {
            const unsigned long long lo = min(key[q - 1], key[q]), hi = max(key[q - 1], key[q]);
            key[q - 1] = lo;
            key[q] = hi;
          }
        }
      }
      const uint32_t m = min(nacc, (uint32_t)K);
#pragma unroll
      for (int q = 0; q < K; ++q) {
        if ((uint32_t)q < m && R.T >= kTStop) {
          shade(A, R, (uint32_t)(key[q] & 0xffffffffu), __uint_as_float((uint32_t)(key[q] >> 32)));
          last = key[q];
        }
      }
      if (R.T < kTStop) return true;
      more = nacc > (uint32_t)K;
    }
    return false;
  }
}

template <int K>
__device__ void trace_pixel(const TraceArgs& A, int px, int py, uint32_t pix) {
  const CamDev& c = A.cam;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  RayState R;
  if (c.ortho) {
    R.o = c.o0 + fx * c.ox + fy * c.oy;
    R.d = c.d0;
  } else {
    R.o = c.o0;
    const float3 d = c.d0 + fx * c.dx + fy * c.dy;
    R.d = (1.0f / sqrtf(dot3(d, d))) * d;
  }
  R.C[0] = R.C[1] = R.C[2] = 0.0f;
  R.T = 1.0f;
  R.first_id = -1;
  R.first_t = __int_as_float(0x7f800000);

  const int n = A.g.n;
  const float N = (float)n;
  float inv[3], og[3], dg[3];
  int step[3];
  float t0 = 0.0f, t1 = __int_as_float(0x7f800000);
  bool miss = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    og[k] = cmp3(R.o, k);
    dg[k] = cmp3(R.d, k);
    step[k] = dg[k] > 0.0f ? 1 : (dg[k] < 0.0f ? -1 : 0);
    if (dg[k] != 0.0f) {
      inv[k] = 1.0f / dg[k];
      float ta = (0.0f - og[k]) * inv[k], tb = (N - og[k]) * inv[k];
      if (ta > tb) { const float q = ta; ta = tb; tb = q; }
      t0 = fmaxf(t0, ta);
      t1 = fminf(t1, tb);
    } else {
      inv[k] = 0.0f;
      if (og[k] < 0.0f || og[k] > N) miss = true;
    }
  }
  bool missed = false;
  uint32_t n_queued = 0;
  if (!miss && t0 <= t1) {
    int v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = min(n - 1, max(0, (int)floorf(fmaf(t0, dg[k], og[k]))));
    float tcur = t0;
    const int max_steps = 3 * n + 16;
    for (int it = 0; it < max_steps; ++it) {
      const uint32_t bidx = ((uint32_t)(v[2] >> 2) << (2 * A.g.log2nb)) |
                            ((uint32_t)(v[1] >> 2) << A.g.log2nb) | (uint32_t)(v[0] >> 2);
      if (!bit_at(A.g.occb, bidx)) {
        // cross the whole empty brick
        float tb = __int_as_float(0x7f800000);
        int kb = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (step[k] == 0) continue;
          const int b0 = v[k] & ~3;
          const float tk = ((float)(step[k] > 0 ? b0 + 4 : b0) - og[k]) * inv[k];
          if (tk < tb) { tb = tk; kb = k; }
        }
        if (tb > t1) break;
        int nv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int b0 = v[k] & ~3;
          if (k == kb) nv[k] = step[k] > 0 ? b0 + 4 : b0 - 1;
          else nv[k] = min(b0 + 3, max(b0, (int)floorf(fmaf(tb, dg[k], og[k]))));
        }
        if (nv[kb] < 0 || nv[kb] >= n) break;
        v[0] = nv[0]; v[1] = nv[1]; v[2] = nv[2];
        tcur = fmaxf(tcur, tb);
        continue;
      }
      float texit = __int_as_float(0x7f800000);
      int ke = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (step[k] == 0) continue;
        const float tk = ((float)(step[k] > 0 ? v[k] + 1 : v[k]) - og[k]) * inv[k];
        if (tk < texit) { texit = tk; ke = k; }
      }
      const uint32_t idx = brick_index(v[0], v[1], v[2], A.g.log2nb);
      const uint32_t cnt = __ldg(&A.g.word[idx]) & 0xffffu;
      if (cnt) {
        if (!bit_at(A.g.vis, idx)) {
          // Culled voxel on the ray: queue it and keep going as if it were
          // empty. Its hits could only end the ray sooner, so every culled
          // voxel the ray truly needs lies before the point where this
          // optimistic march ends and gets queued now; one repair round lists
          // them all and the pixel is traced again.
          const uint32_t bm = 1u << (idx & 31);
          const uint32_t old = atomicOr(&A.need[idx >> 5], bm);
          if (!(old & bm)) {
            const uint32_t q = atomicAdd(A.vq_cnt, 1u);
            if (q < A.vq_cap) A.vq[q] = idx;
            else set_err(A.g.st, kErrOverflow);
          }
          missed = true;
          if (++n_queued >= A.max_queue) break;
          tcur = texit;
          if (tcur > t1) break;
          v[ke] += step[ke];
          if (v[ke] < 0 || v[ke] >= n) break;
          continue;
        }
        // a list past the capacity (reported as overflow) is read only up to it
        const uint32_t end0 = __ldg(&A.g.cur[idx]);
        const uint32_t end = (unsigned long long)end0 > A.g.list_cap ? (uint32_t)A.g.list_cap : end0;
        const uint32_t beg = end0 - cnt < end ? end0 - cnt : end;
        if (end0 < cnt) { set_err(A.g.st, kErrBounds); break; }
        if (process_voxel<K>(A, R, beg, end, tcur, texit)) break;
      }
      tcur = texit;
      if (tcur > t1) break;
      v[ke] += step[ke];
      if (v[ke] < 0 || v[ke] >= n) break;
    }
  }
  if (missed) {
    const uint32_t q = atomicAdd(A.pq_cnt, 1u);
    if (q < A.pq_cap) A.pq[q] = pix;
    else set_err(A.g.st, kErrOverflow);
    return;
  }
  A.rgba[pix] = make_float4(R.C[0], R.C[1], R.C[2], 1.0f - R.T);
  if (A.first_id) A.first_id[pix] = R.first_id;
  if (A.first_t) A.first_t[pix] = R.first_t;
}

template <int K>
__global__ void __launch_bounds__(128) k_trace(TraceArgs A) {
  if (A.pix_list) {
    const uint32_t cnt = min(*A.pix_count, A.pq_cap);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
      const uint32_t pix = A.pix_list[q];
      trace_pixel<K>(A, (int)(pix % (uint32_t)A.cam.width), (int)(pix / (uint32_t)A.cam.width), pix);
    }
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int px = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
  const int py = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
  if (px >= A.cam.width || py >= A.cam.height) return;
  trace_pixel<K>(A, px, py, (uint32_t)(py * A.cam.width + px));
}

int launch_trace(const TraceArgs& a, int K, cudaStream_t s) {
  dim3 grid, block(128);
  if (a.pix_list) {
    grid = dim3(152 * 4);  // grid-stride over the queued pixels; cheap when none
  } else {
    grid = dim3((a.cam.width + 15) / 16, (a.cam.height + 7) / 8);
  }
  switch (K) {
    case 1: k_trace<1><<<grid, block, 0, s>>>(a); break;
    case 8: k_trace<8><<<grid, block, 0, s>>>(a); break;
    case 16: k_trace<16><<<grid, block, 0, s>>>(a); break;
    default: k_trace<32><<<grid, block, 0, s>>>(a); break;
  }
  return 1;
}

// ----------------------------------------------------------------- repair
__global__ void k_repair_alloc(GridDev g, uint32_t* needb, const uint32_t* vq, const uint32_t* vq_cnt,
                               uint32_t vq_cap) {
  const uint32_t nq = min(*vq_cnt, vq_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && nq) {
    atomicAdd(&g.st->repair_rounds, 1u);
    atomicAdd(&g.st->repaired_voxels, nq);
  }
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint32_t idx = vq[q];
    const uint32_t cnt = g.word[idx] & 0xffffu;
    const uint32_t start = atomicAdd(&g.st->list_tail, cnt);
    if ((unsigned long long)start + cnt > g.list_cap) set_err(g.st, kErrOverflow);
    g.cur[idx] = start;
    atomicOr(&g.vis[idx >> 5], 1u << (idx & 31));
    const uint32_t b = idx >> 6;
    atomicOr(&g.visb[b >> 5], 1u << (b & 31));
    atomicOr(&needb[b >> 5], 1u << (b & 31));
  }
}

__global__ void k_repair_clear(GridDev g, uint32_t* need, const uint32_t* vq, const uint32_t* vq_cnt,
                               uint32_t vq_cap, int next) {
  const uint32_t nq = min(*vq_cnt, vq_cap);
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint32_t idx = vq[q];
    atomicAnd(&need[idx >> 5], ~(1u << (idx & 31)));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g.st->vq_cnt[next] = 0;
    g.st->pq_cnt[next] = 0;
  }
}

int launch_repair_alloc(const GridDev& g, uint32_t* needb, const uint32_t* vq,
                         const uint32_t* vq_cnt, uint32_t vq_cap, cudaStream_t s) {
  k_repair_alloc<<<152, 256, 0, s>>>(g, needb, vq, vq_cnt, vq_cap);
  return 1;
}

int launch_repair_clear(const GridDev& g, uint32_t* need, const uint32_t* vq,
                         const uint32_t* vq_cnt, uint32_t vq_cap, int next, cudaStream_t s) {
  k_repair_clear<<<152, 256, 0, s>>>(g, need, vq, vq_cnt, vq_cap, next);
  return 1;
}

}  // namespace vrt
