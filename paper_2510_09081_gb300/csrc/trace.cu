// A6: voxel ray tracing (Sec. 3.5).
//
// One ray per pixel; a warp owns a pixel tile, 4 wide and 8 tall for
// transparent rays, 8 by 4 for opaque ones (in the repair re-trace, 32 queued
// pixels). Each lane steps its own ray by 3D-DDA (Amanatides & Woo)
// through the grid box until it reaches a voxel with a list; in a brick with
// no occupied voxel it crosses, in one step, the whole cube of empty bricks
// that the distance field built after pass 1 guarantees around it. The warp then
// numbers the entries of all its lanes' pending lists one after another and
// takes them 32 at a time, one (ray, entry) pair per lane, so no lane idles on
// another lane's longer list. Very long lists, and a transparent ray with more
// hits in one voxel than its shared-memory slots hold, go to a whole-warp path
// that processes one voxel at a time (lane l takes entries l, l+32, ...).
//
// For each listed segment the lane computes the first entry of the ray into
// the segment's capsule; an entry counts only if it lies in the voxel's ray
// interval [t_enter, t_exit) -- the intervals partition the ray, so each hit
// is counted once and hits come out voxel by voxel in depth order -- and both
// clip planes keep it. A cheap line-to-line distance test skips segments whose
// line passes farther than r from the ray.
//  - opaque: the minimum 64-bit key (depth bits << 32 | segment id) is the
//    voxel's nearest hit; the ray stops at the first voxel that has one.
//  - transparent, shared entries: a ray's hits in the voxel are collected in
//    shared memory, sorted by key and composited by the ray's lane.
//  - transparent, whole-warp path: each lane keeps its 4 smallest keys beyond the last
//    composited one; the warp extracts keys in global (depth, id) order by
//    repeated minimum reductions -- only up to the smallest key a lane had to
//    drop, beyond which it rescans the list -- shades up to 32 of them in
//    parallel (one per lane), and accumulates them in key order,
//    C += T alpha c, T *= 1 - alpha, until T < 1e-4 (ground-truth order).
// Shading: colour = |unit tangent| per component times either cone-traced
// ambient occlusion per hit when enabled (six cones over the occupancy
// pyramid; a cone's occlusion is 1 - prod(1 - s_k) over its samples, so the
// samples of one hit can be taken by different lanes), or one trilinear sample
// of the voxel-space shading field at the hit (Sec. 3.4, built by shade.cu).
//
// Culling validation: a ray that reaches a voxel holding segments but no list
// queues the voxel (deduplicated by a bitmap), marches on as if the voxel were
// empty -- until it has queued max_queue voxels -- and finally queues its pixel
// instead of writing it; the repair round lists the queued voxels and traces
// the pixel again, so the image never depends on the culling heuristic. With
// no limit, the march queues every culled voxel before the point where it
// ends; the voxels' hits could only end the ray sooner, so the next trace
// of that pixel needs nothing more.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "launch.h"
#include "pyramid.cuh"

namespace vrt {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kLaneKeys = 4;              // transparent, shared list: keys kept per lane per scan
// kRayKeys (vrt_internal.cuh): hit slots per transparent ray on the shared-entry
// path, 32 KB of shared memory per block; A.ray_keys <= kRayKeys of them are used.
// 40 slots (40 KB) left the 4 resident blocks of an SM so little L1 that the
// trace of a sparse 512^3 set at 4K ran 5% slower; 24 slots sent too many rays
// to the whole-warp path (bundles trace 2.5% slower).
constexpr int kTraceThreads = 128;
constexpr int kStepRound = 1;             // tile trace: DDA steps a walking lane takes per round

__device__ __forceinline__ bool bit_at(const uint32_t* bits, uint32_t i) {
  return (bits[i >> 5] >> (i & 31)) & 1u;
}

// Instrumented trace: mark element i of a touch bitmap.
__device__ __forceinline__ void touch(uint32_t* bits, uint32_t i) {
  if (bits) atomicOr(&bits[i >> 5], 1u << (i & 31));
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(FULL, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__device__ __forceinline__ float3 shfl3(float3 v, int src) {
  return make_float3(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src),
                     __shfl_sync(FULL, v.z, src));
}

// The voxel-space shading field at P: trilinear over voxel centres, texel
// coordinates clamped to the grid. A hit accepted in voxel v reads only v and
// its neighbours, all of which the shading pass computed.
__device__ __forceinline__ float shade_at(const TraceArgs& A, float3 P) {
  const int n1 = A.g.n - 1;
  const float ux = P.x - 0.5f, uy = P.y - 0.5f, uz = P.z - 0.5f;
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
        const int xi = min(max(x + dx, 0), n1), yi = min(max(y + dy, 0), n1), zi = min(max(z + dz, 0), n1);
        acc = fmaf(w, __ldg(&A.shade[brick_index(xi, yi, zi, A.g.log2nb)]), acc);
      }
  return acc;
}

// Per-hit shading factor: A.ao = 1 cone AO at P, 2 the voxel-space field.
__device__ __noinline__ float hit_shade(const TraceArgs& A, float3 P) {
  return A.ao == 2 ? shade_at(A, P) : ao_lane(A, P);
}

__device__ __forceinline__ float3 tangent_colour(const TraceArgs& A, uint32_t id) {
  const float3 a = f3(__ldg(&A.pos[id])), b = f3(__ldg(&A.pos[id + 1]));
  const float3 dv = b - a;
  const float l2 = dot3(dv, dv);
  if (!(l2 > 0.0f)) return make_float3(1.0f, 1.0f, 1.0f);
  const float il = rsqrtf(l2);  // the hardware's approximate reciprocal square root
  return make_float3(fabsf(dv.x) * il, fabsf(dv.y) * il, fabsf(dv.z) * il);
}

// Sort key of an accepted hit at depth t of segment id, entry li of the voxel's
// list, the voxel's ray interval being [t0, t1). Default: the depth's fp32 bits
// above the id (depth order, ties by id). With A.key16 the paper's per-voxel
// key (Sec. 3.5): the depth within the voxel quantized to 16 bits above the
// 16-bit list index -- hits of equal quantized depth then follow the list's
// order -- with the id below it, for shading.
template <bool KEY16>
__device__ __forceinline__ unsigned long long hit_key(float t, uint32_t id, uint32_t li, float t0,
                                                      float t1) {
  if (!KEY16) return ((unsigned long long)__float_as_uint(t) << 32) | id;
  const float u = __fdividef(t - t0, t1 - t0);
  const uint32_t q = min(65535u, (uint32_t)fmaxf(0.0f, u * 65536.0f));
  return ((unsigned long long)((q << 16) | (li & 0xffffu)) << 32) | id;
}

// Depth of the hit a key names: stored in the default key; recomputed from the
// segment with the 16+16 key, which keeps only its quantized position.
template <bool KEY16>
__device__ __forceinline__ float hit_depth(const TraceArgs& A, unsigned long long k, float3 o,
                                           float3 d) {
  if (!KEY16) return __uint_as_float((uint32_t)(k >> 32));
  const uint32_t id = (uint32_t)(k & 0xffffffffu);
  const float4 p0 = __ldg(&A.pos[id]), p1 = __ldg(&A.pos[id + 1]);
  return capsule_entry(o, d, f3(p0), f3(p1), A.g.r * A.g.r);
}

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

// Key of list entry s for ray (o, d) over [t0, t1): depth bits << 32 | id, or
// ~0 when the segment gives no accepted hit there.
template <bool COUNT, bool KEY16>
__device__ __forceinline__ unsigned long long entry_key(const TraceArgs& A, uint32_t s, uint32_t beg,
                                                        float3 o, float3 d, float t0, float t1,
                                                        float r2, float rrm, unsigned& n_cap) {
  const uint32_t id = __ldg(&A.g.lists[s]);
  if (id + 1 >= A.n_vert) {
    set_err(A.g.st, kErrBounds);
    return ~0ull;
  }
  if (COUNT) {
    touch(A.touch_list, s);
    touch(A.touch_vert, id);
    touch(A.touch_vert, id + 1);
  }
  const float4 p0 = __ldg(&A.pos[id]), p1 = __ldg(&A.pos[id + 1]);
  if (!lines_may_meet(o, d, f3(p0), f3(p1), rrm)) return ~0ull;
  if (COUNT) ++n_cap;
  const float t = capsule_entry(o, d, f3(p0), f3(p1), r2);
  if (!(t >= t0 && t < t1)) return ~0ull;
  if (!clip_keeps(A, o + t * d, p0, p1, id)) return ~0ull;
  return hit_key<KEY16>(t, id, s - beg, t0, t1);
}

// Per-lane ray state. Components are kept as scalars (no runtime-indexed
// arrays) so the DDA state stays in registers.
struct Ray {
  float3 o, d, inv, ooi;  // ooi = o * inv: the boundary b is crossed at b * inv - ooi
  int sx, sy, sz;      // step direction per axis (-1, 0, 1)
  int vx, vy, vz;      // current voxel
  float tcur, t1;
  float C[3], T;
  int first_id;
  float first_t;
  uint32_t pix, n_queued;
  bool active, pending, missed;
  uint32_t beg, end;   // pending voxel's list
  float vt0, vt1;      // pending voxel's ray interval
  unsigned n_steps, n_entries, n_cap, n_vox;  // work counters
  unsigned n_hits, n_ww_vox, n_ww_ent;
  unsigned long long cyc[4];  // warp cycles: DDA, shared-entry path, whole-warp path, capsule stage
};

// Parameter where the ray leaves coordinate range [lo, hi] along an axis
// (the side it moves toward); +inf when it does not move on that axis.
__device__ __forceinline__ float exit_t(int s, int lo, int hi, float ooi, float inv) {
  return s != 0 ? fmaf((float)(s > 0 ? hi : lo), inv, -ooi) : __int_as_float(0x7f800000);
}

// Step the lane's ray toward its next voxel that has a list, at most `budget`
// steps: 1 when it reached one (pending), 0 when the ray leaves the grid (or
// queues too many culled voxels), -1 when the budget ran out first. Every step
// moves the ray forward through the grid, so its walk ends.
template <bool COUNT>
__device__ int advance(const TraceArgs& A, Ray& R, int budget) {
  const int n = A.g.n;
  for (int it = 0; it < budget; ++it) {
    if (R.tcur > R.t1) return 0;
    if (COUNT) ++R.n_steps;
    const uint32_t bidx = ((uint32_t)(R.vz >> 2) << (2 * A.g.log2nb)) |
                          ((uint32_t)(R.vy >> 2) << A.g.log2nb) | (uint32_t)(R.vx >> 2);
    const uint32_t idx = brick_index(R.vx, R.vy, R.vz, A.g.log2nb);
    // the step's loads are independent: issue them together (one latency, not
    // up to three in sequence); the word and the list end -- at or above
    // kCulledStart when the cull gave the voxel no list -- go unused in an
    // empty brick
    const int kd = __ldg(&A.g.bdist[bidx]);
    const uint32_t wv = __ldg(&A.g.word[idx]);
    const uint32_t cv = __ldg(&A.g.cur[idx]);
    if (kd > 0) {
      // cross the cube of empty bricks within kd - 1 of this one: low corner
      // (bx, by, bz), side w voxels
      const int ext = 4 * (kd - 1), w = 4 + 2 * ext;
      const int bx = (R.vx & ~3) - ext, by = (R.vy & ~3) - ext, bz = (R.vz & ~3) - ext;
      const float tx = exit_t(R.sx, bx, bx + w, R.ooi.x, R.inv.x);
      const float ty = exit_t(R.sy, by, by + w, R.ooi.y, R.inv.y);
      const float tz = exit_t(R.sz, bz, bz + w, R.ooi.z, R.inv.z);
      const float tb = fminf(tx, fminf(ty, tz));
      if (tb > R.t1) return 0;
      const int cx = min(min(bx + w, n) - 1, max(max(bx, 0), (int)floorf(fmaf(tb, R.d.x, R.o.x))));
      const int cy = min(min(by + w, n) - 1, max(max(by, 0), (int)floorf(fmaf(tb, R.d.y, R.o.y))));
      const int cz = min(min(bz + w, n) - 1, max(max(bz, 0), (int)floorf(fmaf(tb, R.d.z, R.o.z))));
      if (tb == tx) {
        R.vx = R.sx > 0 ? bx + w : bx - 1; R.vy = cy; R.vz = cz;
        if (R.vx < 0 || R.vx >= n) return 0;
      } else if (tb == ty) {
        R.vy = R.sy > 0 ? by + w : by - 1; R.vx = cx; R.vz = cz;
        if (R.vy < 0 || R.vy >= n) return 0;
      } else {
        R.vz = R.sz > 0 ? bz + w : bz - 1; R.vx = cx; R.vy = cy;
        if (R.vz < 0 || R.vz >= n) return 0;
      }
      R.tcur = fmaxf(R.tcur, tb);
      continue;
    }
    const float tx = exit_t(R.sx, R.vx, R.vx + 1, R.ooi.x, R.inv.x);
    const float ty = exit_t(R.sy, R.vy, R.vy + 1, R.ooi.y, R.inv.y);
    const float tz = exit_t(R.sz, R.vz, R.vz + 1, R.ooi.z, R.inv.z);
    const float texit = fminf(tx, fminf(ty, tz));
    const uint32_t cnt = wv & 0xffffu;
    if (COUNT) touch(A.touch_vox, idx);
    const float tin = R.tcur;
    // step past this voxel before returning, so the next call resumes after it
    R.tcur = texit;
    bool inside;
    if (texit == tx) {
      R.vx += R.sx;
      inside = R.vx >= 0 && R.vx < n;
    } else if (texit == ty) {
      R.vy += R.sy;
      inside = R.vy >= 0 && R.vy < n;
    } else {
      R.vz += R.sz;
      inside = R.vz >= 0 && R.vz < n;
    }
    if (cnt) {
      if (cv >= kCulledStart) {  // the cull gave it no list
        // culled voxel on the ray: queue it, march on as if it were empty; at
        // the first one, keep the ray's state for the re-trace to resume from
        if (R.n_queued == 0 && A.resume) {
          A.resume[2 * R.pix] = make_float4(R.C[0], R.C[1], R.C[2], R.T);
          A.resume[2 * R.pix + 1] = make_float4(__int_as_float(R.first_id), R.first_t,
                                                __uint_as_float(idx), tin);
        }
        const uint32_t bm = 1u << (idx & 31);
        const uint32_t old = atomicOr(&A.need[idx >> 5], bm);
        if (!(old & bm)) {
          const uint32_t q = atomicAdd(A.vq_cnt, 1u);
          if (q < A.vq_cap) A.vq[q] = idx;
          else set_err(A.g.st, kErrOverflow);
        }
        R.missed = true;
        if (++R.n_queued >= A.max_queue) return 0;
      } else {
        // a list past the capacity (reported as overflow) is read only up to it
        const uint32_t end0 = cv;
        if (end0 < cnt) {
          set_err(A.g.st, kErrBounds);
          return 0;
        }
        const uint32_t end = (unsigned long long)end0 > A.g.list_cap ? (uint32_t)A.g.list_cap : end0;
        R.beg = end0 - cnt < end ? end0 - cnt : end;
        R.end = end;
        R.vt0 = tin;
        R.vt1 = texit;
        if (!inside) R.t1 = -1.0f;  // this was the last voxel; stop after it
        return 1;
      }
    }
    if (!inside) return 0;
  }
  return -1;  // budget used up, ray still on its way
}

__device__ void init_ray(const TraceArgs& A, Ray& R, int px, int py, bool valid) {
  const CamDev& c = A.cam;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
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
  R.n_queued = 0;
  R.n_steps = R.n_entries = R.n_cap = R.n_vox = 0;
  R.n_hits = R.n_ww_vox = R.n_ww_ent = 0;
  R.missed = false;
  R.pending = false;
  const float N = (float)A.g.n;
  float t0 = 0.0f, t1 = __int_as_float(0x7f800000);
  bool miss = !valid;
  auto axis = [&](float o, float d, int& s, float& inv) {
    s = d > 0.0f ? 1 : (d < 0.0f ? -1 : 0);
    if (d != 0.0f) {
      inv = 1.0f / d;
      float ta = (0.0f - o) * inv, tb = (N - o) * inv;
      if (ta > tb) { const float q = ta; ta = tb; tb = q; }
      t0 = fmaxf(t0, ta);
      t1 = fminf(t1, tb);
    } else {
      inv = 0.0f;
      if (o < 0.0f || o > N) miss = true;
    }
  };
  axis(R.o.x, R.d.x, R.sx, R.inv.x);
  axis(R.o.y, R.d.y, R.sy, R.inv.y);
  axis(R.o.z, R.d.z, R.sz, R.inv.z);
  R.ooi = make_float3(R.o.x * R.inv.x, R.o.y * R.inv.y, R.o.z * R.inv.z);
  R.active = !miss && t0 <= t1;
  R.tcur = t0;
  R.t1 = t1;
  const int n = A.g.n;
  R.vx = min(n - 1, max(0, (int)floorf(fmaf(t0, R.d.x, R.o.x))));
  R.vy = min(n - 1, max(0, (int)floorf(fmaf(t0, R.d.y, R.o.y))));
  R.vz = min(n - 1, max(0, (int)floorf(fmaf(t0, R.d.z, R.o.z))));
}

// A re-traced ray continues from the state it had when it first met a culled
// voxel (now listed): same colour, transmittance and first hit, at that voxel
// and its entry parameter, so the result equals a trace from the start.
__device__ void resume_ray(const TraceArgs& A, Ray& R) {
  const float4 s0 = A.resume[2 * R.pix], s1 = A.resume[2 * R.pix + 1];
  R.C[0] = s0.x; R.C[1] = s0.y; R.C[2] = s0.z;
  R.T = s0.w;
  R.first_id = __float_as_int(s1.x);
  R.first_t = s1.y;
  int x, y, z;
  brick_coords(__float_as_uint(s1.z), A.g.log2nb, x, y, z);
  R.vx = min(A.g.n - 1, max(0, x));
  R.vy = min(A.g.n - 1, max(0, y));
  R.vz = min(A.g.n - 1, max(0, z));
  R.tcur = s1.w;
}

// The warp processes the pending voxel of lane `L`.
template <bool OPAQUE, bool COUNT, bool KEY16>
__device__ void process_voxel(const TraceArgs& A, Ray& R, int L) {
  const int lane = threadIdx.x & 31;
  const float3 o = shfl3(R.o, L), d = shfl3(R.d, L);
  const uint32_t beg = __shfl_sync(FULL, R.beg, L), end = __shfl_sync(FULL, R.end, L);
  const float t0 = __shfl_sync(FULL, R.vt0, L), t1 = __shfl_sync(FULL, R.vt1, L);
  const float r2 = A.g.r * A.g.r;
  const float rrm = (A.g.r + 1e-3f) * (A.g.r + 1e-3f);
  unsigned n_cap = 0, n_hit = 0;
  if (COUNT && lane == L) {
    ++R.n_vox;
    R.n_entries += end - beg;
    ++R.n_ww_vox;
  }
  if (OPAQUE) {
    unsigned long long best = ~0ull;
    for (uint32_t s = beg + lane; s < end; s += 32) {
      const unsigned long long k = entry_key<COUNT, KEY16>(A, s, beg, o, d, t0, t1, r2, rrm, n_cap);
      if (COUNT && k != ~0ull) ++n_hit;
      best = k < best ? k : best;
    }
    if (COUNT) {
      R.n_hits += n_hit;
      if (lane == L) R.n_ww_ent += end - beg;
    }
    if (COUNT) R.n_cap += n_cap;
    best = warp_min_u64(best);
    if (best != ~0ull) {
      const uint32_t id = (uint32_t)(best & 0xffffffffu);
      const float t = hit_depth<KEY16>(A, best, o, d);
      float3 c = tangent_colour(A, id);
      if (A.ao) c = (A.ao == 2 ? shade_at(A, o + t * d) : ao_warp(A, o + t * d)) * c;
      if (lane == L) {
        R.C[0] = A.alpha * c.x; R.C[1] = A.alpha * c.y; R.C[2] = A.alpha * c.z;
        R.T *= (1.0f - A.alpha);
        R.first_id = (int)id;
        R.first_t = t;
        R.active = false;
      }
    }
    return;
  }
  // transparent
  float T = __shfl_sync(FULL, R.T, L);
  float C0 = __shfl_sync(FULL, R.C[0], L), C1 = __shfl_sync(FULL, R.C[1], L),
        C2 = __shfl_sync(FULL, R.C[2], L);
  int fid = __shfl_sync(FULL, R.first_id, L);
  float ft = __shfl_sync(FULL, R.first_t, L);
  const float om = 1.0f - A.alpha;
  unsigned long long last = 0ull;  // keys <= last are composited
  bool rescan = true;
  while (rescan && T >= kTStop) {
    unsigned long long buf[kLaneKeys];
#pragma unroll
    for (int q = 0; q < kLaneKeys; ++q) buf[q] = ~0ull;
    bool dropped = false;
    if (COUNT && lane == L) R.n_ww_ent += end - beg;
    for (uint32_t s = beg + lane; s < end; s += 32) {
      const unsigned long long k = entry_key<COUNT, KEY16>(A, s, beg, o, d, t0, t1, r2, rrm, n_cap);
      if (COUNT && k != ~0ull) ++n_hit;
      if (k == ~0ull || k <= last) continue;
      if (k < buf[kLaneKeys - 1]) {
        if (buf[kLaneKeys - 1] != ~0ull) dropped = true;
        buf[kLaneKeys - 1] = k;
#pragma unroll
        for (int q = kLaneKeys - 1; q > 0; --q) {
          const unsigned long long lo = buf[q - 1] < buf[q] ? buf[q - 1] : buf[q];
          const unsigned long long hi = buf[q - 1] < buf[q] ? buf[q] : buf[q - 1];
          buf[q - 1] = lo;
          buf[q] = hi;
        }
      } else {
        dropped = true;
      }
    }
    // keys up to `lim` are complete: a lane that dropped keys kept its smallest
    const unsigned long long lim = warp_min_u64(dropped ? buf[kLaneKeys - 1] : ~0ull);
    rescan = lim != ~0ull;
    bool more = true;
    while (more && T >= kTStop) {
      // extract up to 32 keys in order; lane q receives the q-th
      unsigned long long mine = ~0ull;
      int n_out = 0;
      for (; n_out < 32; ++n_out) {
        const unsigned long long m = warp_min_u64(buf[0]);
        if (m == ~0ull || m > lim) break;
        if (buf[0] == m) {
#pragma unroll
          for (int q = 0; q < kLaneKeys - 1; ++q) buf[q] = buf[q + 1];
          buf[kLaneKeys - 1] = ~0ull;
        }
        if (lane == n_out) mine = m;
      }
      more = n_out == 32;
      if (n_out == 0) break;
      // shade in parallel
      float3 c = make_float3(0.f, 0.f, 0.f);
      float tq = 0.0f;
      if (lane < n_out) {
        const uint32_t id = (uint32_t)(mine & 0xffffffffu);
        tq = hit_depth<KEY16>(A, mine, o, d);
        c = tangent_colour(A, id);
        if (A.ao) c = hit_shade(A, o + tq * d) * c;
      }
      // accumulate in key order
      for (int q = 0; q < n_out; ++q) {
        const float3 cq = shfl3(c, q);
        const unsigned long long kq = __shfl_sync(FULL, mine, q);
        const float tqq = KEY16 ? __shfl_sync(FULL, tq, q) : 0.0f;
        if (T < kTStop) break;
        const float w = T * A.alpha;
        C0 = fmaf(w, cq.x, C0);
        C1 = fmaf(w, cq.y, C1);
        C2 = fmaf(w, cq.z, C2);
        T *= om;
        if (fid < 0) {
          fid = (int)(kq & 0xffffffffu);
          ft = KEY16 ? tqq : __uint_as_float((uint32_t)(kq >> 32));
        }
        last = kq;
      }
    }
    // a rescan is needed only when the extraction stopped at the drop limit
    rescan = rescan && T >= kTStop && last == lim;
  }
  if (COUNT) {
    R.n_cap += n_cap;
    R.n_hits += n_hit;
  }
  if (lane == L) {
    R.T = T;
    R.C[0] = C0; R.C[1] = C1; R.C[2] = C2;
    R.first_id = fid;
    R.first_t = ft;
    if (T < kTStop) R.active = false;
  }
}

// The pending voxels of the warp's lanes with lists up to A.short_list
// entries, processed together. Lanes whose rays wait in the same voxel form a
// group (neighbouring rays of the tile usually do); the entries of the
// groups' distinct lists are numbered one after another and the warp takes 32
// at a time, one entry per lane (two such rounds per step), so short lists do
// not wait for the longest one. A lane loads its entry (segment id and end
// points) once and line-tests it against every ray of the entry's group in
// turn. Pairs that pass the line-distance test are queued per warp
// in shared memory and get the capsule test 32 at a time. A hit goes to its ray's slots in shared memory
// (the nearest key for an opaque ray; up to kRayKeys keys of a transparent
// ray, sorted and composited by the ray's own lane afterwards). A transparent
// ray with more hits in the voxel keeps its voxel pending for the whole-warp
// path, which starts it again from scratch.
template <bool OPAQUE, bool COUNT, bool KEY16>
__device__ void process_flat(const TraceArgs& A, Ray& R) {
  extern __shared__ unsigned long long s_key[];  // [kRayKeys][kTraceThreads]
  __shared__ float4 s_ray[2][kTraceThreads];      // (o, t_enter), (d, t_exit)
  __shared__ uint32_t s_cnt[kTraceThreads];
  __shared__ unsigned long long s_best[kTraceThreads];
  __shared__ uint2 s_q[kTraceThreads / 32][64];   // (segment id, owner lane) queued for the capsule test
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.x, wb = tid & ~31;
  const unsigned lt = (1u << lane) - 1u;
  const bool take = R.pending && R.end - R.beg <= A.short_list;
  const uint32_t len = take ? R.end - R.beg : 0u;
  // group of lanes waiting in the same voxel (same list start); its lowest
  // lane numbers the list's entries. Opaque rays mostly end in their first
  // listed voxel, so their groups are small: each ray is its own group there.
  unsigned gm = take ? 1u << lane : 0u;
  if (!OPAQUE) {
    const unsigned tm = __ballot_sync(FULL, take);
    gm = __match_any_sync(FULL, take ? R.beg : 0xffffffffu) & (take ? tm : 0u);
  }
  const uint32_t glen = (take && __ffs(gm) - 1 == lane) ? len : 0u;
  uint32_t incl = glen;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  const uint32_t total = __shfl_sync(FULL, incl, 31);
  if (total == 0) return;
  if (take) {
    s_ray[0][tid] = make_float4(R.o.x, R.o.y, R.o.z, R.vt0);
    s_ray[1][tid] = make_float4(R.d.x, R.d.y, R.d.z, R.vt1);
  }
  if (OPAQUE) s_best[tid] = ~0ull;
  else s_cnt[tid] = 0u;
  __syncwarp();
  const uint32_t first = R.beg - (incl - glen);  // entry g of a group's list is lists[first + g]
  const float r2 = A.g.r * A.g.r;
  const float rrm = (A.g.r + 1e-3f) * (A.g.r + 1e-3f);
  unsigned n_cap = 0, n_hit = 0;
  uint2* q = s_q[tid >> 5];
  uint32_t qn = 0;  // queued pairs (warp-uniform)
  // capsule test of queued pair `lane` for lanes below cnt
  auto capsule_stage = [&](uint32_t cnt) {
    const long long c0 = COUNT ? clock64() : 0;
    if ((uint32_t)lane < cnt) {
      const uint2 it = q[lane];
      const uint32_t id = it.x;
      const int j = (int)(it.y & 255u);
      const float4 p0 = __ldg(&A.pos[id]), p1 = __ldg(&A.pos[id + 1]);
      const float4 ro = s_ray[0][wb + j], rd = s_ray[1][wb + j];
      if (COUNT) ++n_cap;
      const float t = capsule_entry(f3(ro), f3(rd), f3(p0), f3(p1), r2);
      if (t >= ro.w && t < rd.w && clip_keeps(A, f3(ro) + t * f3(rd), p0, p1, id)) {
        const unsigned long long k = hit_key<KEY16>(t, id, it.y >> 8, ro.w, rd.w);
        if (COUNT) ++n_hit;
        if (OPAQUE) {
          atomicMin(&s_best[wb + j], k);
        } else {
          const uint32_t slot = atomicAdd(&s_cnt[wb + j], 1u);
          if (slot < A.ray_keys) s_key[slot * kTraceThreads + wb + j] = k;
        }
      }
    }
    if (COUNT) R.cyc[3] += (unsigned long long)(clock64() - c0);
  };
  auto owner = [&](uint32_t gq) {
    int j = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1)
      if (__shfl_sync(FULL, incl, j + st - 1) <= gq) j += st;
    return min(j, 31);
  };
  // queue entry: segment id, owner lane j | list index li << 8 (16+16 keys)
  auto append = [&](bool pass, uint32_t id, int j, uint32_t li) {
    const unsigned m = __ballot_sync(FULL, pass);
    if (pass) q[qn + __popc(m & lt)] = make_uint2(id, (uint32_t)j | (li << 8));
    qn += __popc(m);
    if (qn >= 32) {
      __syncwarp();
      capsule_stage(32);
      __syncwarp();
      if ((uint32_t)lane < qn - 32) q[lane] = q[32 + lane];
      __syncwarp();
      qn -= 32;
    }
  };
  // line tests of a loaded entry against the rays in mask m, one per round
  auto test_group = [&](unsigned m, uint32_t id, float4 p0, float4 p1, uint32_t li) {
    while (__any_sync(FULL, m)) {
      bool pass = false;
      int j = 0;
      if (m) {
        j = __ffs(m) - 1;
        m &= m - 1;
        const float4 ro = s_ray[0][wb + j], rd = s_ray[1][wb + j];
        pass = lines_may_meet(f3(ro), f3(rd), f3(p0), f3(p1), rrm);
      }
      append(pass, id, j, li);
    }
  };
  // two independent (owner search, list load, vertex loads) chains per step:
  // the loads' latency is paid once per entry, whatever its group's size
  if (OPAQUE) {
    for (uint32_t t0 = 0; t0 < total; t0 += 64) {
      const uint32_t ga = t0 + lane, gb = ga + 32;
      const int ja = owner(ga), jb = owner(gb);
      const uint32_t fa = __shfl_sync(FULL, first, ja), fb = __shfl_sync(FULL, first, jb);
      const bool va = ga < total, vb = gb < total;
      uint32_t ida = 0, idb = 0;
      if (va) ida = __ldg(&A.g.lists[fa + ga]);
      if (vb) idb = __ldg(&A.g.lists[fb + gb]);
      const bool oka = va && ida + 1 < A.n_vert, okb = vb && idb + 1 < A.n_vert;
      if ((va && !oka) || (vb && !okb)) set_err(A.g.st, kErrBounds);
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
      if (oka) { a0 = __ldg(&A.pos[ida]); a1 = __ldg(&A.pos[ida + 1]); }
      if (okb) { b0 = __ldg(&A.pos[idb]); b1 = __ldg(&A.pos[idb + 1]); }
      if (COUNT) {
        if (oka) { touch(A.touch_list, fa + ga); touch(A.touch_vert, ida); touch(A.touch_vert, ida + 1); }
        if (okb) { touch(A.touch_list, fb + gb); touch(A.touch_vert, idb); touch(A.touch_vert, idb + 1); }
      }
      bool pa = false, pb = false;
      if (oka) {
        const float4 ro = s_ray[0][wb + ja], rd = s_ray[1][wb + ja];
        pa = lines_may_meet(f3(ro), f3(rd), f3(a0), f3(a1), rrm);
      }
      if (okb) {
        const float4 ro = s_ray[0][wb + jb], rd = s_ray[1][wb + jb];
        pb = lines_may_meet(f3(ro), f3(rd), f3(b0), f3(b1), rrm);
      }
      uint32_t la = 0, lb = 0;  // list indices (16+16 keys)
      if (KEY16) {
        la = fa + ga - __shfl_sync(FULL, R.beg, ja);
        lb = fb + gb - __shfl_sync(FULL, R.beg, jb);
      }
      append(pa, ida, ja, la);
      append(pb, idb, jb, lb);
    }
  } else for (uint32_t t0 = 0; t0 < total; t0 += 64) {
    const uint32_t ga = t0 + lane, gb = ga + 32;
    const int ja = owner(ga), jb = owner(gb);
    const uint32_t fa = __shfl_sync(FULL, first, ja), fb = __shfl_sync(FULL, first, jb);
    const unsigned ma = __shfl_sync(FULL, gm, ja), mb = __shfl_sync(FULL, gm, jb);
    const bool va = ga < total, vb = gb < total;
    uint32_t ida = 0, idb = 0;
    if (va) ida = __ldg(&A.g.lists[fa + ga]);
    if (vb) idb = __ldg(&A.g.lists[fb + gb]);
    const bool oka = va && ida + 1 < A.n_vert, okb = vb && idb + 1 < A.n_vert;
    if ((va && !oka) || (vb && !okb)) set_err(A.g.st, kErrBounds);
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
    if (oka) { a0 = __ldg(&A.pos[ida]); a1 = __ldg(&A.pos[ida + 1]); }
    if (okb) { b0 = __ldg(&A.pos[idb]); b1 = __ldg(&A.pos[idb + 1]); }
    if (COUNT) {
      if (oka) { touch(A.touch_list, fa + ga); touch(A.touch_vert, ida); touch(A.touch_vert, ida + 1); }
      if (okb) { touch(A.touch_list, fb + gb); touch(A.touch_vert, idb); touch(A.touch_vert, idb + 1); }
    }
    uint32_t la = 0, lb = 0;  // list indices (16+16 keys)
    if (KEY16) {
      la = fa + ga - __shfl_sync(FULL, R.beg, ja);
      lb = fb + gb - __shfl_sync(FULL, R.beg, jb);
    }
    test_group(oka ? ma : 0u, ida, a0, a1, la);
    test_group(okb ? mb : 0u, idb, b0, b1, lb);
  }
  __syncwarp();
  capsule_stage(qn);
  __syncwarp();
  if (COUNT) {
    R.n_cap += n_cap;
    R.n_hits += n_hit;
  }
  if (!take) return;
  if (OPAQUE) {
    if (COUNT) {
      ++R.n_vox;
      R.n_entries += len;
    }
    const unsigned long long best = s_best[tid];
    if (best != ~0ull) {
      const uint32_t id = (uint32_t)(best & 0xffffffffu);
      const float t = hit_depth<KEY16>(A, best, R.o, R.d);
      float3 c = tangent_colour(A, id);
      if (A.ao) c = hit_shade(A, R.o + t * R.d) * c;
      R.C[0] = A.alpha * c.x; R.C[1] = A.alpha * c.y; R.C[2] = A.alpha * c.z;
      R.T *= (1.0f - A.alpha);
      R.first_id = (int)id;
      R.first_t = t;
      R.active = false;
    }
    R.pending = false;
    if (R.t1 < 0.0f) R.active = false;
    return;
  }
  const uint32_t nk = s_cnt[tid];
  if (nk > A.ray_keys) return;  // stays pending: the whole-warp path redoes it
  if (COUNT) {
    ++R.n_vox;
    R.n_entries += len;
  }
  unsigned long long* kb = s_key + tid;
  for (uint32_t q = 1; q < nk; ++q) {
    const unsigned long long k = kb[q * kTraceThreads];
    uint32_t p = q;
    while (p > 0 && kb[(p - 1) * kTraceThreads] > k) {
      kb[p * kTraceThreads] = kb[(p - 1) * kTraceThreads];
      --p;
    }
    kb[p * kTraceThreads] = k;
  }
  const float om = 1.0f - A.alpha;
  for (uint32_t q = 0; q < nk && R.T >= kTStop; ++q) {
    const unsigned long long kq = kb[q * kTraceThreads];
    const uint32_t id = (uint32_t)(kq & 0xffffffffu);
    const float t = hit_depth<KEY16>(A, kq, R.o, R.d);
    float3 c = tangent_colour(A, id);
    if (A.ao) c = hit_shade(A, R.o + t * R.d) * c;
    const float w = R.T * A.alpha;
    R.C[0] = fmaf(w, c.x, R.C[0]);
    R.C[1] = fmaf(w, c.y, R.C[1]);
    R.C[2] = fmaf(w, c.z, R.C[2]);
    R.T *= om;
    if (R.first_id < 0) {
      R.first_id = (int)id;
      R.first_t = t;
    }
  }
  R.pending = false;
  if (R.T < kTStop || R.t1 < 0.0f) R.active = false;
}

// Warp cycles since `t` into the counter `c` (instrumented trace only).
template <bool COUNT>
__device__ __forceinline__ void lap(unsigned long long& c, long long& t) {
  if (COUNT) {
    const long long now = clock64();
    c += (unsigned long long)(now - t);
    t = now;
  }
}

template <bool OPAQUE, bool COUNT, bool KEY16>
__device__ void trace_warp(const TraceArgs& A, Ray& R) {
  const int lane = threadIdx.x & 31;
  long long t = COUNT ? clock64() : 0;
  for (;;) {
    if (R.active && !R.pending) {
      const int rc = advance<COUNT>(A, R, kStepRound);
      R.pending = rc == 1;
      if (rc == 0) R.active = false;
    }
    // The warp steps its walking rays one voxel (or empty cube) per round and
    // processes the waiting lists once a quarter of the rays still in flight
    // wait at one (or none can step on). Stepping each ray to its next list in
    // one go left most lanes idle while the longest walk went on (5.9 of 32
    // lanes active per instruction on a sparse 512^3 set): bounded rounds cut
    // that trace by 41-47% and the dense bundles' by 4%.
    const unsigned pend = __ballot_sync(FULL, R.pending);
    const unsigned walk = __ballot_sync(FULL, R.active && !R.pending);
    if (!pend && !walk) break;
    if (walk && 4 * __popc(pend) < __popc(pend | walk)) continue;
    lap<COUNT>(R.cyc[0], t);
    process_flat<OPAQUE, COUNT, KEY16>(A, R);
    lap<COUNT>(R.cyc[1], t);
    // long lists: the whole warp on one list at a time
    unsigned pm = __ballot_sync(FULL, R.pending);
    while (pm) {
      const int L = __ffs(pm) - 1;
      pm &= pm - 1;
      process_voxel<OPAQUE, COUNT, KEY16>(A, R, L);
      if (lane == L) {
        R.pending = false;
        if (R.t1 < 0.0f) R.active = false;
      }
    }
    lap<COUNT>(R.cyc[2], t);
  }
  lap<COUNT>(R.cyc[0], t);
}

template <bool COUNT>
__device__ __forceinline__ void finish(const TraceArgs& A, const Ray& R, bool valid) {
  if (COUNT) {
    unsigned long long e = R.n_entries, c = R.n_cap, v = R.n_vox, st = R.n_steps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(FULL, e, o);
      c += __shfl_xor_sync(FULL, c, o);
      v += __shfl_xor_sync(FULL, v, o);
      st += __shfl_xor_sync(FULL, st, o);
    }
    unsigned long long h = R.n_hits, wv = R.n_ww_vox, we = R.n_ww_ent;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      h += __shfl_xor_sync(FULL, h, o);
      wv += __shfl_xor_sync(FULL, wv, o);
      we += __shfl_xor_sync(FULL, we, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&A.g.st->tr_entries, e);
      atomicAdd(&A.g.st->tr_capsule, c);
      atomicAdd(&A.g.st->tr_voxels, v);
      atomicAdd(&A.g.st->tr_steps, st);
      atomicAdd(&A.g.st->tr_hits, h);
      atomicAdd(&A.g.st->tr_ww_voxels, wv);
      atomicAdd(&A.g.st->tr_ww_entries, we);
      for (int k = 0; k < 4; ++k) atomicAdd(&A.g.st->tr_cycles[k], R.cyc[k]);
    }
  }
  if (!valid) return;
  if (R.missed) {
    const uint32_t q = atomicAdd(A.pq_cnt, 1u);
    if (q < A.pq_cap) A.pq[q] = R.pix;
    else set_err(A.g.st, kErrOverflow);
    return;
  }
  A.rgba[R.pix] = make_float4(R.C[0], R.C[1], R.C[2], 1.0f - R.T);
  if (A.first_id) A.first_id[R.pix] = R.first_id;
  if (A.first_t) A.first_t[R.pix] = R.first_t;
}

// Transparent main trace: each warp owns one fixed tile of 32 pixels, TW wide
// and 32 / TW tall (a block 2x2 tiles), and its lanes write their pixels
// together at the end. Measured faster than persistent refilling here, since
// the tile's rays share lists. The tile shape is a tuned parameter (default
// 4 x 8, measured slightly faster than 8 x 4 or 16 x 2 on the bundles frame).
template <bool OPAQUE, bool COUNT, bool KEY16, int TW>
__global__ void __launch_bounds__(kTraceThreads) k_trace_tile(TraceArgs A) {
  constexpr int TH = 32 / TW;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int px = blockIdx.x * (2 * TW) + (warp & 1) * TW + (lane % TW);
  const int py = blockIdx.y * (2 * TH) + (warp >> 1) * TH + (lane / TW);
  const bool valid = px < A.cam.width && py < A.cam.height;
  Ray R;
  R.cyc[0] = R.cyc[1] = R.cyc[2] = R.cyc[3] = 0;
  R.pix = valid ? (uint32_t)(py * A.cam.width + px) : 0u;
  init_ray(A, R, px, py, valid);
  trace_warp<OPAQUE, COUNT, KEY16>(A, R);
  finish<COUNT>(A, R, valid);
}

// Write a finished pixel (or queue it for the repair re-trace).
__device__ __forceinline__ void write_pixel(const TraceArgs& A, const Ray& R) {
  if (R.missed) {
    const uint32_t q = atomicAdd(A.pq_cnt, 1u);
    if (q < A.pq_cap) A.pq[q] = R.pix;
    else set_err(A.g.st, kErrOverflow);
    return;
  }
  A.rgba[R.pix] = make_float4(R.C[0], R.C[1], R.C[2], 1.0f - R.T);
  if (A.first_id) A.first_id[R.pix] = R.first_id;
  if (A.first_t) A.first_t[R.pix] = R.first_t;
}

// Opaque and repair traces use persistent warps: a lane whose ray is finished
// writes its pixel and goes idle; idle lanes take the next work items (one
// atomic per refill). Work item w of the image is pixel (w mod 32) of the
// (w / 32)-th 8x4 tile, so a full refill is a coherent tile; in the repair
// re-trace, item w is the w-th queued pixel.
template <bool OPAQUE, bool COUNT, bool KEY16>
__global__ void __launch_bounds__(kTraceThreads) k_trace(TraceArgs A) {
  const int lane = threadIdx.x & 31;
  const uint32_t W = (uint32_t)A.cam.width, H = (uint32_t)A.cam.height;
  const uint32_t tiles_x = (W + 7) / 8;
  const uint32_t total = A.pix_list ? min(*A.pix_count, A.pq_cap) : tiles_x * ((H + 3) / 4) * 32u;
  Ray R;
  R.active = R.pending = false;
  R.n_steps = R.n_entries = R.n_cap = R.n_vox = 0;
  R.n_hits = R.n_ww_vox = R.n_ww_ent = 0;
  R.cyc[0] = R.cyc[1] = R.cyc[2] = R.cyc[3] = 0;
  unsigned c_steps = 0, c_entries = 0, c_cap = 0, c_vox = 0, c_hits = 0, c_wwv = 0, c_wwe = 0;
  long long tclk = COUNT ? clock64() : 0;
  bool has = false;
  // Opaque main trace: refill once half the warp is idle. Queued repair
  // pixels are scattered: a warp takes at most its share of the queue, one
  // pixel each when few are queued.
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  const int threshold = A.pix_list ? 1 : 16;
  const int cap = A.pix_list ? (int)min(32u, max(1u, (total + n_warps - 1) / n_warps)) : 32;
  for (;;) {
    const unsigned idle = __ballot_sync(FULL, !has);
    bool exhausted = false;
    if (__popc(idle) >= threshold) {
      const int take = min(__popc(idle), cap);
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(A.work_next, (uint32_t)take);
      base = __shfl_sync(FULL, base, 0);
      exhausted = base >= total;
      const int rank = __popc(idle & ((1u << lane) - 1u));
      if (!has && rank < take) {
        const uint32_t w = base + (uint32_t)rank;
        if (w < total) {
          uint32_t px, py;
          if (A.pix_list) {
            const uint32_t pix = A.pix_list[w];
            px = pix % W;
            py = pix / W;
          } else {
            const uint32_t tile = w >> 5, within = w & 31u;
            px = (tile % tiles_x) * 8 + (within & 7u);
            py = (tile / tiles_x) * 4 + (within >> 3);
          }
          if (px < W && py < H) {
            if (COUNT) {
              c_steps += R.n_steps; c_entries += R.n_entries; c_cap += R.n_cap; c_vox += R.n_vox;
              c_hits += R.n_hits; c_wwv += R.n_ww_vox; c_wwe += R.n_ww_ent;
            }
            R.pix = py * W + px;
            init_ray(A, R, (int)px, (int)py, true);
            if (A.pix_list && A.resume) resume_ray(A, R);
            has = true;
          }
        }
      }
    }
    if (!__any_sync(FULL, has)) {
      if (__all_sync(FULL, exhausted)) break;
      continue;
    }
    if (has && R.active && !R.pending) {
      R.pending = advance<COUNT>(A, R, 3 * A.g.n + 16) == 1;
      if (!R.pending) R.active = false;
    }
    lap<COUNT>(R.cyc[0], tclk);
    process_flat<OPAQUE, COUNT, KEY16>(A, R);
    lap<COUNT>(R.cyc[1], tclk);
    // long lists: the whole warp on one list at a time
    unsigned pm = __ballot_sync(FULL, R.pending);
    while (pm) {
      const int L = __ffs(pm) - 1;
      pm &= pm - 1;
      process_voxel<OPAQUE, COUNT, KEY16>(A, R, L);
      if (lane == L) {
        R.pending = false;
        if (R.t1 < 0.0f) R.active = false;
      }
    }
    lap<COUNT>(R.cyc[2], tclk);
    if (has && !R.active && !R.pending) {
      write_pixel(A, R);
      has = false;
    }
  }
  if (COUNT) {
    lap<COUNT>(R.cyc[0], tclk);
    unsigned long long e = c_entries + R.n_entries, c = c_cap + R.n_cap, v = c_vox + R.n_vox,
                       st = c_steps + R.n_steps, h = c_hits + R.n_hits, wv = c_wwv + R.n_ww_vox,
                       we = c_wwe + R.n_ww_ent;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(FULL, e, o);
      c += __shfl_xor_sync(FULL, c, o);
      v += __shfl_xor_sync(FULL, v, o);
      st += __shfl_xor_sync(FULL, st, o);
      h += __shfl_xor_sync(FULL, h, o);
      wv += __shfl_xor_sync(FULL, wv, o);
      we += __shfl_xor_sync(FULL, we, o);
    }
    if (lane == 0) {
      atomicAdd(&A.g.st->tr_entries, e);
      atomicAdd(&A.g.st->tr_capsule, c);
      atomicAdd(&A.g.st->tr_voxels, v);
      atomicAdd(&A.g.st->tr_steps, st);
      atomicAdd(&A.g.st->tr_hits, h);
      atomicAdd(&A.g.st->tr_ww_voxels, wv);
      atomicAdd(&A.g.st->tr_ww_entries, we);
      for (int k = 0; k < 4; ++k) atomicAdd(&A.g.st->tr_cycles[k], R.cyc[k]);
    }
  }
}

// Persistent grid: as many blocks as can be resident at once.
template <bool OPAQUE, bool COUNT, bool KEY16>
int persistent_blocks(size_t smem) {
  static int blocks = 0;  // per instantiation; the device does not change under a grid
  if (!blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<OPAQUE, COUNT, KEY16>, kTraceThreads, smem);
    blocks = max(1, sms) * max(1, per_sm);
  }
  return blocks;
}

template <bool OPAQUE, bool COUNT, bool KEY16>
void launch_one(const TraceArgs& a, size_t smem, cudaStream_t s) {
  if (!OPAQUE && !a.pix_list) {
    // the instrumented and 16+16-key traces use the default tile
    const int tw = (COUNT || KEY16) ? 4 : a.tile_w;
    const int th = 32 / tw;
    const dim3 grid((a.cam.width + 2 * tw - 1) / (2 * tw), (a.cam.height + 2 * th - 1) / (2 * th));
    if constexpr (COUNT || KEY16) {
      k_trace_tile<OPAQUE, COUNT, KEY16, 4><<<grid, kTraceThreads, smem, s>>>(a);
    } else {
      if (tw == 2) k_trace_tile<OPAQUE, COUNT, KEY16, 2><<<grid, kTraceThreads, smem, s>>>(a);
      else if (tw == 8) k_trace_tile<OPAQUE, COUNT, KEY16, 8><<<grid, kTraceThreads, smem, s>>>(a);
      else if (tw == 16) k_trace_tile<OPAQUE, COUNT, KEY16, 16><<<grid, kTraceThreads, smem, s>>>(a);
      else k_trace_tile<OPAQUE, COUNT, KEY16, 4><<<grid, kTraceThreads, smem, s>>>(a);
    }
  } else {
    k_trace<OPAQUE, COUNT, KEY16><<<persistent_blocks<OPAQUE, COUNT, KEY16>(smem), kTraceThreads, smem, s>>>(a);
  }
}

template <bool COUNT, bool KEY16>
void launch_mode(const TraceArgs& a, int K, size_t smem, cudaStream_t s) {
  if (K == 1) launch_one<true, COUNT, KEY16>(a, smem, s);
  else launch_one<false, COUNT, KEY16>(a, smem, s);
}

int launch_trace(const TraceArgs& a, int K, cudaStream_t s) {
  const size_t smem = K == 1 ? 0 : sizeof(unsigned long long) * kRayKeys * kTraceThreads;
  if (a.count) {
    if (a.key16) launch_mode<true, true>(a, K, smem, s);
    else launch_mode<true, false>(a, K, smem, s);
  } else {
    if (a.key16) launch_mode<false, true>(a, K, smem, s);
    else launch_mode<false, false>(a, K, smem, s);
  }
  return 1;
}

// --------------------------------------------------- instrumented trace
__global__ void k_touch_count(const uint32_t* bits, size_t words, unsigned long long* out) {
  unsigned long long c = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words;
       i += (size_t)gridDim.x * blockDim.x)
    c += __popc(bits[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

int launch_touch_count(const uint32_t* list_bits, size_t list_words, const uint32_t* vert_bits,
                       size_t vert_words, const uint32_t* vox_bits, size_t vox_words,
                       DevStatus* st, cudaStream_t s) {
  k_touch_count<<<152 * 4, 256, 0, s>>>(list_bits, list_words, &st->tr_u_entries);
  k_touch_count<<<152 * 4, 256, 0, s>>>(vert_bits, vert_words, &st->tr_u_vertices);
  k_touch_count<<<152 * 4, 256, 0, s>>>(vox_bits, vox_words, &st->tr_u_voxels);
  return 3;
}

// ----------------------------------------------------------------- repair
__global__ void k_repair_alloc(GridDev g, const uint32_t* vq, const uint32_t* vq_cnt,
                               const uint32_t* pq_cnt, uint32_t vq_cap) {
  const uint32_t nq = min(*vq_cnt, vq_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && nq) {
    atomicAdd(&g.st->repair_rounds, 1u);
    atomicAdd(&g.st->repaired_voxels, nq);
    atomicAdd(&g.st->retraced_pixels, *pq_cnt);
  }
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint32_t idx = vq[q];
    const uint32_t cnt = g.word[idx] & 0xffffu;
    const uint32_t start = atomicAdd(&g.st->list_tail, cnt);
    if ((unsigned long long)start + cnt > g.list_cap) set_err(g.st, kErrOverflow);
    g.cur[idx] = start;
    atomicOr(&g.vis[idx >> 5], 1u << (idx & 31));
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

int launch_repair_alloc(const GridDev& g, const uint32_t* vq, const uint32_t* vq_cnt,
                        const uint32_t* pq_cnt, uint32_t vq_cap, cudaStream_t s) {
  k_repair_alloc<<<152, 256, 0, s>>>(g, vq, vq_cnt, pq_cnt, vq_cap);
  return 1;
}

int launch_repair_clear(const GridDev& g, uint32_t* need, const uint32_t* vq,
                         const uint32_t* vq_cnt, uint32_t vq_cap, int next, cudaStream_t s) {
  k_repair_clear<<<152, 256, 0, s>>>(g, need, vq, vq_cnt, vq_cap, next);
  return 1;
}

}  // namespace vrt
