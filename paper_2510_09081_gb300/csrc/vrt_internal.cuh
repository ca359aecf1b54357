// Internal device-side definitions shared by the kernels of libvrt.
//
// Geometry follows Kraaijeveld et al., "Real-Time Rendering of Dynamic Line
// Sets using Voxel Ray Tracing" (arXiv 2510.09081): capsule primitives with
// clip planes (Sec. 3.1, Alg. 2), PWAA-clamped occupancy (Alg. 3), capsule
// ray intersection with clip planes (Sec. 3.5).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vrt {

// ---------------------------------------------------------------- constants
constexpr int kUnitsLog2 = 14;
constexpr float kUnits = 16384.0f;             // snapping grid: 2^-14 voxel
constexpr int kListMarginUnits = 32;           // list radius = r + 2^-9 voxel
constexpr float kCoordMin = -256.0f;           // accepted coordinate range
constexpr float kCoordMax = 768.0f;
constexpr float kTStop = 1e-4f;                // transmittance where a ray stops
constexpr int kMaxRepairRounds = 4;
constexpr uint32_t kRayQueueLimit = 8;          // culled voxels one ray queues per round
constexpr uint32_t kShortList = 1024;           // trace: longer lists go to the whole-warp path
constexpr int kRayKeys = 32;                    // trace: hit slots per transparent ray on the shared-entry path
constexpr int kBrickDistMax = 15;               // cap of the empty-brick distance field
constexpr int kMipsF32 = 0, kMipsF16 = 1, kMipsBF16 = 2;  // occupancy pyramid storage

// per-vertex flag bits, stored in pos[i].w as raw bits
constexpr uint32_t kFirst = 1u, kLast = 2u, kClipOn = 4u;

// device status bits
constexpr uint32_t kErrRange = 1u;      // coordinate out of range / not finite
constexpr uint32_t kErrOverflow = 2u;   // packed field or list capacity overflow
constexpr uint32_t kErrTimeout = 4u;    // bounded wait gave up
constexpr uint32_t kErrBounds = 8u;     // index out of its buffer
constexpr uint32_t kErrRepair = 16u;    // repair rounds exhausted

// List start the scan gives a voxel the cull left without a list; list
// capacities stay below it, so a cursor at or above it marks such a voxel.
constexpr uint32_t kCulledStart = 0xC0000000u;

struct DevStatus {
  unsigned int err;
  unsigned int occupied_voxels;
  unsigned long long F;              // fragments of pass 1
  unsigned long long sum_q;          // occupancy codes of pass 1
  unsigned long long exact_decisions;  // list decisions on the exact path
  unsigned long long rec_cnt;        // record slots taken by pass 1 and its exact path
  // --- reset by every list build from here on
  unsigned long long sum_count_field;  // checked by the scan
  unsigned long long sum_occ_field;
  unsigned long long listed;         // entries written by pass 2 and repairs
  unsigned int xq_cnt;               // undecided (segment, voxel) pairs of pass 1
  unsigned int cq_cnt;               // records of unlisted voxels pass 2 copied to xq
  unsigned int list_tail;            // next free list entry (scan total + repairs)
  unsigned int visible_voxels;
  unsigned int max_count;
  unsigned int scan_tile_counter;
  unsigned int vq_cnt[2];            // culled voxels a ray needed (ping-pong per round)
  unsigned int pq_cnt[2];            // pixels to trace again (ping-pong per round)
  unsigned int repaired_voxels;
  unsigned int repair_rounds;
  unsigned int retraced_pixels;
  unsigned int occq_cnt;             // occupied voxels the erosion queued for the cull's march
  // trace work counters (only with VRT_OPT_TRACE_COUNTERS)
  unsigned long long tr_entries;     // list entries examined
  unsigned long long tr_capsule;     // entries past the line-distance test
  unsigned long long tr_voxels;      // voxel lists processed
  unsigned long long tr_steps;       // DDA steps (voxels and empty bricks)
  unsigned int tr_next[kMaxRepairRounds + 1];  // work items handed out per trace launch
  unsigned int tr_pad;
  unsigned long long tr_ww_voxels;   // voxel lists taken by the whole-warp path
  unsigned long long tr_ww_entries;  // entries it examined (rescans included)
  unsigned long long tr_hits;        // accepted hits (keys a ray received)
  unsigned long long tr_cycles[4];   // warp cycles: DDA, shared-entry path, whole-warp path,
                                     // and the capsule tests within the shared-entry path
  // distinct list entries, vertices and voxel words the rays of the last
  // instrumented trace read (its repair rounds included)
  unsigned long long tr_u_entries, tr_u_vertices, tr_u_voxels;
};

// -------------------------------------------------------------- grid layout
// Voxels are stored in 4^3 bricks of 64 consecutive words, bricks in x-fastest
// order, so one ray step or one segment's neighbourhood touches few lines and
// the list build (scan order) keeps spatial neighbours together.
__host__ __device__ __forceinline__ uint32_t brick_index(int x, int y, int z, int log2nb) {
  uint32_t b = ((uint32_t)(z >> 2) << (2 * log2nb)) | ((uint32_t)(y >> 2) << log2nb) |
               (uint32_t)(x >> 2);
  return (b << 6) | ((uint32_t)(z & 3) << 4) | ((uint32_t)(y & 3) << 2) | (uint32_t)(x & 3);
}
// Inverse of brick_index.
__host__ __device__ __forceinline__ void brick_coords(uint32_t idx, int log2nb, int& x, int& y, int& z) {
  const uint32_t b = idx >> 6, l = idx & 63u;
  const uint32_t mask = (1u << log2nb) - 1u;
  x = (int)(((b & mask) << 2) | (l & 3u));
  y = (int)((((b >> log2nb) & mask) << 2) | ((l >> 2) & 3u));
  z = (int)(((b >> (2 * log2nb)) << 2) | (l >> 4));
}

struct GridDev {
  int n, log2n, log2nb;    // side, log2 side, log2 bricks per side
  float r;                 // render radius (snapped)
  float rl;                // list radius = r + 2^-9
  int R, RL;               // the same in 2^-14 units
  float r_clamp, corr;     // Alg. 3: max(r, r_min), (r / r_clamp)^2
  float occ_scale;
  int force_exact;
  uint32_t* word;          // [n^3] packed (occupancy code sum << 16) | count
  uint32_t* cur;           // [n^3] list end cursor (start = cur - count); >= kCulledStart: no list
  uint32_t* vis;           // [n^3 / 32] voxel has a list
  const uint8_t* bdist;    // [bricks] Chebyshev distance (bricks) to an occupied brick, capped
  uint32_t* lists;         // [list_cap]
  unsigned long long list_cap;
  uint2* xq;               // [xq_cap] undecided (segment id, packed voxel) pairs
  uint32_t xq_cap;
  unsigned long long* rec; // [rec_cap] fragment records: voxel << 32 | segment
  uint16_t* rank;          // [rec_cap] a record's position among its voxel's fragments
  uint32_t rec_cap;
  DevStatus* st;
};

__device__ __forceinline__ void set_err(DevStatus* st, uint32_t bit) { atomicOr(&st->err, bit); }

// --------------------------------------------------------------- small math
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float cmp3(float3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ------------------------------------------------- list membership predicate
// Decides dist(segment [a, a + d], unit box [0,1]^3) <= rl, with a and d in
// voxel units relative to the box's lower corner (exact fp32 multiples of
// 2^-14). Returns 1 (within), 0 (not within) or -1 (too close to call in fp32).
//
// Stage 1 takes a point p = a + t d of the segment near the box centre c (t
// from the projection of c, clamped to [0, 1]), e = c - p:
//   dist(p, box) <= rl -> within (p is on the segment)
//   |e| - (|e_x| + |e_y| + |e_z|) / (2 |e|) - reach > rl -> not within: along
//     the unit normal e / |e| the box lies at least |e| - (half its 1-norm)
//     beyond p, and the segment reaches at most
//     reach = max(0, -t d.e, (1 - t) d.e) / |e| beyond p (its endpoints are
//     p - t d and p + (1 - t) d). This holds for any t, so the projection
//     needs no exact division.
// Stage 2 runs Newton steps on the convex, C^1, piecewise-quadratic squared
// box distance f(t) and brackets its minimum: f(t) is an upper bound, and
// convexity gives f(t) - |f'(t)| * (t or 1 - t) as a lower bound, again for
// any t.
// Both stages add a rounding allowance proportional to the squared magnitude
// of the local coordinates.
// Rounding allowance of both stages for local coordinates a, a + d.
__device__ __forceinline__ float seg_box_tol(float3 a, float3 d) {
  const float M = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fabsf(a.z)),
                        fmaxf(fmaxf(fabsf(a.x + d.x), fabsf(a.y + d.y)), fabsf(a.z + d.z)));
  return 4.8e-7f * (M + 2.0f) * (M + 2.0f);
}

// Stage 1: 1 within, 0 not within, -1 undecided.
__device__ __forceinline__ int seg_box_stage1(float3 a, float3 d, float rl) {
  const float tol = seg_box_tol(a, d);
  const float dd = dot3(d, d);
  const float3 w = make_float3(0.5f - a.x, 0.5f - a.y, 0.5f - a.z);
  const float t = dd > 0.0f ? fminf(1.0f, fmaxf(0.0f, __fdividef(dot3(w, d), dd))) : 0.0f;
  const float3 e = w - t * d;  // c - p
  const float ex = fmaxf(fabsf(e.x) - 0.5f, 0.0f), ey = fmaxf(fabsf(e.y) - 0.5f, 0.0f),
              ez = fmaxf(fabsf(e.z) - 0.5f, 0.0f);
  const float up2 = ex * ex + ey * ey + ez * ez;  // dist(p, box)^2
  if (up2 + tol <= rl * rl) return 1;
  const float e2 = dot3(e, e);
  if (e2 > 0.0f) {
    const float len = sqrtf(e2);
    const float de = dot3(d, e);
    const float reach = fmaxf(0.0f, fmaxf(-t * de, (1.0f - t) * de));
    const float lb = len - __fdividef(0.5f * (fabsf(e.x) + fabsf(e.y) + fabsf(e.z)) + reach, len);
    if (lb > rl && lb * lb - tol > rl * rl) return 0;
  }
  return -1;
}

// Stage 2: 1 within, 0 not within, -1 undecided (left to the exact decision).
__device__ __forceinline__ int seg_box_stage2(float3 a, float3 d, float rl) {
  const float tol = seg_box_tol(a, d);
  const float dd = dot3(d, d);
  const float3 w = make_float3(0.5f - a.x, 0.5f - a.y, 0.5f - a.z);
  float t = dd > 0.0f ? fminf(1.0f, fmaxf(0.0f, __fdividef(dot3(w, d), dd))) : 0.0f;
  float f = 0.0f, g = 0.0f;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    float gg = 0.0f, gp = 0.0f, ff = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float ak = cmp3(a, k), dk = cmp3(d, k);
      const float x = fmaf(t, dk, ak);
      const float e = x < 0.0f ? x : (x > 1.0f ? x - 1.0f : 0.0f);
      gg = fmaf(dk, e, gg);
      ff = fmaf(e, e, ff);
      if (e != 0.0f) gp = fmaf(dk, dk, gp);
    }
    f = ff;
    g = gg;
    if (it == 3 || gp == 0.0f) break;
    t = fminf(1.0f, fmaxf(0.0f, t - __fdividef(gg, gp)));
  }
  const float rl2 = rl * rl;
  if (f + tol <= rl2) return 1;
  const float lb = f - 2.0f * fabsf(g) * (g > 0.0f ? t : 1.0f - t);
  if (lb - tol > rl2) return 0;
  return -1;
}

// Exact decision in 64/128-bit integers (units of 2^-14; box [0, S]^3).
// The points within R of the box are the union of the box grown by R along a
// single axis (3 pieces), the 12 edge cylinders of radius R cut to their
// edge's slab, and the 8 corner balls; the segment is within R of the box iff
// it meets one of the pieces.
struct TRange {  // t in [n0/d0, n1/d1], d > 0
  long long n0, d0, n1, d1;
};
__device__ __forceinline__ bool t_le(long long na, long long da, long long nb, long long db) {
  return (__int128)na * db <= (__int128)nb * da;
}
// Narrow r to the t where lo <= A + t D <= hi; false when empty.
__device__ __forceinline__ bool t_clip(TRange& r, long long A, long long D, long long lo, long long hi) {
  if (D == 0) return lo <= A && A <= hi;
  long long na, nb, den;
  if (D > 0) { na = lo - A; nb = hi - A; den = D; }
  else       { na = A - hi; nb = A - lo; den = -D; }
  if (t_le(r.n0, r.d0, na, den)) { r.n0 = na; r.d0 = den; }
  if (t_le(nb, den, r.n1, r.d1)) { r.n1 = nb; r.d1 = den; }
  return t_le(r.n0, r.d0, r.n1, r.d1);
}
// min over t in r of |W + t E|^2 <= R2 (dim 2 or 3)
template <int DIM>
__device__ __forceinline__ bool seg_near_point(const long long* W, const long long* E, TRange r,
                                               __int128 R2) {
  __int128 ee = 0, we = 0, ww = 0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    ee += (__int128)E[k] * E[k];
    we += (__int128)W[k] * E[k];
    ww += (__int128)W[k] * W[k];
  }
  if (ee == 0) return ww <= R2;
  // unconstrained minimiser -we/ee inside r?  (ee > 0)
  const bool after_lo = (__int128)r.n0 * ee <= -we * (__int128)r.d0;
  const bool before_hi = -we * (__int128)r.d1 <= (__int128)r.n1 * ee;
  if (after_lo && before_hi) {
    __int128 c2;
    if (DIM == 2) {
      __int128 c = (__int128)W[0] * E[1] - (__int128)W[1] * E[0];
      c2 = c * c;
    } else {
      __int128 cx = (__int128)W[1] * E[2] - (__int128)W[2] * E[1];
      __int128 cy = (__int128)W[2] * E[0] - (__int128)W[0] * E[2];
      __int128 cz = (__int128)W[0] * E[1] - (__int128)W[1] * E[0];
      c2 = cx * cx + cy * cy + cz * cz;
    }
    return c2 <= R2 * ee;
  }
  // otherwise the nearer end of r; testing both is enough for a convex function
  const long long tn[2] = {r.n0, r.n1}, td[2] = {r.d0, r.d1};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    __int128 s = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      __int128 v = (__int128)W[k] * td[e] + (__int128)tn[e] * E[k];
      s += v * v;
    }
    if (s <= R2 * (__int128)td[e] * td[e]) return true;
  }
  return false;
}

static __device__ __noinline__ bool seg_box_exact(const long long* A, const long long* D, long long S,
                                           long long R) {
  const __int128 R2 = (__int128)R * R;
  // grown boxes
  for (int g = 0; g < 3; ++g) {
    TRange r = {0, 1, 1, 1};
    bool ok = true;
    for (int k = 0; k < 3 && ok; ++k) {
      long long lo = (k == g) ? -R : 0, hi = (k == g) ? S + R : S;
      ok = t_clip(r, A[k], D[k], lo, hi);
    }
    if (ok) return true;
  }
  // edge cylinders
  for (int m = 0; m < 3; ++m) {
    TRange r = {0, 1, 1, 1};
    if (!t_clip(r, A[m], D[m], 0, S)) continue;
    const int k = m == 0 ? 1 : 0, l = m == 2 ? 1 : 2;
    for (int c = 0; c < 4; ++c) {
      const long long ck = (c & 1) ? S : 0, cl = (c & 2) ? S : 0;
      const long long W[2] = {A[k] - ck, A[l] - cl};
      const long long E[2] = {D[k], D[l]};
      if (seg_near_point<2>(W, E, r, R2)) return true;
    }
  }
  // corner balls
  for (int c = 0; c < 8; ++c) {
    const long long W[3] = {A[0] - ((c & 1) ? S : 0), A[1] - ((c & 2) ? S : 0),
                            A[2] - ((c & 4) ? S : 0)};
    const TRange r = {0, 1, 1, 1};
    if (seg_near_point<3>(W, D, r, R2)) return true;
  }
  return false;
}

// Filter stages for voxel (x, y, z): 1 within, 0 not, -1 undecided. a, b are
// the snapped global endpoints (local coordinates are exact in fp32).
__device__ __forceinline__ int seg_stage1_at(float3 a, float3 b, int x, int y, int z, float rl) {
  const float3 la = make_float3(a.x - (float)x, a.y - (float)y, a.z - (float)z);
  return seg_box_stage1(la, b - a, rl);
}
__device__ __forceinline__ int seg_stage2_at(float3 a, float3 b, int x, int y, int z, float rl) {
  const float3 la = make_float3(a.x - (float)x, a.y - (float)y, a.z - (float)z);
  return seg_box_stage2(la, b - a, rl);
}

// Exact decision for voxel (x, y, z) on the 2^-14 lattice.
__device__ __forceinline__ bool seg_exact_at(float3 a, float3 b, int x, int y, int z, int RL) {
  const float3 la = make_float3(a.x - (float)x, a.y - (float)y, a.z - (float)z);
  const long long A[3] = {__float2ll_rn(la.x * kUnits), __float2ll_rn(la.y * kUnits),
                          __float2ll_rn(la.z * kUnits)};
  const long long D[3] = {__float2ll_rn(b.x * kUnits) - __float2ll_rn(a.x * kUnits),
                          __float2ll_rn(b.y * kUnits) - __float2ll_rn(a.y * kUnits),
                          __float2ll_rn(b.z * kUnits) - __float2ll_rn(a.z * kUnits)};
  return seg_box_exact(A, D, (long long)kUnits, (long long)RL);
}

// (segment, voxel) pairs the filter could not decide, packed for the exact pass.
__device__ __forceinline__ uint32_t pack_voxel(int x, int y, int z) {
  return (uint32_t)x | ((uint32_t)y << 10) | ((uint32_t)z << 20);
}
__device__ __forceinline__ void unpack_voxel(uint32_t p, int& x, int& y, int& z) {
  x = (int)(p & 1023u); y = (int)((p >> 10) & 1023u); z = (int)(p >> 20);
}

// ------------------------------------------------------------- Alg. 2 and 3
// Occupancy of the clipped capsule sampled at p (Alg. 3 around Alg. 2), with
// local coordinates (p, a, b relative to the same origin).
__device__ __forceinline__ float capsule_occupancy(float3 p, float3 a, float3 b, float3 n0, float3 n1,
                                                   bool en0, bool en1, float r_clamp, float corr) {
  const float3 d = b - a;
  const float3 pa = p - a, pb = p - b;
  const float dd = dot3(d, d);
  const float h = dd > 0.0f ? fminf(1.0f, fmaxf(0.0f, __fdividef(dot3(pa, d), dd))) : 0.0f;
  const float3 q = pa - h * d;
  // an approximate square root (a few ulp) moves the code Q * occupancy by far
  // less than the 1e-3 within which the oracle accepts either rounding
  const float q2 = dot3(q, q);
  float s = (q2 > 0.0f ? q2 * rsqrtf(q2) : 0.0f) - r_clamp;
  if (en0) s = fmaxf(s, -dot3(pa, n0));
  if (en1) s = fmaxf(s, dot3(pb, n1));
  return fminf(1.0f, fmaxf(0.0f, 0.5f - s)) * corr;
}

// ------------------------------------------------------------ ray / capsule
// Can the line o + t d come within r of the segment [a, b]? A hit needs the
// two lines within r of each other: with n = d x (b - a), their distance is
// |(o - a) . n| / |n|. Conservative (margin 1e-3 voxel on r; nearly parallel
// lines always pass), so it only skips capsules the full test would miss.
__device__ __forceinline__ bool lines_may_meet(float3 o, float3 d, float3 a, float3 b, float rr_margin) {
  const float3 ba = b - a;
  const float3 n = make_float3(d.y * ba.z - d.z * ba.y, d.z * ba.x - d.x * ba.z, d.x * ba.y - d.y * ba.x);
  const float nn = dot3(n, n);
  if (!(nn > 1e-4f * dot3(ba, ba))) return true;
  const float s = dot3(o - a, n);
  return s * s <= rr_margin * nn;
}

// First entry of the line o + t d (|d| = 1) into the ball of radius^2 r2
// centred at o - oc; +inf when the line misses it.
__device__ __forceinline__ float ball_entry(float3 oc, float3 d, float r2) {
  const float bq = dot3(oc, d);
  const float3 w = oc - bq * d;
  const float disc = r2 - dot3(w, w);
  return disc >= 0.0f ? -bq - (disc > 0.0f ? disc * rsqrtf(disc) : 0.0f) : __int_as_float(0x7f800000);
}

// First entry of the line o + t d (|d| = 1) into the capsule (a, b, r); +inf
// when the line misses it. Both end balls lie inside the infinite cylinder
// around the axis, so the line meets the capsule only if it meets that
// cylinder, and where it enters the cylinder decides the rest: between the two
// end planes that entry is the capsule's; before a (after b) the line can
// reach the rest of the capsule only through the ball at a (at b), whose entry
// is then the capsule's. The perpendicular offsets are formed explicitly so
// that the discriminants do not cancel when the origin is far away.
__device__ __forceinline__ float capsule_entry(float3 o, float3 d, float3 a, float3 b, float r2) {
  const float3 oa = o - a;
  const float3 ba = b - a;
  const float L2 = dot3(ba, ba);
  if (!(L2 > 0.0f)) return ball_entry(oa, d, r2);
  const float inv = __fdividef(1.0f, L2);
  const float3 dp = d - (dot3(d, ba) * inv) * ba;
  const float3 op = oa - (dot3(oa, ba) * inv) * ba;
  const float A = dot3(dp, dp);
  if (!(A > 1e-30f))  // along the axis: the nearer ball
    return fminf(ball_entry(oa, d, r2), ball_entry(o - b, d, r2));
  const float ts = __fdividef(-dot3(op, dp), A);
  const float3 w = op + ts * dp;
  const float disc = r2 - dot3(w, w);
  if (disc < 0.0f) return __int_as_float(0x7f800000);
  const float q = __fdividef(disc, A);
  const float t = ts - (q > 0.0f ? q * rsqrtf(q) : 0.0f);
  const float y = dot3(oa + t * d, ba);
  if (y < 0.0f) return ball_entry(oa, d, r2);
  if (y > L2) return ball_entry(o - b, d, r2);
  return t;
}

}  // namespace vrt
