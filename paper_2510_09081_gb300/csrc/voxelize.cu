// A1 / A5: the two voxelization passes of the voxelize-(cull-)scan-voxelize
// list build (Sec. 3.1, 3.3).
//
// Both passes enumerate the same candidate voxels per segment -- the
// slab-by-slab traversal of Alg. 1 along the major axis a0 of d = v1 - v0, each
// slab visiting a 2D box of minor-axis voxels around the segment -- and keep a
// voxel iff the segment lies within the list radius of the voxel's closed box.
// The minor half-extent of a slab uses the exact half-width of the tube's
// cross-section in a major-axis plane, rl * sqrt(1 + (d_ai / d_a0)^2), which is
// never below Eq. 1's projected radius. Every slab's box is indexed with the
// same width bound (the slab's extent along a minor axis is at most
// |d_ai / d_a0| + 2 * half-extent), so candidate q of a segment decodes in O(1).
//
// Work layout: each lane loads one segment (coalesced), sets up its walk and
// stores it, packed, in shared memory; the warp numbers the candidates of its
// 32 segments consecutively and takes them 32 at a time, each lane reading the
// walk of the segment its candidate belongs to, so segments of different
// lengths do not leave lanes idle. The fp32 filter decides almost every candidate; pairs it
// cannot decide go to a queue that a separate kernel decides exactly (keeping
// the 128-bit integer path out of the hot kernels' registers).
//
// Pass 1 adds (occupancy code << 16) | 1 to the voxel's packed word with a
// 32-bit atomic (Sec. 3.1) and writes the fragment as an 8-byte record (voxel << 32 |
// segment) with its rank, the count field the atomic returned (fragments of
// the voxel added before it), beside it. A block takes record slots for all its
// walks' candidates with one atomic; each warp writes its fragments at the
// start of its share and marks the rest (candidates that were not kept)
// kNoRecord. The paper re-voxelizes in its second pass to save memory; with the
// records in HBM the second pass is a streaming scatter instead: for every
// record whose voxel received a list, write the segment id at the slot its
// rank gives below the voxel's list end (Sec. 3.3), with no atomic.
#include "launch.h"

namespace vrt {

constexpr float kWalkEps = 1e-3f;
constexpr unsigned FULLW = 0xffffffffu;

struct Walk {
  float3 a, b;
  float am, a1, a2, s1, s2, rho1, rho2, lo_m, hi_m;
  float inv_w12, inv_w2;  // reciprocals of W1 * W2 and W2 for the uniform decode
  int m, c0, W1, W2;
  bool exact;             // candidates are exactly the slab boxes' voxels
  bool boxed;             // exact, with at most kBoxedSlabs slabs: boxes kept
  uint32_t pre[4];        // exact: 16-bit cumulative counts after slabs 0..7
  uint32_t box[6];        // boxed: slab k's box, j0 | l0 << 10 | (l1 - l0 + 1) << 20
  uint32_t n;             // candidates
};

constexpr int kExactSlabs = 9;  // slabs whose boxes the exact decode indexes
constexpr int kBoxedSlabs = 6;  // slabs whose boxes the packed walk can hold

// Minor-axis voxel ranges of slab c (clamped to the grid): the axis line
// a_k + (x - a_m) s_k over the slab's part of [lo_m, hi_m], widened by rho_k.
__device__ __forceinline__ void slab_box(float am, float a1, float a2, float s1, float s2,
                                         float rho1, float rho2, float lo_m, float hi_m, int n,
                                         int c, int& j0, int& j1, int& l0, int& l1) {
  const float x0 = fmaxf((float)c, lo_m), x1 = fminf((float)(c + 1), hi_m);
  const float p1a = fmaf(x0 - am, s1, a1), p1b = fmaf(x1 - am, s1, a1);
  const float p2a = fmaf(x0 - am, s2, a2), p2b = fmaf(x1 - am, s2, a2);
  j0 = max(0, (int)floorf(fminf(p1a, p1b) - rho1));
  j1 = min(n - 1, (int)floorf(fmaxf(p1a, p1b) + rho1));
  l0 = max(0, (int)floorf(fminf(p2a, p2b) - rho2));
  l1 = min(n - 1, (int)floorf(fmaxf(p2a, p2b) + rho2));
}

__device__ __forceinline__ void walk_setup(float3 a, float3 b, const GridDev& g, Walk& w) {
  const float rl = g.rl;
  const int n = g.n;
  const float3 d = b - a;
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  const int m = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  const int k1 = m == 0 ? 1 : 0, k2 = m == 2 ? 1 : 2;
  w.a = a;
  w.b = b;
  w.m = m;
  w.am = cmp3(a, m);
  const float dm = cmp3(b, m) - w.am;
  w.s1 = dm != 0.0f ? cmp3(d, k1) / dm : 0.0f;
  w.s2 = dm != 0.0f ? cmp3(d, k2) / dm : 0.0f;
  w.rho1 = rl * sqrtf(fmaf(w.s1, w.s1, 1.0f)) + kWalkEps;
  w.rho2 = rl * sqrtf(fmaf(w.s2, w.s2, 1.0f)) + kWalkEps;
  w.lo_m = fminf(w.am, w.am + dm) - rl;
  w.hi_m = fmaxf(w.am, w.am + dm) + rl;
  w.a1 = cmp3(a, k1);
  w.a2 = cmp3(a, k2);
  w.c0 = max(0, (int)floorf(w.lo_m - kWalkEps));
  const int c1 = min(n - 1, (int)floorf(w.hi_m + kWalkEps));
  // Up to kExactSlabs slabs: candidates are the voxels of each slab's own box,
  // numbered slab after slab (cumulative counts kept); longer segments index
  // every slab's box with the widest slab's widths.
  int W1 = 1, W2 = 1;
  uint32_t total = 0;
  w.pre[0] = w.pre[1] = w.pre[2] = w.pre[3] = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < kExactSlabs; ++k) {  // unrolled: pre[] stays in registers
    const int c = w.c0 + k;
    if (c > c1) break;
    int j0, j1, l0, l1;
    slab_box(w.am, w.a1, w.a2, w.s1, w.s2, w.rho1, w.rho2, w.lo_m, w.hi_m, n, c, j0, j1, l0, l1);
    W1 = max(W1, j1 - j0 + 1);
    W2 = max(W2, l1 - l0 + 1);
    total += (uint32_t)(max(0, j1 - j0 + 1) * max(0, l1 - l0 + 1));
    if (k < kBoxedSlabs)
      w.box[k] = ((uint32_t)j0 & 1023u) | (((uint32_t)l0 & 1023u) << 10) |
                 ((uint32_t)max(1, l1 - l0 + 1) << 20);
    if (k < 8) {  // cumulative count after slab k
      const uint32_t v = min(total, 0xffffu);
      w.pre[k >> 1] = (w.pre[k >> 1] & ~(0xffffu << (16 * (k & 1)))) | (v << (16 * (k & 1)));
    }
  }
  for (int c = w.c0 + kExactSlabs; c <= c1; ++c) {  // longer segments: widths only
    int j0, j1, l0, l1;
    slab_box(w.am, w.a1, w.a2, w.s1, w.s2, w.rho1, w.rho2, w.lo_m, w.hi_m, n, c, j0, j1, l0, l1);
    W1 = max(W1, j1 - j0 + 1);
    W2 = max(W2, l1 - l0 + 1);
  }
  const int slabs = c1 - w.c0 + 1;
  w.W1 = W1;
  w.W2 = W2;
  w.exact = slabs > 0 && slabs <= kExactSlabs && total < 0xffffu;
  w.boxed = w.exact && slabs <= kBoxedSlabs;
  w.n = slabs <= 0 ? 0u : (w.exact ? total : (uint32_t)slabs * (uint32_t)(W1 * W2));
  w.inv_w12 = 1.0f / (float)(W1 * W2);
  w.inv_w2 = 1.0f / (float)W2;
}

// A walk as five float4s in shared memory (plus the clip normals in two more):
//   w0 = (a, s1), w1 = (b, s2), w2 = (rho1, rho2, lo_m, hi_m),
//   w3 = (1 / (W1 W2), 1 / W2, bits, first candidate number of the warp),
//   w4 = cumulative counts after slabs 0..7, 16 bits each (exact decode),
//   bits = m | c0 << 2 | W1 << 11 | W2 << 19 | clip flags << 27 | exact << 29
//          | boxed << 30.
// A boxed walk keeps its slab boxes, as walk_setup found them, where the
// uniform decode's fields would be: slabs 0-3 in w2, slabs 4-5 in w3.x, w3.y.
// W1, W2 <= 2 + |s_k| + 2 rho_k < 16 since radius <= 4, and c0 < 512.
struct PackedWalk {
  float4 w0, w1, w2, w3;
  uint4 w4;
};

__device__ __forceinline__ PackedWalk pack_walk(const Walk& w, uint32_t clip, uint32_t first) {
  PackedWalk p;
  p.w0 = make_float4(w.a.x, w.a.y, w.a.z, w.s1);
  p.w1 = make_float4(w.b.x, w.b.y, w.b.z, w.s2);
  const uint32_t bits = (uint32_t)w.m | ((uint32_t)w.c0 << 2) | ((uint32_t)w.W1 << 11) |
                        ((uint32_t)w.W2 << 19) | (clip << 27) | ((uint32_t)w.exact << 29) |
                        ((uint32_t)w.boxed << 30);
  if (w.boxed) {
    p.w2 = make_float4(__uint_as_float(w.box[0]), __uint_as_float(w.box[1]),
                       __uint_as_float(w.box[2]), __uint_as_float(w.box[3]));
    p.w3 = make_float4(__uint_as_float(w.box[4]), __uint_as_float(w.box[5]), __uint_as_float(bits),
                       __uint_as_float(first));
  } else {
    p.w2 = make_float4(w.rho1, w.rho2, w.lo_m, w.hi_m);
    p.w3 = make_float4(w.inv_w12, w.inv_w2, __uint_as_float(bits), __uint_as_float(first));
  }
  p.w4 = make_uint4(w.pre[0], w.pre[1], w.pre[2], w.pre[3]);
  return p;
}

// Candidate q of a packed walk: its voxel, or false when q falls outside its
// slab's box (uniform decode only).
__device__ __forceinline__ bool decode_candidate(const PackedWalk& p, int n, uint32_t q, int& x,
                                                 int& y, int& z) {
  const uint32_t bits = __float_as_uint(p.w3.z);
  const int m = bits & 3, c0 = (bits >> 2) & 511, W1 = (bits >> 11) & 255, W2 = (bits >> 19) & 255;
  const float am = m == 0 ? p.w0.x : (m == 1 ? p.w0.y : p.w0.z);
  const float a1 = m == 0 ? p.w0.y : p.w0.x;
  const float a2 = m == 2 ? p.w0.y : p.w0.z;
  // (q + 1/2) / w is at least 1/(2w) from an integer, far beyond fp32 error for
  // these small counts, so truncation gives the exact quotient
  int slab, rem;
  if (bits & (1u << 29)) {  // exact: the slab whose cumulative range holds q
    // the number of cumulative counts <= q (non-decreasing, 16 bits each, two
    // per word; q < 65535), by packed half-word comparisons
    const uint32_t qq = q * 0x00010001u;
    slab = (__popc(__vcmpleu2(p.w4.x, qq)) + __popc(__vcmpleu2(p.w4.y, qq)) +
            __popc(__vcmpleu2(p.w4.z, qq)) + __popc(__vcmpleu2(p.w4.w, qq))) >> 4;
    const int s1 = slab - 1;
    const uint32_t word = s1 < 2 ? p.w4.x : (s1 < 4 ? p.w4.y : (s1 < 6 ? p.w4.z : p.w4.w));
    const uint32_t base = slab ? (word >> (16 * (s1 & 1))) & 0xffffu : 0u;
    rem = (int)(q - base);
  } else {
    slab = (int)(((float)q + 0.5f) * p.w3.x);
    rem = (int)q - slab * (W1 * W2);
  }
  const int c = c0 + slab;
  if (bits & (1u << 30)) {  // boxed: the slab's box as walk_setup found it; q lies inside it
    const uint32_t bx = __float_as_uint(
        slab < 2 ? (slab == 0 ? p.w2.x : p.w2.y)
                 : (slab < 4 ? (slab == 2 ? p.w2.z : p.w2.w) : (slab == 4 ? p.w3.x : p.w3.y)));
    const int w2 = (int)(bx >> 20);
    // an approximate reciprocal suffices: (rem + 1/2) / w2 lies at least 1/(2 w2)
    // from an integer and rem < 256
    const int dj = (int)(((float)rem + 0.5f) * __fdividef(1.0f, (float)w2));
    const int j = (int)(bx & 1023u) + dj, l = (int)((bx >> 10) & 1023u) + rem - dj * w2;
    x = m == 0 ? c : j;
    y = m == 1 ? c : (m == 0 ? j : l);
    z = m == 2 ? c : l;
    return true;
  }
  int j0, j1, l0, l1;
  slab_box(am, a1, a2, p.w0.w, p.w1.w, p.w2.x, p.w2.y, p.w2.z, p.w2.w, n, c, j0, j1, l0, l1);
  const int w2 = (bits & (1u << 29)) ? l1 - l0 + 1 : W2;
  // an approximate reciprocal suffices: (rem + 1/2) / w2 lies at least 1/(2 w2)
  // from an integer and rem < 256
  const float inv_w2 = (bits & (1u << 29)) ? __fdividef(1.0f, (float)w2) : p.w3.y;
  const int dj = (int)(((float)rem + 0.5f) * inv_w2);
  const int dl = rem - dj * w2;
  const int j = j0 + dj, l = l0 + dl;
  if (j > j1 || l > l1) return false;
  x = m == 0 ? c : j;
  y = m == 1 ? c : (m == 0 ? j : l);
  z = m == 2 ? c : l;
  return true;
}

// Queue the (segment, voxel) pairs of the lanes with q set for the exact
// decision, one atomic per warp (all lanes call).
__device__ __forceinline__ void queue_exact(const GridDev& g, bool q, uint32_t seg, int x, int y,
                                            int z, int lane) {
  const unsigned m = __ballot_sync(FULLW, q);
  if (!m) return;
  uint32_t base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(&g.st->xq_cnt, (uint32_t)__popc(m));
  base = __shfl_sync(FULLW, base, __ffs(m) - 1);
  if (q) {
    const uint32_t k = base + __popc(m & ((1u << lane) - 1u));
    if (k < g.xq_cap) g.xq[k] = make_uint2(seg, pack_voxel(x, y, z));
    else set_err(g.st, kErrOverflow);
  }
}

// The block's pass-1 counters into the status, three atomics per block (all
// threads of the block call).
__device__ __forceinline__ void flush_counters_block(DevStatus* st, unsigned long long F,
                                                     unsigned long long q, unsigned long long ex) {
  __shared__ unsigned long long s_c[3][8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F += __shfl_down_sync(FULLW, F, o);
    q += __shfl_down_sync(FULLW, q, o);
    ex += __shfl_down_sync(FULLW, ex, o);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_c[0][wid] = F;
    s_c[1][wid] = q;
    s_c[2][wid] = ex;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    unsigned long long v = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += s_c[threadIdx.x][k];
    if (v) atomicAdd(threadIdx.x == 0 ? &st->F : (threadIdx.x == 1 ? &st->sum_q : &st->exact_decisions), v);
  }
}

__device__ __forceinline__ void flush_counters(DevStatus* st, unsigned long long F,
                                               unsigned long long q, unsigned long long ex) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F += __shfl_down_sync(FULLW, F, o);
    q += __shfl_down_sync(FULLW, q, o);
    ex += __shfl_down_sync(FULLW, ex, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (F) atomicAdd(&st->F, F);
    if (q) atomicAdd(&st->sum_q, q);
    if (ex) atomicAdd(&st->exact_decisions, ex);
  }
}

// The packed-word increment (occupancy code << 16) | 1 of one fragment (Alg. 3
// at the voxel centre, quantized); counts it in F and sq.
__device__ __forceinline__ uint32_t fragment_word(const GridDev& g, float3 a, float3 b, float3 n0,
                                                  float3 n1, bool en0, bool en1, int x, int y,
                                                  int z, unsigned long long& F,
                                                  unsigned long long& sq) {
  const float3 o = make_float3((float)x, (float)y, (float)z);
  const float occ = capsule_occupancy(make_float3(0.5f, 0.5f, 0.5f), a - o, b - o, n0, n1, en0,
                                      en1, g.r_clamp, g.corr);
  const uint32_t q = (uint32_t)floorf(fmaf(g.occ_scale, occ, 0.5f));
  F += 1;
  sq += q;
  return (q << 16) | 1u;
}

// Adds a fragment to its voxel's packed word; returns its rank in the voxel.
__device__ __forceinline__ uint32_t add_fragment(const GridDev& g, float3 a, float3 b, float3 n0,
                                                 float3 n1, bool en0, bool en1, int x, int y,
                                                 int z, unsigned long long& F,
                                                 unsigned long long& sq) {
  return atomicAdd(&g.word[brick_index(x, y, z, g.log2nb)],
                   fragment_word(g, a, b, n0, n1, en0, en1, x, y, z, F, sq)) & 0xffffu;
}

// A record slot pass 1 took for a candidate it did not keep.
constexpr unsigned long long kNoRecord = ~0ull;

__device__ __forceinline__ void append_record(const GridDev& g, uint32_t idx, uint32_t seg,
                                              uint32_t rank) {
  const unsigned long long r = atomicAdd(&g.st->rec_cnt, 1ull);
  if (r < g.rec_cap) {
    g.rec[r] = ((unsigned long long)idx << 32) | seg;
    g.rank[r] = (uint16_t)rank;
  } else {
    set_err(g.st, kErrOverflow);
  }
}

constexpr int kWarpRecords = 256;  // pass 2: culled records a warp stages per append
constexpr uint32_t kNoCopy = 0xffffffffu;  // cq_cnt: pass 2 copied no culled records

// Append a warp's staged culled records to cq (all lanes call); records past
// the queue's capacity are counted but dropped, which sends the repair rounds
// back to the full record stream.
__device__ __forceinline__ void flush_culled(const GridDev& g, unsigned long long* cq,
                                             const unsigned long long* srec, int n, int lane) {
  if (n == 0) return;
  uint32_t r0 = 0;
  if (lane == 0) r0 = atomicAdd(&g.st->cq_cnt, (uint32_t)n);
  r0 = __shfl_sync(FULLW, r0, 0);
  for (int k = lane; k < n; k += 32) {
    const uint32_t r = r0 + (uint32_t)k;
    if (r < g.xq_cap) cq[r] = srec[k];
  }
  __syncwarp();
}

__global__ void __launch_bounds__(256) k_pass1(const float4* __restrict__ pos,
                                               const float4* __restrict__ nrm,
                                               const uint32_t* __restrict__ order, long long V,
                                               GridDev g) {
  const int lane = threadIdx.x & 31;
  const long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
  // slots in spatial order (nearby segments in the same and neighbouring
  // warps keep the packed-word atomics within a smaller part of the grid)
  const long long k = base + lane;
  const long long i = k < V ? (order ? (long long)__ldg(&order[k]) : k) : V;
  Walk w;
  w.n = 0;
  float3 n0 = make_float3(0.f, 0.f, 0.f), n1 = n0;
  uint32_t en = 0;
  if (i + 1 < V) {
    const float4 p0 = pos[i];
    const uint32_t f0 = __float_as_uint(p0.w);
    if (!(f0 & kLast)) {
      const float4 p1 = pos[i + 1];
      walk_setup(f3(p0), f3(p1), g, w);
      n0 = f3(nrm[i]);
      n1 = f3(nrm[i + 1]);
      en = ((f0 & kClipOn) ? 1u : 0u) | ((__float_as_uint(p1.w) & kClipOn) ? 2u : 0u);
    }
  }
  unsigned long long F = 0, sq = 0, ex = 0;
  const unsigned lt = (1u << lane) - 1u;
  // every lane's walk, packed, read by the lanes that take its candidates
  __shared__ PackedWalk s_w[256];
  __shared__ float4 s_n[2][256];  // clip normals at v0 and v1
  __shared__ uint32_t s_seg[256];  // segment id of each lane's walk
  const int tid = threadIdx.x, wb = tid & ~31;
  uint32_t wcount = 0;  // records this warp has written (uniform)
  // segment id of lane j's walk
  auto seg_of = [&](int j) { return order ? s_seg[wb + j] : (uint32_t)(base + j); };
  // The warp's candidates, segment after segment, are numbered 0..total-1;
  // lane l takes number t0 + l and finds its segment by a binary search over
  // the inclusive prefix of the candidate counts.
  uint32_t incl = w.n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(FULLW, incl, o);
    if (lane >= o) incl += v;
  }
  const uint32_t total = __shfl_sync(FULLW, incl, 31);
  // record slots: one atomic per block for all its candidates, warp shares in
  // warp order (a fragment per warp step took 2-3 flushes of staged records
  // per warp on one global counter, which contended)
  __shared__ uint32_t s_wtot[8];
  __shared__ unsigned long long s_rbase;
  const int wid = threadIdx.x >> 5;
  if (lane == 0) s_wtot[wid] = total;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t sum = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      const uint32_t t = s_wtot[k];
      s_wtot[k] = sum;
      sum += t;
    }
    s_rbase = sum ? atomicAdd(&g.st->rec_cnt, (unsigned long long)sum) : 0ull;
  }
  __syncthreads();
  const unsigned long long rbase = s_rbase + s_wtot[wid];
  if (w.n) {
    if (order) s_seg[tid] = (uint32_t)i;
    s_w[tid] = pack_walk(w, en, incl - w.n);
    s_n[0][tid] = make_float4(n0.x, n0.y, n0.z, 0.0f);
    s_n[1][tid] = make_float4(n1.x, n1.y, n1.z, 0.0f);
  }
  __syncwarp();
  // Candidates the first filter stage leaves undecided (a few percent) wait in
  // a per-warp queue and get the Newton stage 32 at a time, so the warp does
  // not run it for one or two lanes per step.
  __shared__ uint2 s_uq[8][64];  // (owner lane, packed voxel)
  uint2* uq = s_uq[threadIdx.x >> 5];
  uint32_t un = 0;  // queued (uniform)
  // A fragment's rank is stored one emit later, so the latency of the
  // returning atomic that gives it overlaps a step of work: pend_r is the
  // record slot still waiting for its rank, the count field of the word
  // pend_old that the lane's atomic returned.
  unsigned long long pend_r = ~0ull;
  uint32_t pend_old = 0;
  auto flush_rank = [&]() {  // all lanes call
    if (pend_r < g.rec_cap) g.rank[pend_r] = (uint16_t)pend_old;  // low 16 bits: count
    pend_r = ~0ull;
  };
  // a kept fragment: occupancy into the packed word, record written (all lanes call)
  auto emit = [&](bool keep, int j, const PackedWalk& p, int x, int y, int z) {
    uint32_t idx = 0;
    flush_rank();
    const unsigned am = __ballot_sync(FULLW, keep);
    if (keep) {
      idx = brick_index(x, y, z, g.log2nb);
      const uint32_t clip = __float_as_uint(p.w3.z) >> 27;
      const uint32_t inc = fragment_word(g, f3(p.w0), f3(p.w1), f3(s_n[0][wb + j]),
                                         f3(s_n[1][wb + j]), clip & 1u, clip & 2u, x, y, z, F, sq);
      pend_old = atomicAdd(&g.word[idx], inc);
    }
    if (keep) {
      const unsigned long long r = rbase + wcount + __popc(am & lt);
      if (r < g.rec_cap) {
        g.rec[r] = ((unsigned long long)idx << 32) | seg_of(j);
        pend_r = r;
      } else {
        set_err(g.st, kErrOverflow);
      }
    }
    wcount += __popc(am);
  };
  // stage 2 for queued entries below cnt (all lanes call)
  auto stage2 = [&](uint32_t cnt) {
    int dec = 0, j = 0, x = 0, y = 0, z = 0;
    PackedWalk p;
    if ((uint32_t)lane < cnt) {
      const uint2 it = uq[lane];
      j = (int)it.x;
      unpack_voxel(it.y, x, y, z);
      p = s_w[wb + j];
      dec = g.force_exact ? -1 : seg_stage2_at(f3(p.w0), f3(p.w1), x, y, z, g.rl);
      if (dec < 0) ++ex;
    }
    queue_exact(g, dec < 0, (uint32_t)lane < cnt ? seg_of(j) : 0u, x, y, z, lane);
    emit(dec > 0, j, p, x, y, z);
  };
  for (uint32_t t0 = 0; t0 < total; t0 += 32) {
    const uint32_t gq = t0 + lane;
    int j = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1)
      if (__shfl_sync(FULLW, incl, j + st - 1) <= gq) j += st;
    j = min(j, 31);
    int x = 0, y = 0, z = 0, dec = 0;
    PackedWalk p;
    if (gq < total) {
      p = s_w[wb + j];
      // with the force_exact test option every pair goes on to the exact path
      if (decode_candidate(p, g.n, gq - __float_as_uint(p.w3.w), x, y, z))
        dec = g.force_exact ? -1 : seg_stage1_at(f3(p.w0), f3(p.w1), x, y, z, g.rl);
    }
    const unsigned um = __ballot_sync(FULLW, dec < 0);
    if (dec < 0) uq[un + __popc(um & lt)] = make_uint2((uint32_t)j, pack_voxel(x, y, z));
    un += __popc(um);
    emit(dec > 0, j, p, x, y, z);
    if (un >= 32) {
      __syncwarp();
      stage2(32);
      __syncwarp();
      // entries past the first 32 move to the front (reads 32.., writes ..31)
      if ((uint32_t)lane < un - 32) uq[lane] = uq[32 + lane];
      __syncwarp();
      un -= 32;
    }
  }
  __syncwarp();
  stage2(un);
  flush_rank();
  for (uint32_t k = wcount + lane; k < total; k += 32) {  // slots of candidates not kept
    const unsigned long long r = rbase + k;
    if (r < g.rec_cap) g.rec[r] = kNoRecord;
  }
  flush_counters_block(g.st, F, sq, ex);
}

// Exact decisions of pass 1's undecided pairs.
__global__ void __launch_bounds__(256) k_exact1(const float4* __restrict__ pos,
                                                const float4* __restrict__ nrm, GridDev g) {
  const uint32_t cnt = min(g.st->xq_cnt, g.xq_cap);
  unsigned long long F = 0, sq = 0;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const uint2 it = g.xq[e];
    int x, y, z;
    unpack_voxel(it.y, x, y, z);
    const float4 p0 = pos[it.x], p1 = pos[it.x + 1];
    if (!seg_exact_at(f3(p0), f3(p1), x, y, z, g.RL)) continue;
    const uint32_t rank =
        add_fragment(g, f3(p0), f3(p1), f3(nrm[it.x]), f3(nrm[it.x + 1]),
                     __float_as_uint(p0.w) & kClipOn, __float_as_uint(p1.w) & kClipOn, x, y, z, F, sq);
    append_record(g, brick_index(x, y, z, g.log2nb), it.x, rank);
  }
  unsigned long long z0 = 0;
  flush_counters(g.st, F, sq, z0);
}

__device__ __forceinline__ bool bit_set(const uint32_t* bits, uint32_t i) {
  return (bits[i >> 5] >> (i & 31)) & 1u;
}

// Pass 2: stream the fragment records; mode 0 lists every fragment, mode 1
// those whose voxel the cull marked, mode 2 (repair) those whose voxel's
// `need` bit is set. Modes 0 and 1 read the voxel's list end from the scan's
// cursor -- kCulledStart when the cull gave it no list -- and write the segment
// id at end - 1 - rank: no atomic, and the cursor carries the cull's decision, so the
// mark is not read. The repair, whose copied records carry no rank, bumps the
// cursor of each listed voxel from its list start with a returning atomic.
// Mode 1 also copies the records of unmarked voxels to the (by then unused)
// exact-path queue, warp-staged, so that the repair rounds stream only those;
// when they do not all fit, the repair streams every record. The copy is made
// only when under half of the fragments are culled: past that, a repair round
// streaming every record reads less than twice the bytes the copy would write
// in every frame, and repairs are rare (ABC pathlines at 512^3 cull 97% of their
// fragments and need none); k_scatter_culled lists the fragments of such a
// build instead.
__global__ void __launch_bounds__(256) k_scatter(GridDev g, int mode, const uint32_t* __restrict__ need,
                                                 const uint32_t* __restrict__ pending) {
  if (mode == 2 && *pending == 0) return;
  __shared__ unsigned long long s_rec[8][kWarpRecords];
  unsigned long long* cq = reinterpret_cast<unsigned long long*>(g.xq);
  bool copy = false;  // mode 1: copy the culled records (grid-uniform)
  if (mode == 1) {
    const unsigned long long F = g.st->F, culled = F - g.st->list_tail;
    copy = 2 * culled < F;
    if (!copy) return;  // k_scatter_culled's build
  }
  const bool compact = mode == 2 && g.st->cq_cnt != kNoCopy && g.st->cq_cnt <= g.xq_cap;
  const unsigned long long* src = compact ? cq : g.rec;
  const unsigned long long cnt =
      compact ? g.st->cq_cnt : min(g.st->rec_cnt, (unsigned long long)g.rec_cap);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long* srec = s_rec[threadIdx.x >> 5];
  int wcount = 0;  // culled records staged by this warp (mode 1, uniform)
  unsigned long long listed = 0;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  for (unsigned long long e0 = warp * 32ull; e0 < cnt; e0 += n_warps * 32ull) {
    const unsigned long long e = e0 + lane;
    bool skip = true, have = false;
    unsigned long long r = 0;
    uint32_t rank = 0;
    if (e < cnt) {
      r = __ldcs(&src[e]);
      if (mode != 2) rank = __ldcs(&g.rank[e]);
    }
    if (e < cnt && r != kNoRecord) {
      have = true;
      const uint32_t idx = (uint32_t)(r >> 32);
      uint32_t slot = 0;
      if (mode != 2) {
        const uint32_t end = __ldg(&g.cur[idx]);
        skip = end >= kCulledStart;
        slot = end - 1u - rank;
      } else {
        skip = !bit_set(need, idx);
        if (!skip) slot = atomicAdd(&g.cur[idx], 1u);
      }
      if (!skip) {
        if (slot < g.list_cap) {
          g.lists[slot] = (uint32_t)r;
          ++listed;
        } else {
          set_err(g.st, kErrOverflow);
        }
      }
    }
    if (copy) {
      const bool keep = have && skip;
      const unsigned km = __ballot_sync(FULLW, keep);
      if (keep) srec[wcount + __popc(km & lt)] = r;
      wcount += __popc(km);
      if (wcount > kWarpRecords - 32) {
        __syncwarp();
        flush_culled(g, cq, srec, wcount, lane);
        wcount = 0;
      }
    }
  }
  if (copy) {
    __syncwarp();
    flush_culled(g, cq, srec, wcount, lane);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) listed += __shfl_down_sync(FULLW, listed, o);
  if (lane == 0 && listed) atomicAdd(&g.st->listed, listed);
}

// Pass 2 (mode 1) of a build whose cull dropped at least half of the
// fragments, which k_scatter leaves to it: no culled-record copy, and mostly
// reads, so a warp takes 4 x 32 consecutive records per round, each lane one
// of every 32, and loads the lane's four records, then their list ends,
// together -- four independent load chains in flight per lane (ABC pathlines
// at 512^3: pass 2 0.71 -> 0.47 ms; where most fragments are listed, four
// rounds' scattered list stores at once measured slower: bundles 0.90 -> 1.11).
__global__ void __launch_bounds__(256) k_scatter_culled(GridDev g) {
  const unsigned long long F = g.st->F;
  if (2 * (F - g.st->list_tail) < F) return;  // k_scatter's build
  if (blockIdx.x == 0 && threadIdx.x == 0) g.st->cq_cnt = kNoCopy;
  const unsigned long long cnt = min(g.st->rec_cnt, (unsigned long long)g.rec_cap);
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long listed = 0;
  for (unsigned long long e0 = warp * (32ull * U); e0 < cnt; e0 += n_warps * (32ull * U)) {
    unsigned long long r[U];
    uint32_t rank[U], end[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned long long e = e0 + 32ull * u + lane;
      r[u] = e < cnt ? __ldcs(&g.rec[e]) : kNoRecord;
      rank[u] = e < cnt ? (uint32_t)__ldcs(&g.rank[e]) : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      end[u] = r[u] != kNoRecord ? __ldg(&g.cur[(uint32_t)(r[u] >> 32)]) : kCulledStart;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (end[u] >= kCulledStart) continue;  // no record, or the cull gave its voxel no list
      const uint32_t slot = end[u] - 1u - rank[u];
      if (slot < g.list_cap) {
        g.lists[slot] = (uint32_t)r[u];
        ++listed;
      } else {
        set_err(g.st, kErrOverflow);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) listed += __shfl_down_sync(FULLW, listed, o);
  if (lane == 0 && listed) atomicAdd(&g.st->listed, listed);
}

int launch_pass1(const float4* pos, const float4* nrm, const uint32_t* order, long long V,
                 const GridDev& g, cudaStream_t s) {
  if (V < 2) return 0;
  const int T = 256;
  // One atomic per fragment at every grid side: summing the increments of the
  // lanes of a warp step that share a voxel first (a match on the voxel index)
  // measured slower at 256^3 (bundles pass 1 2.3 -> 3.5 ms) and, since pass 1's
  // atomics return the rank, at 512^3 too (ABC pathlines 4.70 -> 6.83 ms; it
  // paid there while they returned nothing, 7.8 -> 7.4 ms).
  k_pass1<<<(unsigned)((V + T - 1) / T), T, 0, s>>>(pos, nrm, order, V, g);
  k_exact1<<<152 * 4, T, 0, s>>>(pos, nrm, g);
  return 2;
}

int launch_scatter(const GridDev& g, int mode, const uint32_t* need, const uint32_t* pending,
                   cudaStream_t s) {
  if (mode == 1) k_scatter_culled<<<152 * 8, 256, 0, s>>>(g);
  k_scatter<<<152 * 8, 256, 0, s>>>(g, mode, need, pending);
  return mode == 1 ? 2 : 1;
}

}  // namespace vrt
