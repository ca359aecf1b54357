// A4: per-voxel list offsets by an exclusive prefix sum over the counts of the
// voxels that receive a list (Sec. 3.3; the first half of the linearized
// layered fragment buffer it extends). Single-pass decoupled look-back scan:
// tiles take ids in launch order from an atomic counter, publish their
// aggregate, then their inclusive prefix once a warp has looked back to a
// published prefix. Every wait is bounded; a wait that gives up sets the
// timeout bit and the tile carries on with the sum it has.
//
// The same pass checks the packed words: the sums of the count and occupancy
// fields over all voxels must equal the fragment and occupancy totals that
// pass 1 accumulated separately, otherwise a 16-bit field overflowed. It also
// marks bricks that hold an occupied voxel (for empty-space skipping).
#include "launch.h"

namespace vrt {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 voxels = 64 bricks
constexpr unsigned long long kFlagAgg = 1ull << 32, kFlagPrefix = 2ull << 32;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ unsigned long long load_state(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}

__global__ void __launch_bounds__(kScanThreads) k_scan(GridDev g, int all_visible,
                                                       unsigned long long* tile_state,
                                                       uint32_t n_tiles, int stall_tile,
                                                       int spin_limit) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_prefix;
  __shared__ unsigned long long s_red[4][kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(&g.st->scan_tile_counter, 1u);
  }
  __syncthreads();
  const uint32_t tile = s_tile;
  const size_t base = (size_t)tile * kScanTile + (size_t)tid * kScanItems;

  uint32_t w[kScanItems];
  const uint4* src = reinterpret_cast<const uint4*>(g.word + base);
#pragma unroll
  for (int q = 0; q < kScanItems / 4; ++q) {
    const uint4 v = src[q];
    w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
  }
  const uint32_t visw = all_visible ? 0xffffu : (g.vis[base >> 5] >> (base & 31)) & 0xffffu;
  uint32_t val[kScanItems];
  uint32_t sum = 0, occupied = 0, visible = 0, maxc = 0;
  unsigned long long cf = 0, of = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const uint32_t c = w[k] & 0xffffu;
    cf += c;
    of += w[k] >> 16;
    occupied += c != 0;
    maxc = max(maxc, c);
    val[k] = ((visw >> k) & 1u) ? c : 0u;
    visible += val[k] != 0;
    sum += val[k];
  }
  // block exclusive scan of per-thread sums
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t warp_off = 0, agg = 0;
#pragma unroll
  for (int q = 0; q < kScanThreads / 32; ++q) {
    const uint32_t v = s_warp[q];
    if (q < warp) warp_off += v;
    agg += v;
  }
  const uint32_t thread_excl = warp_off + incl - sum;

  // decoupled look-back (warp 0); a stalled tile (testing) publishes nothing,
  // so the waits of the tiles after it run out
  const bool publish = (int)tile != stall_tile;
  if (warp == 0) {
    uint32_t excl = 0;
    if (tile == 0) {
      if (lane == 0 && publish) atomicExch(&tile_state[0], kFlagPrefix | agg);
    } else {
      if (lane == 0 && publish) atomicExch(&tile_state[tile], kFlagAgg | agg);
      long long j = (long long)tile - 1;
      int spins = 0;
      bool done = false;
      while (!done) {
        const long long idx = j - lane;
        unsigned long long s = idx >= 0 ? load_state(&tile_state[idx]) : (kFlagPrefix | 0ull);
        // wait until every lane sees a published state
        while (__any_sync(0xffffffffu, (s >> 32) == 0)) {
          if (++spins > spin_limit) break;
          if ((s >> 32) == 0) {
            __nanosleep(64);
            s = load_state(&tile_state[idx]);
          }
        }
        if (spins > spin_limit) {
          if (lane == 0) set_err(g.st, kErrTimeout);
          break;
        }
        const uint32_t pmask = __ballot_sync(0xffffffffu, (s >> 32) == 2);
        const int stop = pmask ? __ffs(pmask) - 1 : 31;  // nearest published prefix
        uint32_t v = lane <= stop ? (uint32_t)s : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        done = pmask != 0;
        j -= 32;
      }
      if (lane == 0 && publish) atomicExch(&tile_state[tile], kFlagPrefix | (excl + agg));
    }
    if (lane == 0) {
      s_prefix = excl;
      if (tile == n_tiles - 1) {
        const unsigned long long total = (unsigned long long)excl + agg;
        g.st->list_tail = (uint32_t)total;
        if (total > g.list_cap) set_err(g.st, kErrOverflow);
      }
    }
  }
  __syncthreads();
  uint32_t run = s_prefix + thread_excl;
  uint32_t outv[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    run += val[k];
    outv[k] = ((visw >> k) & 1u) ? run : kCulledStart;  // list end (pass 2 fills below it)
  }
  uint4* dst = reinterpret_cast<uint4*>(g.cur + base);
#pragma unroll
  for (int q = 0; q < kScanItems / 4; ++q)
    dst[q] = make_uint4(outv[4 * q], outv[4 * q + 1], outv[4 * q + 2], outv[4 * q + 3]);

  // counters
  unsigned long long r0 = cf, r1 = of, r2 = ((unsigned long long)visible << 32) | occupied;
  uint32_t mc = maxc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r0 += __shfl_xor_sync(0xffffffffu, r0, o);
    r1 += __shfl_xor_sync(0xffffffffu, r1, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
  }
  if (lane == 0) {
    s_red[0][warp] = r0; s_red[1][warp] = r1; s_red[2][warp] = r2; s_red[3][warp] = mc;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int q = 0; q < kScanThreads / 32; ++q) {
      a0 += s_red[0][q]; a1 += s_red[1][q]; a2 += s_red[2][q];
      a3 = max(a3, s_red[3][q]);
    }
    if (a0) atomicAdd(&g.st->sum_count_field, a0);
    if (a1) atomicAdd(&g.st->sum_occ_field, a1);
    if (a2 & 0xffffffffull) atomicAdd(&g.st->occupied_voxels, (uint32_t)(a2 & 0xffffffffull));
    if (a2 >> 32) atomicAdd(&g.st->visible_voxels, (uint32_t)(a2 >> 32));
    atomicMax(&g.st->max_count, (uint32_t)a3);
  }
}

__global__ void k_finalize(GridDev g) {
  DevStatus* st = g.st;
  if (st->sum_count_field != st->F || st->sum_occ_field != st->sum_q) set_err(st, kErrOverflow);
}

int launch_scan(const GridDev& g, int all_visible, unsigned long long* tile_state, uint32_t n_tiles,
                int stall_tile, int spin_limit, cudaStream_t s) {
  k_scan<<<n_tiles, kScanThreads, 0, s>>>(g, all_visible, tile_state, n_tiles, stall_tile,
                                          spin_limit > 0 ? spin_limit : kSpinLimit);
  return 1;
}

int launch_finalize(const GridDev& g, cudaStream_t s) {
  k_finalize<<<1, 1, 0, s>>>(g);
  return 1;
}

}  // namespace vrt
