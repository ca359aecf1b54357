// vrt_scan_counts_noalloc: the list-offset scan as a stand-alone entry point
// that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the scan:
// code running inside a memory pool or arena that owns all device memory of
// the process, callers that must not fragment or grow memory mid-frame, and
// real-time loops where an allocation could block on the driver. This variant
// takes the look-back scratch (one 64-bit state per tile and a tile counter)
// from a fixed file-scope device array instead of a caller or library
// allocation. The array is part of the library image, so every GPU that loads
// the library holds it (about 256 KB) until the process exits.
//
// The kernel is a variant of the grid scan (decoupled look-back over tiles of
// 4096 voxels); it computes the exclusive prefix sum of the per-voxel counts
// (low 16 bits of each packed word) of marked voxels, and their total. The
// look-back carries 62-bit sums (a 2-bit flag above them), so a total beyond
// 2^32 - 1, where the 32-bit offsets wrap, is detected and reported.
#include <atomic>
#include <mutex>
#include <string>

#include "launch.h"
#include "vrt.h"

namespace vrt {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 16;
constexpr int kNaTile = kNaThreads * kNaItems;   // 4096 voxels
constexpr uint32_t kNaMaxTiles = 32768;          // 134,217,728 voxels (512^3)
// tile state: flag (0 none, 1 aggregate, 2 inclusive prefix) in bits 62-63,
// the 62-bit sum below it
constexpr unsigned long long kNaAgg = 1ull << 62, kNaPrefix = 2ull << 62;
constexpr unsigned long long kNaValue = (1ull << 62) - 1;
constexpr int kNaSpinLimit = 1 << 22;
// status bits of status_out
constexpr uint32_t kNaGaveUp = 1u, kNaWrapped = 2u;

// Scratch: tile states, then the tile counter. Shared by every call.
struct NoAllocScratch {
  unsigned long long state[kNaMaxTiles];
  unsigned int tile_counter;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__global__ void __launch_bounds__(kNaThreads) k_scan_noalloc(
    NoAllocScratch* scratch, const uint32_t* __restrict__ words, const uint32_t* __restrict__ marks,
    uint32_t* __restrict__ offsets, uint32_t* total_out, uint32_t* status_out, uint32_t n_tiles,
    int stall_tile, int spin_limit) {
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_warp[kNaThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(&scratch->tile_counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const size_t base = (size_t)tile * kNaTile + (size_t)tid * kNaItems;
  const uint32_t mw = marks ? (marks[base >> 5] >> (base & 31)) & 0xffffu : 0xffffu;
  uint32_t val[kNaItems];
  uint32_t sum = 0;  // at most 16 * 65535
  const uint4* src = reinterpret_cast<const uint4*>(words + base);
#pragma unroll
  for (int q = 0; q < kNaItems / 4; ++q) {
    const uint4 v = src[q];
    const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = 4 * q + k;
      val[i] = ((mw >> i) & 1u) ? (w4[k] & 0xffffu) : 0u;
      sum += val[i];
    }
  }
  uint32_t incl = sum;  // the tile's sums stay below 4096 * 65535 < 2^28
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t warp_off = 0, agg = 0;
#pragma unroll
  for (int q = 0; q < kNaThreads / 32; ++q) {
    if (q < warp) warp_off += s_warp[q];
    agg += s_warp[q];
  }
  // a stalled tile (testing) publishes nothing, so the waits after it run out
  const bool publish = (int)tile != stall_tile;
  if (warp == 0) {
    unsigned long long excl = 0;
    if (tile == 0) {
      if (lane == 0 && publish) atomicExch(&scratch->state[0], kNaPrefix | agg);
    } else {
      if (lane == 0 && publish) atomicExch(&scratch->state[tile], kNaAgg | agg);
      long long j = (long long)tile - 1;
      int spins = 0;
      for (;;) {
        const long long idx = j - lane;
        unsigned long long s =
            idx >= 0 ? *(volatile unsigned long long*)&scratch->state[idx] : (2ull << 62);
        while (__any_sync(0xffffffffu, (s >> 62) == 0) && ++spins <= spin_limit) {
          if ((s >> 62) == 0) {
            __nanosleep(64);
            s = *(volatile unsigned long long*)&scratch->state[idx];
          }
        }
        if (spins > spin_limit) {  // give up: report, publish what we have
          if (lane == 0 && status_out) atomicOr(status_out, kNaGaveUp);
          break;
        }
        const uint32_t pmask = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        const int stop = pmask ? __ffs(pmask) - 1 : 31;
        unsigned long long v = lane <= stop ? (s & kNaValue) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pmask) break;
        j -= 32;
      }
      if (lane == 0 && publish) atomicExch(&scratch->state[tile], kNaPrefix | ((excl + agg) & kNaValue));
    }
    if (lane == 0) {
      s_prefix = excl;
      if (tile == n_tiles - 1) {
        const unsigned long long total = excl + agg;
        if (total_out) *total_out = (uint32_t)total;
        if (total > 0xffffffffull && status_out) atomicOr(status_out, kNaWrapped);
      }
    }
  }
  __syncthreads();
  // offsets are the low 32 bits of the prefix sums (they wrap past 2^32 - 1)
  uint32_t run = (uint32_t)s_prefix + warp_off + incl - sum;
  uint32_t out[kNaItems];
#pragma unroll
  for (int i = 0; i < kNaItems; ++i) {
    out[i] = run;
    run += val[i];
  }
  uint4* dst = reinterpret_cast<uint4*>(offsets + base);
#pragma unroll
  for (int q = 0; q < kNaItems / 4; ++q)
    dst[q] = make_uint4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
}

// Testing: the tile that skips its publish (-1: none).
std::atomic<long long> g_stall_tile{-1};

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

void set_noalloc_scan_stall(long long tile) { g_stall_tile.store(tile); }

}  // namespace vrt

extern thread_local std::string g_create_error;  // message returned by vrt_last_error(NULL)

extern "C" vrt_status vrt_scan_counts_noalloc(const uint32_t* words, const uint32_t* marks,
                                              uint32_t* offsets, uint64_t n_voxels,
                                              uint32_t* total_out, uint32_t* status_out,
                                              void* cuda_stream) {
  using namespace vrt;
  auto fail = [](vrt_status s, const char* m) {
    g_create_error = m;
    return s;
  };
  if (!words || !offsets) return fail(VRT_ERR_INVALID_ARG, "words and offsets must not be NULL");
  if (n_voxels == 0 || n_voxels % kNaTile != 0)
    return fail(VRT_ERR_INVALID_ARG, "n_voxels must be a positive multiple of 4096");
  if (n_voxels > (uint64_t)kNaMaxTiles * kNaTile)
    return fail(VRT_ERR_INVALID_ARG,
                "n_voxels exceeds the no-allocation scan's fixed scratch (at most 134217728)");
  if (((uintptr_t)words | (uintptr_t)offsets) & 15u)
    return fail(VRT_ERR_INVALID_ARG, "words and offsets must be 16-byte aligned");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(VRT_ERR_CUDA, "cudaGetDevice failed");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return fail(VRT_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  const uint32_t n_tiles = (uint32_t)(n_voxels / kNaTile);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // states of the tiles this call uses, and the tile counter, start at zero
  NoAllocScratch* sc = (NoAllocScratch*)scratch;
  cudaError_t e = cudaMemsetAsync(sc->state, 0, sizeof(unsigned long long) * n_tiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&sc->tile_counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return fail(VRT_ERR_CUDA, cudaGetErrorString(e));
  const long long stall = g_stall_tile.load();
  k_scan_noalloc<<<n_tiles, kNaThreads, 0, s>>>(sc, words, marks, offsets, total_out, status_out,
                                               n_tiles, stall >= 0 ? (int)stall : -1,
                                               stall >= 0 ? kSpinLimitTest : kNaSpinLimit);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VRT_ERR_CUDA, cudaGetErrorString(e));
  return VRT_OK;
}
