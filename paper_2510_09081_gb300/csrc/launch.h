// Host-side launch wrappers of the libvrt kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vrt.h"
#include "vrt_internal.cuh"

namespace vrt {

// Camera as given through the C ABI, widened to fp64 on the host.
struct HostCamera {
  int width, height, ortho;
  double eye[3], target[3], up[3], fovy_deg, ortho_h;
};

// Camera in the form the trace kernel consumes (built on the host in fp64).
struct CamDev {
  float3 o0, ox, oy;  // origin: o0 (+ (px+.5) ox + (py+.5) oy when orthographic)
  float3 d0, dx, dy;  // direction: d0 + (px+.5) dx + (py+.5) dy, normalised
  int width, height, ortho;
};

struct TraceArgs {
  GridDev g;
  CamDev cam;
  const float4* pos;
  const float4* nrm;
  uint32_t n_vert;           // vertices; list entries must be < n_vert - 1
  float alpha;
  int ao;                    // per-hit shading: 0 none, 1 cone AO, 2 voxel-space field
  const void* mips;          // occupancy pyramid, texels in format mips_fmt
  int mips_fmt;              // kMipsF32, kMipsF16 or kMipsBF16
  long long lev_off[11];
  int n_levels;
  float4* rgba;
  int* first_id;
  float* first_t;
  const uint32_t* pix_list;  // trace only these pixels (repair) when non-null
  const uint32_t* pix_count; // number of entries of pix_list (device)
  uint32_t* need;            // [n^3 / 32] voxels queued for listing
  uint32_t* vq;              // out: queued voxels
  uint32_t* vq_cnt;
  uint32_t* pq;              // out: pixels to trace again
  uint32_t* pq_cnt;
  uint32_t vq_cap, pq_cap;
  uint32_t max_queue;        // culled voxels one ray may queue before it stops
  uint32_t* work_next;       // next work item (persistent warps)
  float4* resume;            // [2 * pixels] state of a ray at its first culled voxel:
                             // (C, T), (first id bits, first t, voxel index bits, entry t)
  uint32_t short_list;       // lists up to this length share the warp entry by entry
  uint32_t ray_keys;         // hit slots per transparent ray on that path (<= kRayKeys)
  int key16;                 // order hits by the paper's 16+16-bit per-voxel key
  int tile_w;                // transparent trace: warp tile width (2, 4, 8 or 16 pixels)
  int count;                 // accumulate trace work counters
  uint32_t* touch_list;      // instrumented trace: bit per list entry read
  uint32_t* touch_vert;      //   bit per vertex read (segment end points)
  uint32_t* touch_vox;       //   bit per voxel whose words the DDA read
  const float* shade;        // voxel-space shading field [n^3] (brick order), or null
};

// Voxel-space shading (Sec. 3.4, Shading): per voxel, cone AO at its centre
// times 1/2 + 1/2 * the transmittance of a ray toward the light through the
// base occupancy level, for every voxel within one step (26-neighbourhood) of a
// listed voxel -- the voxels whose centres a trilinear sample at a hit reads.
struct ShadeArgs {
  GridDev g;
  const void* mips;          // occupancy pyramid (format mips_fmt)
  int mips_fmt;
  long long lev_off[11];
  int n_levels;
  int ao;                    // 1: include the cone AO
  float lx, ly, lz;          // unit direction toward the light
  float* shade;              // [n^3] shading value per voxel (brick order)
  uint32_t* mask;            // [n^3 / 32] voxels whose value is current this frame
  const uint32_t* vq;        // repair: voxels listed in this round
  const uint32_t* vq_cnt;
  uint32_t vq_cap;
};
// Every voxel next to a listed one (one block per brick); rewrites the mask.
int launch_shade(const ShadeArgs& a, cudaStream_t s);
// Voxels next to the voxels a repair round listed, not yet shaded this frame.
int launch_shade_repair(const ShadeArgs& a, cudaStream_t s);

// Ingest of vertices [lo, hi) (nothing when hi <= lo).
int launch_ingest(const float* raw, const uint8_t* flags, long long lo, long long hi, float4* pos,
                  float4* nrm, DevStatus* st, cudaStream_t s);
// Pass 1 over the segments in the order `order` (V vertex indices, each
// polyline's vertices consecutive; a polyline's last vertex starts no
// segment), or in index order when `order` is null.
int launch_pass1(const float4* pos, const float4* nrm, const uint32_t* order, long long V,
                 const GridDev& g, cudaStream_t s);
// 12-bit spatial keys (Morton code of the 16^3 cell) of the vertices mid[0..P).
int launch_poly_keys(const float* raw, const uint32_t* mid, uint32_t P, int n, uint16_t* key,
                     cudaStream_t s);
// Empty-brick distance field from the counts of pass 1 (tmp: one byte per brick).
int launch_brick_dist(const GridDev& g, uint8_t* tmp, uint8_t* dist, cudaStream_t s);
// The three distance passes from per-brick bytes in tmp (0 = occupied, else
// kBrickDistMax); tmp is overwritten.
int launch_brick_dist_passes(int log2nb, uint8_t* tmp, uint8_t* dist, cudaStream_t s);
// Pass 2 over the fragment records. mode 0: every occupied voxel has a list;
// 1: voxels marked by the cull; 2: repair, only voxels whose `need` bit is set
// (skipped when *pending is 0).
int launch_scatter(const GridDev& g, int mode, const uint32_t* need, const uint32_t* pending,
                   cudaStream_t s);
// stall_tile >= 0 (testing): that tile never publishes its look-back state,
// so the tiles after it give up their waits after spin_limit polls.
int launch_scan(const GridDev& g, int all_visible, unsigned long long* tile_state, uint32_t n_tiles,
                int stall_tile, int spin_limit, cudaStream_t s);
int launch_finalize(const GridDev& g, cudaStream_t s);
int launch_mips(const GridDev& g, void* mips, int fmt, const long long* lev_off, int n_levels,
                cudaStream_t s);
// Cull marks; btmp, cdist: one byte per brick (scratch; distance to a brick
// with eroded occupancy); emean: one float per brick (mean eroded occupancy);
// depth_max: estimated optical depth past which a voxel is culled (<= 0: the
// default, ln(1e4) + 3); occq: scratch for the indices of the occupied voxels
// (occq_cap entries; when fewer than n^3, every voxel's thread tests its own).
int launch_cull(const GridDev& g, const HostCamera& cam, float alpha, uint8_t* eroded,
                uint8_t* btmp, uint8_t* cdist, float* emean, float depth_max, uint32_t* occq,
                unsigned long long occq_cap, cudaStream_t s);
int launch_trace(const TraceArgs& a, int K, cudaStream_t s);
// Instrumented trace: the set bits of the three touch bitmaps into
// st->tr_u_entries, tr_u_vertices, tr_u_voxels (which the caller cleared).
int launch_touch_count(const uint32_t* list_bits, size_t list_words, const uint32_t* vert_bits,
                       size_t vert_words, const uint32_t* vox_bits, size_t vox_words,
                       DevStatus* st, cudaStream_t s);
// Repair round: list the voxels of vq (count *vq_cnt), pass 2 restricted to
// them, then clear their `need` bits and the next round's queue counters.
int launch_repair_alloc(const GridDev& g, const uint32_t* vq, const uint32_t* vq_cnt,
                        const uint32_t* pq_cnt, uint32_t vq_cap, cudaStream_t s);
int launch_repair_clear(const GridDev& g, uint32_t* need, const uint32_t* vq,
                         const uint32_t* vq_cnt, uint32_t vq_cap, int next, cudaStream_t s);

// Host-side checks shared by the C ABI and the serving loop: nullptr when the
// camera and render parameters are acceptable to vrt_cull and vrt_trace, else
// what is wrong.
const char* frame_args_error(const vrt_camera* cam, const vrt_render_params* p);

// Allocate every buffer a frame of `g` with these parameters sizes lazily, so
// that the frame's calls allocate nothing and can be captured into a CUDA
// graph (may synchronize the grid's stream).
vrt_status prepare_frame(vrt_grid g, const vrt_camera* cam, const vrt_render_params* p);

// Testing hook of vrt_scan_counts_noalloc (vrt_set_option(NULL,
// VRT_OPT_TEST_SCAN_STALL, tile)): tile >= 0 makes that look-back tile skip
// its publish and shortens every wait; -1 restores the normal scan.
void set_noalloc_scan_stall(long long tile);

constexpr int kSpinLimitTest = 1 << 10;  // look-back polls while a test stalls a tile

}  // namespace vrt
