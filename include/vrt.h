/*
 * vrt.h -- C ABI of the GB300 (sm_103a) voxel ray-tracing library for dynamic
 * line sets, after Kraaijeveld, Jalba, Vilanova & Chamberland, "Real-Time
 * Rendering of Dynamic Line Sets using Voxel Ray Tracing" (arXiv 2510.09081).
 *
 * The problem (Sec. 3, overview): a set of polylines (no branches, no loops)
 * with one uniform tube radius, and a camera, go in; an image of the tubes with
 * optional ambient occlusion and ground-truth transparency comes out. Every
 * acceleration structure is rebuilt each frame, so the vertices may change
 * arbitrarily between frames. One frame is
 *
 *   vrt_update_vertices (optional) -> vrt_voxelize -> vrt_build_mips (for AO)
 *     -> vrt_cull -> vrt_trace
 *
 * Conventions shared by every call:
 *  - Units: world coordinates are in voxels; the grid is [0, n)^3 and voxel
 *    (x, y, z) is the closed box [x, x+1] x [y, y+1] x [z, z+1]. Coordinates are
 *    snapped to multiples of 2^-14 voxel on ingest and must lie in [-256, 768).
 *  - Segment i joins vertex i to vertex i+1 of the same polyline (Sec. 3.3);
 *    segment ids in lists and outputs are these vertex indices.
 *  - Ordering: every call is asynchronous on the stream given at creation,
 *    except vrt_sync, vrt_get_stats and the vrt_read_* calls, which wait.
 *  - Ownership: the library owns all of its device buffers (grid words, list
 *    offsets, lists, pyramids, scratch). The caller owns its input and output
 *    buffers; inputs are copied, so the caller may reuse an input buffer once
 *    the call's stream work has completed.
 *  - Errors: a call returns VRT_OK or an error code at once for problems the
 *    host can see (null pointers, bad sizes, host coordinates out of range,
 *    calls out of order). Problems only the device sees (device coordinates out
 *    of range, a 16-bit field or the list capacity overflowing, a bounded wait
 *    giving up) set a per-grid device status word that vrt_sync returns.
 *    vrt_last_error gives a message for the last error of a grid.
 *  - Threading: a grid is used from one host thread at a time; distinct grids
 *    are independent.
 */
#ifndef VRT_H
#define VRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vrt_grid_s* vrt_grid;

typedef enum {
  VRT_OK = 0,
  VRT_ERR_INVALID_ARG = 1, /* bad argument or coordinate out of range */
  VRT_ERR_OOM = 2,         /* device allocation failed */
  VRT_ERR_OVERFLOW = 3,    /* a 16-bit voxel field or the list capacity overflowed */
  VRT_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  VRT_ERR_TIMEOUT = 5,     /* a bounded device wait or repair loop gave up */
  VRT_ERR_STATE = 6,       /* call out of order (e.g. trace before cull) */
  VRT_ERR_BOUNDS = 7       /* an index left its buffer (checked builds) */
} vrt_status;

/* Grid description (Sec. 3.1). */
typedef struct {
  int32_t n;              /* grid side: power of two in [16, 512] */
  float radius;           /* tube radius in voxels, (0, 4]; snapped to 2^-14 */
  float r_min;            /* PWAA radius clamp of Alg. 3; <= 0 selects 0.5 */
  int32_t occ_scale;      /* occupancy codes per unit occupancy in the packed
                             word; 0 selects 32 */
  uint64_t max_fragments; /* list capacity in entries (all voxels), also the
                             capacity of the fragment record and rank
                             buffers (10 bytes per entry); 0 selects
                             0.9 (L + 2 rl + 2)(2 rl + 2)^2, at least 16,
                             entries per uploaded vertex, with L the mean
                             segment length of the vrt_upload_segments call
                             and rl = radius + 2^-9; at most 3 * 2^30 - 1;
                             exceeding it reports VRT_ERR_OVERFLOW */
} vrt_grid_desc;

/* Pinhole or orthographic camera. Basis: f = normalize(target - eye),
 * right = normalize(f x up), true up = right x f. Pixel (x, y), row 0 at the
 * top, is sampled at its centre (x + 0.5, y + 0.5).
 *  perspective: origin eye, direction normalize(f + sx right + sy up') with
 *    sx = (2 (x+0.5)/W - 1) tan(fovy/2) W/H, sy = (1 - 2 (y+0.5)/H) tan(fovy/2)
 *  orthographic: direction f, origin eye + ((x+0.5)/W - 0.5) ortho_h W/H right
 *    + (0.5 - (y+0.5)/H) ortho_h up'. */
typedef struct {
  int32_t width, height, ortho;
  float eye[3], target[3], up[3];
  float fovy_deg; /* perspective vertical field of view, degrees */
  float ortho_h;  /* orthographic view height, voxels */
} vrt_camera;

/* Rendering parameters (Sec. 3.2, 3.4, 3.5). */
typedef struct {
  float alpha;      /* opacity of every tube in (0, 1]; 1 = opaque */
  int32_t ao_cones; /* 0: no ambient occlusion; 6: six cones per hit */
  int32_t cull;     /* 0: lists for every voxel (voxelize-scan-voxelize);
                       1: lists for camera-visible voxels only
                       (voxelize-cull-scan-voxelize);
                       2: automatic: as 1, except that the grid skips the
                       cull (as 0) while the last culled build it has seen
                       (through vrt_sync or vrt_get_stats) kept more than 95%
                       of the occupied voxels, culling again every 8th build.
                       The image is the same in every mode. */
  int32_t k;        /* 0, 1, 8, 16 or 32; kept for compatibility: the trace
                       keeps 4 nearest keys per lane (128 per warp) and
                       rescans a list when it must, so the image does not
                       depend on k */
  int32_t voxel_shading; /* 0: shade per hit (ao_cones); 1: voxel-space
                       shading (Sec. 3.4): before the trace, every voxel
                       within one step of a listed voxel gets the value
                       AO(centre) * (1/2 + 1/2 * S), AO the six-cone occlusion
                       at the voxel centre when ao_cones = 6 (else 1) and S the
                       transmittance of a ray from the centre toward the light
                       through the base pyramid level (samples one voxel
                       apart from one voxel out, trilinear, A <- A + (1-A)s,
                       S = 1 - A; the march may stop once S < 1e-4); each hit
                       is shaded by one trilinear sample of that field */
  float light[3];   /* voxel_shading: direction toward the directional light
                       (any finite non-zero vector; normalized) */
} vrt_render_params;

typedef struct {
  uint64_t fragments;        /* F: (segment, voxel) pairs of the last voxelize */
  uint64_t fragments_listed; /* entries written to the lists by the last frame */
  uint64_t sum_occupancy;    /* sum of occupancy codes of the last voxelize */
  uint64_t exact_decisions;  /* list decisions taken by the exact integer path */
  uint32_t occupied_voxels;  /* voxels with count > 0 */
  uint32_t visible_voxels;   /* voxels given lists by the last cull */
  uint32_t repaired_voxels;  /* culled voxels a ray needed, listed by repair */
  uint32_t repair_rounds;    /* repair rounds that found work */
  uint32_t max_count;        /* largest per-voxel count */
  uint32_t status_bits;      /* raw device status word */
  uint64_t kernel_launches;  /* kernels launched by this grid since creation */
  uint32_t retraced_pixels;  /* pixels traced again by the last frame's repair */
  uint32_t reserved;
  /* trace work, counted only while VRT_OPT_TRACE_COUNTERS is on (cumulative): */
  uint64_t trace_entries;       /* list entries examined */
  uint64_t trace_capsule_tests; /* entries that passed the line-distance test */
  uint64_t trace_voxels;        /* voxel lists processed */
  uint64_t trace_steps;         /* DDA steps (voxels and empty bricks) */
  uint64_t trace_wholewarp_voxels;  /* voxel lists taken by the whole-warp path */
  uint64_t trace_wholewarp_entries; /* entries it examined, rescans included */
  uint64_t trace_hits;              /* accepted hits handed to the rays */
  uint64_t trace_cycles[4];         /* SM cycles summed over warps: DDA steps,
                                       shared-entry path (with its compositing),
                                       whole-warp path; [3]: the capsule tests
                                       within the shared-entry path */
  /* distinct list entries, vertices and voxels (their packed word and list
     end) that the rays of the last instrumented vrt_trace read, repair rounds
     included (0 unless VRT_OPT_TRACE_COUNTERS was on for it) */
  uint64_t trace_unique_entries;
  uint64_t trace_unique_vertices;
  uint64_t trace_unique_voxels;
} vrt_stats;

/* Create a grid (Sec. 3.1). `cuda_stream` is a cudaStream_t (NULL = legacy
 * default stream). On success *out receives the handle; on failure *out is
 * NULL. Allocates the per-voxel words, offsets and bitmaps (about 9 bytes per
 * voxel). */
vrt_status vrt_create_grid(const vrt_grid_desc* desc, void* cuda_stream, vrt_grid* out);

/* Set the polyline topology and the vertices. `xyz`: n_vertices rows of
 * `stride` floats (stride 3 or 4; the 4th is ignored), host memory if
 * on_device == 0, else device memory. `polyline_offsets`: HOST array of
 * n_polylines + 1 non-decreasing int64, first 0 and last n_vertices; polyline
 * p owns vertices [offsets[p], offsets[p+1]). Copies everything; (re)allocates
 * the vertex buffers and, when max_fragments was 0, the list capacity. On a
 * grid of side 512 or more it also fixes the order in which voxelization takes
 * the polylines (sorted by the coarse cell of their middle vertex; one small
 * kernel and a host counting sort, 4 bytes per vertex on the device), which
 * later vertex updates keep; the order affects speed only. Host coordinates
 * outside [-256, 768) or not finite give VRT_ERR_INVALID_ARG. Waits for the
 * copies before returning. */
vrt_status vrt_upload_segments(vrt_grid g, const float* xyz, int32_t stride, int64_t n_vertices,
                               const int64_t* polyline_offsets, int64_t n_polylines,
                               int32_t on_device);

/* Overwrite vertices [first_vertex, first_vertex + n_vertices) with new
 * coordinates (same topology); a dynamic frame's update. Same layout and
 * memory rules as vrt_upload_segments, except that coordinates (host or
 * device) are checked on the device by the next vrt_voxelize: one outside
 * [-256, 768) or not finite makes vrt_sync return VRT_ERR_INVALID_ARG. */
vrt_status vrt_update_vertices(vrt_grid g, int64_t first_vertex, int64_t n_vertices,
                               const float* xyz, int32_t stride, int32_t on_device);

/* Ingest (snap, flags, clip normals) of the vertices uploaded or updated since
 * the last vrt_voxelize (and their polyline neighbours), and voxelization pass 1
 * (Sec. 3.1, Alg. 1 walk, Alg. 3 occupancy): for every segment and every voxel within the list
 * radius of it (r + 2^-9, decided exactly), one 32-bit atomic add of
 * (occupancy code << 16) | 1 into the voxel's packed word; the count it returns
 * is the fragment's rank in the voxel, kept with the fragment for pass 2. */
vrt_status vrt_voxelize(vrt_grid g);

/* Averaging occupancy pyramid (Sec. 3.1): level 0 = min(1, occupancy code sum /
 * occ_scale), level l+1 = mean of 8 children, down to 1^3. Needs vrt_voxelize. */
vrt_status vrt_build_mips(vrt_grid g);

/* Culling and list build (Sec. 3.2, 3.3): with p->cull = 1, mark voxels whose
 * centre sees the camera through the eroded occupancy; exclusive scan of the
 * counts of marked voxels into list offsets; voxelization pass 2 writes segment
 * ids into the lists of marked voxels, each at the slot its rank gives. With
 * p->cull = 0 every occupied voxel is marked. Needs vrt_voxelize. */
vrt_status vrt_cull(vrt_grid g, const vrt_camera* cam, const vrt_render_params* p);

/* Ray tracing (Sec. 3.5): one ray per pixel through the grid by 3D-DDA; in
 * each voxel every listed segment's first entry into its capsule is tested
 * (a warp splits each voxel's list), kept if it lies in the voxel and the clip
 * planes keep it; opaque: nearest hit; transparent: all hits composited front
 * to back in (depth, id) order until transmittance < 1e-4. A ray that meets a culled
 * voxel holding segments has that voxel listed and is traced again, so the
 * image never depends on culling. Outputs are DEVICE buffers of width*height
 * entries, row-major from the top row: rgba_out float4 premultiplied (colour =
 * |unit tangent| * shading, alpha = 1 - transmittance; shading = per-hit AO,
 * the voxel-space shading field or 1), first_id_out the nearest accepted
 * segment id or -1 (nullable), first_t_out its depth or +inf (nullable).
 * Needs vrt_cull (and vrt_build_mips when p->ao_cones > 0 or
 * p->voxel_shading). With p->voxel_shading the call first computes the
 * shading field (stage 8) -- unless the last shaded trace computed it from the
 * same list build, pyramid, light and AO setting (a static scene traced again
 * from another camera) -- and each repair round extends it next to the voxels
 * it lists. Tracing again without a new vrt_cull reuses the lists: a static
 * scene needs only this call per frame (Sec. 4), with lists built for every
 * occupied voxel (p->cull = 0) or, when culled, extended by the repair
 * rounds for the new camera. */
vrt_status vrt_trace(vrt_grid g, const vrt_camera* cam, const vrt_render_params* p,
                     float* rgba_out, int32_t* first_id_out, float* first_t_out);

/* Wait for the grid's stream; return the device status (VRT_OK or the first
 * device-detected error) and clear it. */
vrt_status vrt_sync(vrt_grid g);

/* Counters of the last frame (waits). */
vrt_status vrt_get_stats(vrt_grid g, vrt_stats* out);

/* Test readback (waits): packed words in canonical order (x fastest, then y,
 * then z), n^3 entries. */
vrt_status vrt_read_grid(vrt_grid g, uint32_t* words_host);

/* Test readback (waits): for each voxel in canonical order its list start and
 * length (0 when the voxel has no list), and the list storage itself
 * (*n_ids entries, at most `cap` copied). Entry order within a list is
 * unspecified. */
vrt_status vrt_read_lists(vrt_grid g, uint32_t* start_host, uint32_t* len_host, uint32_t* ids_host,
                          uint64_t cap, uint64_t* n_ids);

/* Test readback (waits): all pyramid levels, level 0 first, each canonical. */
vrt_status vrt_read_mips(vrt_grid g, float* host, uint64_t n_floats);

/* Test readback (waits): the voxel-space shading field of the last trace with
 * p->voxel_shading, canonical order (n^3 floats); valid_host (nullable, n^3
 * bytes) is 1 where the value was computed for that trace, and values_host
 * is 0 elsewhere. VRT_ERR_STATE if no trace has used voxel shading. */
vrt_status vrt_read_shading(vrt_grid g, float* values_host, uint8_t* valid_host);

/* Options. VRT_OPT_FORCE_EXACT (1): value 1 decides every list membership on
 * the exact integer path instead of the fp32 filter (for testing).
 * VRT_OPT_STAGE_TIMING (2): value 1 records CUDA events on the grid's stream
 * around each stage (see vrt_get_stage_ms).
 * VRT_OPT_TRACE_COUNTERS (3): value 1 runs an instrumented trace that counts
 * its work into vrt_stats (slower; for analysis).
 * VRT_OPT_MIPS_FORMAT (4): storage of the occupancy pyramid texels, VRT_MIPS_F32
 * (default), VRT_MIPS_F16 or VRT_MIPS_BF16; every level is averaged in fp32
 * from its stored children and rounded to nearest once, and the trace widens
 * the samples to fp32. Changing it invalidates the pyramid (vrt_build_mips
 * again). vrt_read_mips returns the stored values widened to fp32.
 * VRT_OPT_GRAPH (5): value 1 makes vrt_frame run as a CUDA graph (see there).
 * VRT_OPT_CULL_DEPTH (6): value v > 0 culls a voxel once the estimated
 * optical depth in front of it exceeds v / 1000 instead of ln(1e4) + 3; 0
 * restores the default. For testing: a small threshold culls voxels that rays
 * reach, which the repair rounds then list; the image does not change.
 * VRT_OPT_TEST_SCAN_STALL (7), for testing the bounded waits: value t >= 0
 * makes tile t of the list-offset scan (4096 voxels per tile) skip publishing
 * its look-back state and lets every look-back wait give up after 1024 polls
 * instead of about 4 million, so the waits of the tiles after it run out:
 * vrt_sync then returns VRT_ERR_TIMEOUT and the lists of that build are
 * wrong (every list access stays bounded). -1 restores the normal scan. With
 * g == NULL it applies, process-wide, to vrt_scan_counts_noalloc (status bit
 * 0). No wait is left unbounded in either case.
 * VRT_OPT_TRACE_SHORT_LIST (8): value in [0, 1024] (default 1024): voxel lists
 * up to this length share the warp entry by entry in the trace; longer ones
 * take the whole-warp path (one list at a time). The image does not depend on
 * it; for testing that path.
 * VRT_OPT_TRACE_RAY_KEYS (9): value in [1, 32] (default 32): hit slots per
 * transparent ray and voxel on the shared-entry path; a ray with more hits in
 * one voxel takes the whole-warp path for it. The image does not depend on
 * it; for testing.
 * VRT_OPT_HIT_KEY (10): the order of the hits a ray composites within one
 * voxel (Sec. 3.5). VRT_HIT_KEY_DEPTH_ID (default): by depth in fp32, equal
 * depths by segment id -- the ground-truth order, independent of how the list
 * build ordered each list. VRT_HIT_KEY_16_16: the paper's 32-bit key, the
 * hit's depth within the voxel's ray interval quantized to 16 bits above its
 * 16-bit index in the voxel's list, so hits whose depths fall in the same
 * 1/65536 of the interval follow the list's order (which the list build's
 * atomics leave arbitrary); depths and shading still use the exact hit.
 * VRT_OPT_TRACE_TILE (11): the pixel tile a warp of the transparent trace owns:
 * 32 pixels, 2, 4 (default), 8 or 16 wide (16, 8, 4 or 2 tall). Rays of a tile
 * that wait in the same voxel share each list entry's loads, so the best shape
 * depends on the scene and camera (vrt_tune_shapes measures it). The image
 * does not depend on it. The instrumented trace and the 16+16 key use 4. */
#define VRT_OPT_FORCE_EXACT 1
#define VRT_OPT_STAGE_TIMING 2
#define VRT_OPT_TRACE_COUNTERS 3
#define VRT_OPT_MIPS_FORMAT 4
#define VRT_OPT_GRAPH 5
#define VRT_OPT_CULL_DEPTH 6
#define VRT_OPT_TEST_SCAN_STALL 7
#define VRT_OPT_TRACE_SHORT_LIST 8
#define VRT_OPT_TRACE_RAY_KEYS 9
#define VRT_OPT_HIT_KEY 10
#define VRT_OPT_TRACE_TILE 11
#define VRT_HIT_KEY_DEPTH_ID 0
#define VRT_HIT_KEY_16_16 1
#define VRT_MIPS_F32 0
#define VRT_MIPS_F16 1
#define VRT_MIPS_BF16 2
vrt_status vrt_set_option(vrt_grid g, int32_t option, int64_t value);

/* One frame in one call: the vertex update (when n_vertices > 0; same rules as
 * vrt_update_vertices), vrt_voxelize, vrt_build_mips when p->ao_cones, vrt_cull
 * and vrt_trace. With VRT_OPT_GRAPH on, the chain is captured (on a stream the
 * grid owns) into a CUDA graph that is launched on the grid's stream; the
 * executable graph is updated in place from each frame's capture, so cameras,
 * parameters and updates may change freely, and is re-instantiated when the
 * launch sequence changes shape. Buffers the chain sizes lazily are allocated
 * before the capture (this may synchronize the grid's stream). Frames with
 * pageable host input run uncaptured. Stage timing works in both forms. The
 * result is that of the separate calls. */
vrt_status vrt_frame(vrt_grid g, int64_t first_vertex, int64_t n_vertices, const float* xyz,
                     int32_t stride, int32_t on_device, const vrt_camera* cam,
                     const vrt_render_params* p, float* rgba_out, int32_t* first_id_out,
                     float* first_t_out);

/* Autotuning of the voxel resolution: renders the scene (host vertices in the
 * units of a grid of side base->n, camera in the same units) in grids of each
 * side in `sides` -- coordinates, radius and camera scaled with the side -- for
 * `frames` frames after a warm-up, and returns the side with the lowest mean
 * frame time in *best_side (ms_out[i]: its mean time, +inf when that side
 * could not render the scene). Without AO the image does not depend on the
 * side beyond fp32 rounding at voxel boundaries. */
vrt_status vrt_tune_grid_side(const vrt_grid_desc* base, const float* xyz, int32_t stride,
                              int64_t n_vertices, const int64_t* polyline_offsets,
                              int64_t n_polylines, const vrt_camera* cam,
                              const vrt_render_params* p, const int32_t* sides, int32_t n_sides,
                              int32_t frames, int32_t* best_side, float* ms_out);

/* Autotuning of the voxel resolution and the trace's tile shape: as
 * vrt_tune_grid_side, for every grid side in `sides` and every tile width in
 * `tiles` (VRT_OPT_TRACE_TILE: 2, 4, 8 or 16); ms_out (nullable) receives
 * n_sides * n_tiles mean frame times, side-major (+inf where that pair could
 * not render the scene); *best_side and *best_tile the fastest pair. */
vrt_status vrt_tune_shapes(const vrt_grid_desc* base, const float* xyz, int32_t stride,
                           int64_t n_vertices, const int64_t* polyline_offsets,
                           int64_t n_polylines, const vrt_camera* cam, const vrt_render_params* p,
                           const int32_t* sides, int32_t n_sides, const int32_t* tiles,
                           int32_t n_tiles, int32_t frames, int32_t* best_side,
                           int32_t* best_tile, float* ms_out);

/* Device memory the grid holds, in bytes (its buffers as currently sized). */
vrt_status vrt_grid_device_bytes(vrt_grid g, uint64_t* bytes);

/* Issue the grid's later work on another CUDA stream (NULL: the legacy default
 * stream). Does not wait: the caller orders the switch, i.e. the grid's work
 * issued so far must have finished, or be ordered before the new stream's work
 * (an event), when the grid's next call runs. */
vrt_status vrt_set_stream(vrt_grid g, void* cuda_stream);

/* Stage durations of the last frame in milliseconds (waits), measured with
 * CUDA events on the grid's stream while VRT_OPT_STAGE_TIMING is on. Order:
 * 0 ingest, 1 voxelize pass 1, 2 mips, 3 cull marks, 4 scan, 5 voxelize
 * pass 2, 6 trace, 7 repair rounds (list + re-trace), 8 voxel-space shading.
 * Stages that did not run since the last vrt_voxelize read -1. Writes
 * min(n, 9) entries. */
#define VRT_N_STAGES 9
vrt_status vrt_get_stage_ms(vrt_grid g, float* ms, int32_t n);

/* Exclusive prefix sum of per-voxel counts that allocates no device memory.
 * The paper has no counterpart: it is a stand-alone form of the list-offset
 * scan that vrt_cull runs, for callers that cannot allocate device memory
 * where they need it -- code whose device memory is owned by a pool or arena,
 * loops that must not grow or fragment memory mid-frame, real-time paths where
 * an allocation could block in the driver. Its look-back scratch is a fixed
 * array inside the library image (about 256 KB), which every GPU that loads
 * the library holds until the process exits.
 *   words:      DEVICE, n_voxels packed words; the count is the low 16 bits.
 *   marks:      DEVICE bitmap (bit i%32 of word i/32 marks voxel i), or NULL
 *               to count every voxel.
 *   offsets:    DEVICE output, n_voxels entries: the exclusive prefix sum of
 *               the counts of marked voxels in the order given.
 *   n_voxels:   a multiple of 4096, at most 134217728 (512^3); anything else
 *               returns VRT_ERR_INVALID_ARG before any device work.
 *   total_out:  DEVICE, one entry (nullable): the sum of the marked counts
 *               (its low 32 bits when it exceeds 2^32 - 1).
 *   status_out: DEVICE, one entry (nullable), bits set (never cleared here):
 *               bit 0 if a bounded wait gave up (the offsets are then wrong);
 *               bit 1 if the total exceeds 2^32 - 1, so that the offsets
 *               past that point wrapped (each is its prefix sum mod 2^32).
 * words and offsets must be 16-byte aligned. The grid's own list build
 * orders voxels in 4^3 bricks (brick index x-fastest, then 16 z + 4 y + x
 * inside the brick); pass words in that order to reproduce its offsets.
 * The call issues two cudaMemsetAsync (clearing its scratch) and one kernel
 * on `cuda_stream`; it calls no cudaMalloc, cudaFree or allocating library
 * routine. Every call shares the scratch array and leaves its contents
 * behind; calls that overlap on the GPU (two streams, two threads) race and
 * give wrong results. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. Errors: VRT_ERR_INVALID_ARG, VRT_ERR_CUDA;
 * vrt_last_error(NULL) gives the message. */
vrt_status vrt_scan_counts_noalloc(const uint32_t* words, const uint32_t* marks, uint32_t* offsets,
                                   uint64_t n_voxels, uint32_t* total_out, uint32_t* status_out,
                                   void* cuda_stream);

/* Message for the last error of `g` (or, when g is NULL, of the last failed
 * call without a grid -- create, vrt_scan_counts_noalloc, vrt_tune_grid_side,
 * the vrt_server_* calls -- made by the calling host thread; each thread keeps
 * its own). Valid until that thread's next such call, or the next call on the
 * grid. */
const char* vrt_last_error(vrt_grid g);

/* Wait for the stream, free every device buffer and the handle. */
vrt_status vrt_destroy(vrt_grid g);

/* ------------------------------------------------------------------ serving
 * A request loop over resident line sets (continuous batching of frames).
 * Line sets are registered once; a frame request names a set, an optional
 * vertex update, a camera and render parameters, and a device output buffer.
 * A scheduler thread issues requests as soon as a stream slot is free and the
 * set has no frame in flight (frames of one set run in submission order; frames
 * of different sets overlap on the device, one CUDA stream per slot). A set is
 * resident on the device while its grid, lists and pyramid are allocated;
 * admitting a frame of a non-resident set first evicts least-recently-used idle
 * sets until its footprint fits the HBM budget (the server keeps a host copy of
 * every set, updated by each issued frame, to upload it again). Each frame is
 * exactly the frame of the plain calls on that set, so its result does not
 * depend on what else runs. Latency is measured from vrt_server_submit to the
 * host seeing the frame's stream work finish. Thread safety: submit, poll and
 * stats may be called from any host threads. */
typedef struct vrt_server_s* vrt_server;

typedef struct {
  uint64_t hbm_budget;  /* device bytes the resident sets may hold; 0 selects
                           80% of the free device memory at creation */
  int32_t max_inflight; /* frames on the device at once (stream slots), >= 1;
                           0 selects 4 */
  int32_t device;       /* CUDA device ordinal */
  int32_t small_segments; /* > 0: frames of sets with fewer segments than
                           this are issued in batches: the pending frames of up
                           to max_batch idle small sets are captured into one
                           CUDA graph (one branch per set, each set's chain on
                           its own stream) and launched at once on one slot;
                           <= 0 (default): no batching. (Measured: frames of
                           sets under 100k segments at 720p are bound by their
                           trace on the GPU, and the per-batch capture makes
                           batching slower there, 1028 vs 1154 frames/s.) */
  int32_t max_batch;    /* frames per batch, 0 selects 16 (at most 64) */
} vrt_server_desc;

typedef struct {
  int64_t request_id;
  int32_t set_id;
  int32_t status;       /* the frame's vrt_status (vrt_sync of its grid) */
  double latency_ms;    /* submit -> completion seen by the host */
  double queue_ms;      /* submit -> issue */
} vrt_server_result;

typedef struct {
  uint64_t hbm_budget;
  uint64_t resident_bytes;   /* device bytes of the resident sets */
  uint64_t completed;        /* requests finished so far */
  int32_t resident_sets;
  int32_t evictions;         /* sets evicted so far */
  int32_t pending;           /* submitted, not yet issued */
  int32_t inflight;          /* issued, not yet finished */
  uint64_t batches;          /* small-set batches issued (one graph launch each) */
  uint64_t batched_frames;   /* frames issued in those batches */
} vrt_server_stats;

vrt_status vrt_server_create(const vrt_server_desc* desc, vrt_server* out);

/* Register a line set (host vertices, same layout and checks as
 * vrt_upload_segments; copied). It is uploaded when a frame first needs it. */
vrt_status vrt_server_add_set(vrt_server s, const vrt_grid_desc* grid, const float* xyz,
                              int32_t stride, int64_t n_vertices, const int64_t* polyline_offsets,
                              int64_t n_polylines, int32_t* set_id);

/* Queue a frame of set `set_id`: vertices [first_vertex, first_vertex +
 * n_vertices) take the HOST coordinates `xyz` (stride 3 or 4; copied at once;
 * n_vertices may be 0), then voxelize, mips when cam params ask for AO, cull,
 * trace into the DEVICE buffers rgba_out (width * height * 4 floats) and, when
 * not NULL, first_id_out / first_t_out, which must stay valid until the
 * request completes. Returns at once with its id. */
vrt_status vrt_server_submit(vrt_server s, int32_t set_id, int64_t first_vertex,
                             int64_t n_vertices, const float* xyz, int32_t stride,
                             const vrt_camera* cam, const vrt_render_params* p, float* rgba_out,
                             int32_t* first_id_out, float* first_t_out, int64_t* request_id);

/* Move up to `cap` finished requests (in completion order) into `out`;
 * *n_out = how many. With wait != 0, first waits until every submitted request
 * has finished. */
vrt_status vrt_server_poll(vrt_server s, vrt_server_result* out, int32_t cap, int32_t* n_out,
                           int32_t wait);

vrt_status vrt_server_get_stats(vrt_server s, vrt_server_stats* out);

/* Waits for every submitted request, then frees the sets and the server. */
vrt_status vrt_server_destroy(vrt_server s);

#ifdef __cplusplus
}
#endif
#endif /* VRT_H */
