// C ABI of libvrt (include/vrt.h): handle, device memory, stream ordering and
// status. Every step of the frame runs in the kernels of this library; this
// file only validates arguments, allocates, and issues launches and copies on
// the grid's stream.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "launch.h"
#include "vrt.h"

using namespace vrt;

struct vrt_grid_s {
  int n = 0, log2n = 0, log2nb = 0;
  float r = 0, r_min = 0.5f;
  int R = 0, RL = 0;
  int occ_scale = 32;
  uint64_t max_frag_desc = 0;
  cudaStream_t stream = nullptr;
  // vertices
  long long V = 0, P = 0, V_alloc = 0;
  // vertices uploaded or updated since the last ingest, with their polyline
  // neighbours: [dirty_lo, dirty_hi), empty when dirty_lo >= dirty_hi
  long long dirty_lo = 0, dirty_hi = 0;
  float* raw = nullptr;
  uint8_t* flags = nullptr;
  float4* pos = nullptr;
  float4* nrm = nullptr;
  // voxels
  uint32_t *word = nullptr, *cur = nullptr, *vis = nullptr;
  uint8_t *bdist = nullptr, *btmp = nullptr;  // empty-brick distance field and its scratch
  uint32_t* need = nullptr;
  uint8_t* eroded = nullptr;
  uint8_t* cdist = nullptr;  // [bricks] distance to a brick with eroded occupancy
  float* emean = nullptr;    // [bricks] mean eroded occupancy
  uint32_t* lists = nullptr;
  unsigned long long list_cap = 0;
  uint2* xq = nullptr;      // pairs the fp32 filter left to the exact path
  uint32_t xq_cap = 0;
  unsigned long long* rec = nullptr;  // fragment records of pass 1 (list_cap entries)
  uint16_t* rank = nullptr;           // each record's rank within its voxel (list_cap entries)
  unsigned long long* tile_state = nullptr;
  uint32_t n_tiles = 0;
  void* mips = nullptr;            // occupancy pyramid (room for fp32 texels)
  int mips_fmt = kMipsF32;
  long long lev_off[11] = {0};
  int n_levels = 0;
  uint32_t* vq[2] = {nullptr, nullptr};
  uint32_t vq_cap = 0;
  uint32_t* pq[2] = {nullptr, nullptr};
  uint32_t pq_cap = 0;
  float4* resume = nullptr;  // [2 * pq_cap] ray state at the first culled voxel
  uint32_t* order = nullptr;      // [V] pass-1 processing order of the vertices' segments
  float* shade = nullptr;         // [n^3] voxel-space shading field (brick order)
  uint32_t* shade_mask = nullptr; // [n^3 / 32] voxels the last shaded trace computed
  // instrumented trace (VRT_OPT_TRACE_COUNTERS): bitmaps of the list entries,
  // vertices and voxels the rays read, sized at first use
  uint32_t *touch_list = nullptr, *touch_vert = nullptr, *touch_vox = nullptr;
  size_t touch_list_words = 0, touch_vert_words = 0;
  bool shade_valid = false;
  // what the field was computed from: list build, pyramid build, AO, light;
  // a trace with the same inputs (a static scene) reuses it
  uint64_t build_id = 0, mips_id = 0;
  uint64_t shade_key[4] = {~0ull, ~0ull, ~0ull, ~0ull};
  DevStatus* st = nullptr;
  int force_exact = 0;
  int trace_counters = 0;
  // stage timing
  unsigned long long launches = 0;  // kernels launched by this grid
  bool timing = false;
  cudaEvent_t ev[VRT_N_STAGES][2] = {};
  bool ev_used[VRT_N_STAGES] = {};
  // frame state
  int stage = 0;  // 0 created, 1 vertices set, 2 voxelized, 3 lists built
  bool mips_valid = false;
  int culled = 0;
  // automatic culling: visible / occupied voxels of the last culled list build
  // seen on the host (-1: not yet), and list builds since the last cull
  double auto_vis_frac = -1.0;
  int auto_skipped = 0;
  // vrt_frame as a CUDA graph: the executable graph (updated in place while
  // the frame's launch sequence keeps its shape) and the grid's own stream the
  // frame is captured on (the legacy default stream cannot be captured)
  float cull_depth = 0.0f;  // VRT_OPT_CULL_DEPTH (0: the default threshold)
  int scan_stall = -1;      // VRT_OPT_TEST_SCAN_STALL (-1: off)
  uint32_t short_list = kShortList;  // VRT_OPT_TRACE_SHORT_LIST
  uint32_t ray_keys = kRayKeys;      // VRT_OPT_TRACE_RAY_KEYS
  int key16 = 0;                     // VRT_OPT_HIT_KEY
  int tile_w = 4;                    // VRT_OPT_TRACE_TILE
  bool use_graph = false;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  bool capturing = false;
  std::string err;
  // device memory held by this grid
  std::unordered_map<void*, size_t> alloc_bytes;
  uint64_t dev_bytes = 0;
};

// Last error without a grid (creation, stand-alone and server calls), one per
// host thread, so failing calls on different threads do not race on it.
thread_local std::string g_create_error;

namespace {

vrt_status fail(vrt_grid g, vrt_status s, const std::string& msg) {
  if (g) g->err = msg; else g_create_error = msg;
  return s;
}

vrt_status cuda_fail(vrt_grid g, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(g, e == cudaErrorMemoryAllocation ? VRT_ERR_OOM : VRT_ERR_CUDA, m);
}

#define VRT_CUDA(g, call)                              \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(g, e_, #call); \
  } while (0)

// Device allocations of a grid, counted in g->dev_bytes.
template <class T>
cudaError_t dalloc(vrt_grid g, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  const cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) {
    g->alloc_bytes[(void*)*p] = count * sizeof(T);
    g->dev_bytes += count * sizeof(T);
  }
  return e;
}

template <class T>
void dfree(vrt_grid g, T*& p) {
  if (p) {
    auto it = g->alloc_bytes.find((void*)p);
    if (it != g->alloc_bytes.end()) {
      g->dev_bytes -= it->second;
      g->alloc_bytes.erase(it);
    }
    cudaFree(p);
  }
  p = nullptr;
}

GridDev gdev(vrt_grid g) {
  GridDev d;
  d.n = g->n; d.log2n = g->log2n; d.log2nb = g->log2nb;
  d.r = g->r;
  d.rl = (float)(g->RL) / kUnits;
  d.R = g->R; d.RL = g->RL;
  d.r_clamp = fmaxf(g->r, g->r_min);
  d.corr = (g->r / d.r_clamp) * (g->r / d.r_clamp);
  d.occ_scale = (float)g->occ_scale;
  d.force_exact = g->force_exact;
  d.word = g->word; d.cur = g->cur; d.vis = g->vis; d.bdist = g->bdist;
  d.lists = g->lists; d.list_cap = g->list_cap;
  d.xq = g->xq; d.xq_cap = g->xq_cap;
  d.rec = g->rec; d.rank = g->rank; d.rec_cap = (uint32_t)g->list_cap;
  d.st = g->st;
  return d;
}

// Every coordinate finite and in [kCoordMin, kCoordMax). Accumulates without an
// early exit so that the compiler vectorizes it (NaN fails both comparisons).
// fp16 / bf16 bit patterns widened to fp32 (exact), for the test readback.
float half_to_float(uint16_t h) {
  const uint32_t s = (uint32_t)(h >> 15) << 31, e = (h >> 10) & 31u, m = h & 1023u;
  float v;
  if (e == 0) {
    v = std::ldexp((float)m, -24);  // zero and subnormals
  } else if (e == 31) {
    v = m ? NAN : INFINITY;
  } else {
    v = std::ldexp((float)(m | 1024u), (int)e - 25);
  }
  uint32_t b;
  std::memcpy(&b, &v, 4);
  b |= s;
  std::memcpy(&v, &b, 4);
  return v;
}

float bf16_to_float(uint16_t h) {
  const uint32_t b = (uint32_t)h << 16;
  float v;
  std::memcpy(&v, &b, 4);
  return v;
}

bool host_coords_ok(const float* xyz, int stride, long long V) {
  unsigned bad = 0;
  if (stride == 3) {
    const long long m = 3 * V;
    for (long long i = 0; i < m; ++i) {
      const float x = xyz[i];
      bad |= (unsigned)!(x >= kCoordMin) | (unsigned)!(x < kCoordMax);
    }
  } else {
    for (long long i = 0; i < V; ++i)
      for (int k = 0; k < 3; ++k) {
        const float x = xyz[i * stride + k];
        bad |= (unsigned)!(x >= kCoordMin) | (unsigned)!(x < kCoordMax);
      }
  }
  return bad == 0;
}

vrt_status copy_vertices(vrt_grid g, long long first, long long V, const float* xyz, int stride,
                         int on_device) {
  if (V == 0) return VRT_OK;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (stride == 3) {  // contiguous rows: one plain copy
    VRT_CUDA(g, cudaMemcpyAsync(g->raw + 3 * first, xyz, 3 * sizeof(float) * (size_t)V, kind,
                                g->stream));
  } else {
    VRT_CUDA(g, cudaMemcpy2DAsync(g->raw + 3 * first, 3 * sizeof(float), xyz,
                                  (size_t)stride * sizeof(float), 3 * sizeof(float), (size_t)V,
                                  kind, g->stream));
  }
  return VRT_OK;
}

// Pass-1 processing order, fixed at upload (the topology does not change
// after it): polylines sorted by the 16^3 cell of their middle vertex (a
// counting sort on the 12-bit Morton code), each polyline's vertices kept
// together. Neighbouring warps then voxelize nearby segments, so the
// packed-word atomics of the blocks in flight cover a small part of the grid.
// Used from a side of kOrderMinSide, where the packed words (512 MB at 512^3)
// far exceed the L2 cache; below it the words stay in L2 and the input order
// is as good. The order only affects speed: every segment is voxelized once.
constexpr int kOrderMinSide = 512;

vrt_status build_order(vrt_grid g, const int64_t* offsets, long long P) {
  const long long V = g->V;
  std::vector<uint32_t> mid, poly;
  mid.reserve((size_t)P);
  poly.reserve((size_t)P);
  for (long long p = 0; p < P; ++p)
    if (offsets[p + 1] > offsets[p]) {
      mid.push_back((uint32_t)(offsets[p] + (offsets[p + 1] - offsets[p] - 1) / 2));
      poly.push_back((uint32_t)p);
    }
  const uint32_t Pn = (uint32_t)mid.size();
  std::vector<uint16_t> key(Pn);
  if (Pn > 0) {
    uint32_t* d_mid = nullptr;
    uint16_t* d_key = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_mid, Pn * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_key, Pn * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mid, mid.data(), Pn * sizeof(uint32_t), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) {
      launch_poly_keys(g->raw, d_mid, Pn, g->n, d_key, g->stream);
      e = cudaMemcpyAsync(key.data(), d_key, Pn * sizeof(uint16_t), cudaMemcpyDeviceToHost, g->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaFree(d_mid);
    cudaFree(d_key);
    if (e != cudaSuccess) return cuda_fail(g, e, "pass-1 order keys");
  }
  std::vector<uint32_t> start(4097, 0);
  for (uint32_t q = 0; q < Pn; ++q) ++start[key[q] + 1];
  for (int b = 0; b < 4096; ++b) start[b + 1] += start[b];
  std::vector<uint32_t> sorted(Pn);
  for (uint32_t q = 0; q < Pn; ++q) sorted[start[key[q]]++] = poly[q];
  std::vector<uint32_t> order((size_t)V);
  size_t k = 0;
  for (uint32_t q = 0; q < Pn; ++q)
    for (int64_t v = offsets[sorted[q]]; v < offsets[sorted[q] + 1]; ++v) order[k++] = (uint32_t)v;
  if ((long long)k != V) return fail(g, VRT_ERR_INVALID_ARG, "offsets do not cover the vertices");
  VRT_CUDA(g, cudaMemcpyAsync(g->order, order.data(), (size_t)V * sizeof(uint32_t), cudaMemcpyHostToDevice,
                              g->stream));
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));  // order is a host temporary
  return VRT_OK;
}

void make_camdev(const HostCamera& c, CamDev& cd) {
  auto sub = [](const double* a, const double* b, double* o) { for (int k = 0; k < 3; ++k) o[k] = a[k] - b[k]; };
  auto nrm = [](double* v) { double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); for (int k = 0; k < 3; ++k) v[k] /= l; };
  auto crs = [](const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0];
  };
  double f[3], rt[3], up[3];
  sub(c.target, c.eye, f); nrm(f);
  crs(f, c.up, rt); nrm(rt);
  crs(rt, f, up);
  const double W = c.width, H = c.height;
  auto F3 = [](double x, double y, double z) { return make_float3((float)x, (float)y, (float)z); };
  cd.width = c.width; cd.height = c.height; cd.ortho = c.ortho;
  if (c.ortho) {
    const double oh = c.ortho_h, ow = oh * W / H;
    double o0[3], ox[3], oy[3];
    for (int k = 0; k < 3; ++k) {
      o0[k] = c.eye[k] - 0.5 * ow * rt[k] + 0.5 * oh * up[k];
      ox[k] = ow / W * rt[k];
      oy[k] = -oh / H * up[k];
    }
    cd.o0 = F3(o0[0], o0[1], o0[2]); cd.ox = F3(ox[0], ox[1], ox[2]); cd.oy = F3(oy[0], oy[1], oy[2]);
    cd.d0 = F3(f[0], f[1], f[2]);
    cd.dx = cd.dy = make_float3(0.f, 0.f, 0.f);
  } else {
    const double th = std::tan(c.fovy_deg * 3.14159265358979323846 / 360.0);
    const double as = W / H;
    double d0[3], dx[3], dy[3];
    for (int k = 0; k < 3; ++k) {
      d0[k] = f[k] - th * as * rt[k] + th * up[k];
      dx[k] = 2.0 * th * as / W * rt[k];
      dy[k] = -2.0 * th / H * up[k];
    }
    cd.o0 = F3(c.eye[0], c.eye[1], c.eye[2]);
    cd.ox = cd.oy = make_float3(0.f, 0.f, 0.f);
    cd.d0 = F3(d0[0], d0[1], d0[2]); cd.dx = F3(dx[0], dx[1], dx[2]); cd.dy = F3(dy[0], dy[1], dy[2]);
  }
}

bool camera_ok(const vrt_camera* c) {
  if (!c || c->width <= 0 || c->height <= 0) return false;
  if ((long long)c->width * c->height >= (1ll << 31)) return false;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(c->eye[k]) || !std::isfinite(c->target[k]) || !std::isfinite(c->up[k])) return false;
  double f[3], up[3] = {c->up[0], c->up[1], c->up[2]};
  for (int k = 0; k < 3; ++k) f[k] = (double)c->target[k] - c->eye[k];
  const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(fl > 0)) return false;
  const double cx = f[1] * up[2] - f[2] * up[1], cy = f[2] * up[0] - f[0] * up[2], cz = f[0] * up[1] - f[1] * up[0];
  if (!(cx * cx + cy * cy + cz * cz > 0)) return false;
  if (c->ortho) return c->ortho_h > 0;
  return c->fovy_deg > 0 && c->fovy_deg < 180;
}

}  // namespace

const char* vrt::frame_args_error(const vrt_camera* cam, const vrt_render_params* p) {
  if (!p) return "params is NULL";
  if (!camera_ok(cam)) return "bad camera";
  if (!(p->alpha > 0.0f && p->alpha <= 1.0f)) return "alpha must be in (0, 1]";
  if (p->ao_cones != 0 && p->ao_cones != 6) return "ao_cones must be 0 or 6";
  if (p->cull < 0 || p->cull > 2) return "cull must be 0, 1 or 2";
  if (p->k != 0 && p->k != 1 && p->k != 8 && p->k != 16 && p->k != 32)
    return "k must be 0, 1, 8, 16 or 32";
  if (p->voxel_shading != 0 && p->voxel_shading != 1) return "voxel_shading must be 0 or 1";
  if (p->voxel_shading) {
    const double l2 = (double)p->light[0] * p->light[0] + (double)p->light[1] * p->light[1] +
                      (double)p->light[2] * p->light[2];
    if (!(l2 > 0.0) || !std::isfinite(l2)) return "light must be a finite non-zero direction";
  }
  return nullptr;
}

namespace {

HostCamera host_cam(const vrt_camera* c) {
  HostCamera h;
  h.width = c->width; h.height = c->height; h.ortho = c->ortho;
  for (int k = 0; k < 3; ++k) { h.eye[k] = c->eye[k]; h.target[k] = c->target[k]; h.up[k] = c->up[k]; }
  h.fovy_deg = c->fovy_deg; h.ortho_h = c->ortho_h;
  return h;
}

enum { ST_INGEST, ST_PASS1, ST_MIPS, ST_CULL, ST_SCAN, ST_PASS2, ST_TRACE, ST_REPAIR, ST_SHADE };
static_assert(ST_SHADE + 1 == VRT_N_STAGES, "stage list");

void stage_mark(vrt_grid g, int stage, int end) {
  if (!g->timing) return;
  // inside a capture the record becomes an event node, so the replayed graph
  // still times its stages
  cudaEventRecordWithFlags(g->ev[stage][end], g->stream,
                           g->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  if (end) g->ev_used[stage] = true;
}

// Capacity of the exact-path queue: the fp32 filter leaves about 1% of the
// candidate voxels undecided; 4 per vertex (at least 4M) covers that with a
// wide margin. The forced-exact test mode sends every candidate, so it gets
// the list capacity's worth.
vrt_status size_exact_queue(vrt_grid g) {
  unsigned long long want = std::max<unsigned long long>(4ull * (unsigned long long)g->V_alloc, 1ull << 22);
  if (g->force_exact) want = std::max<unsigned long long>(want, std::min<unsigned long long>(g->list_cap, 1ull << 28));
  want = std::min<unsigned long long>(want, 0xffffffffull);
  if (g->xq && g->xq_cap >= want) return VRT_OK;
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  dfree(g, g->xq);
  g->xq_cap = 0;
  VRT_CUDA(g, dalloc(g, &g->xq, (size_t)want));
  g->xq_cap = (uint32_t)want;
  return VRT_OK;
}

// Instrumented trace: the touch bitmaps, (re)sized for the current list
// capacity and vertex count.
vrt_status size_touch_bitmaps(vrt_grid g) {
  const size_t lw = (size_t)(g->list_cap / 32 + 1), vw = (size_t)(g->V / 32 + 1);
  const size_t nv = (size_t)g->n * g->n * g->n;
  if (g->touch_list_words < lw) {
    dfree(g, g->touch_list);
    g->touch_list_words = 0;
    VRT_CUDA(g, dalloc(g, &g->touch_list, lw));
    g->touch_list_words = lw;
  }
  if (g->touch_vert_words < vw) {
    dfree(g, g->touch_vert);
    g->touch_vert_words = 0;
    VRT_CUDA(g, dalloc(g, &g->touch_vert, vw));
    g->touch_vert_words = vw;
  }
  if (!g->touch_vox) VRT_CUDA(g, dalloc(g, &g->touch_vox, nv / 32));
  return VRT_OK;
}

void free_all(vrt_grid g) {
  if (g->graph_exec) {
    cudaGraphExecDestroy(g->graph_exec);
    g->graph_exec = nullptr;
  }
  if (g->cap_stream) {
    cudaStreamDestroy(g->cap_stream);
    g->cap_stream = nullptr;
  }
  for (int i = 0; i < VRT_N_STAGES; ++i)
    for (int j = 0; j < 2; ++j)
      if (g->ev[i][j]) { cudaEventDestroy(g->ev[i][j]); g->ev[i][j] = nullptr; }
  dfree(g, g->raw); dfree(g, g->flags); dfree(g, g->pos); dfree(g, g->nrm); dfree(g, g->order);
  dfree(g, g->word); dfree(g, g->cur); dfree(g, g->vis); dfree(g, g->bdist); dfree(g, g->btmp);
  dfree(g, g->need); dfree(g, g->eroded); dfree(g, g->cdist); dfree(g, g->emean); dfree(g, g->lists); dfree(g, g->tile_state);
  dfree(g, g->xq); dfree(g, g->rec); dfree(g, g->rank);
  dfree(g, g->mips); dfree(g, g->vq[0]); dfree(g, g->vq[1]); dfree(g, g->pq[0]); dfree(g, g->pq[1]);
  dfree(g, g->resume);
  dfree(g, g->shade); dfree(g, g->shade_mask);
  dfree(g, g->touch_list); dfree(g, g->touch_vert); dfree(g, g->touch_vox);
  g->touch_list_words = g->touch_vert_words = 0;
  dfree(g, g->st);
}

}  // namespace

extern "C" {

vrt_status vrt_create_grid(const vrt_grid_desc* desc, void* cuda_stream, vrt_grid* out) {
  if (!out) return fail(nullptr, VRT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(nullptr, VRT_ERR_INVALID_ARG, "desc is NULL");
  const int n = desc->n;
  if (n < 16 || n > 512 || (n & (n - 1)))
    return fail(nullptr, VRT_ERR_INVALID_ARG, "grid side must be a power of two in [16, 512]");
  if (!(desc->radius > 0.0f) || desc->radius > 4.0f)
    return fail(nullptr, VRT_ERR_INVALID_ARG, "radius must be in (0, 4]");
  if (desc->occ_scale < 0 || desc->occ_scale > 65535)
    return fail(nullptr, VRT_ERR_INVALID_ARG, "occ_scale must be in [0, 65535]");
  vrt_grid g = new (std::nothrow) vrt_grid_s();
  if (!g) return fail(nullptr, VRT_ERR_OOM, "host allocation failed");
  g->n = n;
  while ((1 << g->log2n) < n) ++g->log2n;
  g->log2nb = g->log2n - 2;
  g->R = (int)std::nearbyint((double)desc->radius * 16384.0);
  g->RL = g->R + kListMarginUnits;
  g->r = (float)g->R / kUnits;
  g->r_min = desc->r_min > 0 ? desc->r_min : 0.5f;
  g->occ_scale = desc->occ_scale > 0 ? desc->occ_scale : 32;
  g->max_frag_desc = desc->max_fragments;
  g->stream = (cudaStream_t)cuda_stream;
  const size_t nv = (size_t)n * n * n;
  const size_t nb = nv / 64;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  chk(dalloc(g, &g->word, nv));
  chk(dalloc(g, &g->cur, nv));
  chk(dalloc(g, &g->vis, nv / 32));
  chk(dalloc(g, &g->need, nv / 32));
  chk(dalloc(g, &g->bdist, nb));
  chk(dalloc(g, &g->btmp, nb));
  g->n_tiles = (uint32_t)(nv / 4096);
  chk(dalloc(g, &g->tile_state, g->n_tiles));
  chk(dalloc(g, &g->st, 1));
  g->vq_cap = (uint32_t)nv;  // a voxel enters the repair queue at most once per list build
  chk(dalloc(g, &g->vq[0], g->vq_cap));
  chk(dalloc(g, &g->vq[1], g->vq_cap));
  if (e == cudaSuccess) chk(cudaMemsetAsync(g->st, 0, sizeof(DevStatus), g->stream));
  if (e == cudaSuccess) chk(cudaMemsetAsync(g->word, 0, nv * 4, g->stream));
  if (e == cudaSuccess) chk(cudaMemsetAsync(g->need, 0, nv / 8, g->stream));
  if (e != cudaSuccess) {
    vrt_status s = cuda_fail(nullptr, e, "vrt_create_grid");
    free_all(g);
    delete g;
    return s;
  }
  // pyramid offsets
  long long off = 0, m = n;
  g->n_levels = 0;
  while (m >= 1) {
    g->lev_off[g->n_levels++] = off;
    off += m * m * m;
    m >>= 1;
  }
  *out = g;
  return VRT_OK;
}

vrt_status vrt_upload_segments(vrt_grid g, const float* xyz, int32_t stride, int64_t n_vertices,
                               const int64_t* offsets, int64_t n_polylines, int32_t on_device) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (stride != 3 && stride != 4) return fail(g, VRT_ERR_INVALID_ARG, "stride must be 3 or 4");
  if (n_vertices < 0 || n_polylines < 0 || n_vertices >= (1ll << 31))
    return fail(g, VRT_ERR_INVALID_ARG, "bad vertex or polyline count");
  if (n_vertices > 0 && !xyz) return fail(g, VRT_ERR_INVALID_ARG, "xyz is NULL");
  if (!offsets) return fail(g, VRT_ERR_INVALID_ARG, "polyline_offsets is NULL");
  if (offsets[0] != 0 || offsets[n_polylines] != n_vertices)
    return fail(g, VRT_ERR_INVALID_ARG, "offsets must start at 0 and end at n_vertices");
  std::vector<uint8_t> fl((size_t)n_vertices, 0);
  for (long long p = 0; p < n_polylines; ++p) {
    if (offsets[p + 1] < offsets[p]) return fail(g, VRT_ERR_INVALID_ARG, "offsets must not decrease");
    if (offsets[p + 1] > offsets[p]) {
      fl[offsets[p]] |= kFirst;
      fl[offsets[p + 1] - 1] |= kLast;
    }
  }
  if (!on_device && !host_coords_ok(xyz, stride, n_vertices))
    return fail(g, VRT_ERR_INVALID_ARG, "coordinates must be finite and in [-256, 768)");
  const long long V = n_vertices;
  if (V > g->V_alloc) {
    VRT_CUDA(g, cudaStreamSynchronize(g->stream));
    dfree(g, g->raw); dfree(g, g->flags); dfree(g, g->pos); dfree(g, g->nrm); dfree(g, g->order);
    g->V_alloc = 0;
    VRT_CUDA(g, dalloc(g, &g->raw, 3 * (size_t)V + 6));
    VRT_CUDA(g, dalloc(g, &g->flags, (size_t)V));
    if (g->n >= kOrderMinSide) VRT_CUDA(g, dalloc(g, &g->order, (size_t)V));
    VRT_CUDA(g, dalloc(g, &g->pos, (size_t)V + 1));
    VRT_CUDA(g, dalloc(g, &g->nrm, (size_t)V + 1));
    g->V_alloc = V;
  }
  // Default capacity: a tube of length L and list radius rl touches fewer than
  // (L + 2 rl + 2) (2 rl + 2)^2 voxels; 0.9 of that at the mean segment
  // length (about 2.5x the fragments measured on the synthetic sets), at
  // least 16 per vertex.
  const double rl = (double)g->RL / 16384.0;
  double mean_len = 0.0;
  {
    std::vector<float> hx;
    const float* hp = xyz;
    int hs = stride;
    if (on_device && V > 0) {
      hx.resize((size_t)V * 3);
      VRT_CUDA(g, cudaMemcpy2D(hx.data(), 3 * sizeof(float), xyz, (size_t)stride * sizeof(float),
                               3 * sizeof(float), (size_t)V, cudaMemcpyDeviceToHost));
      hp = hx.data();
      hs = 3;
    }
    double sum = 0.0;
    long long nseg = 0;
    for (long long i = 0; i + 1 < V; ++i) {
      if (fl[i] & kLast) continue;
      const double dx = hp[(i + 1) * hs] - hp[i * hs], dy = hp[(i + 1) * hs + 1] - hp[i * hs + 1],
                   dz = hp[(i + 1) * hs + 2] - hp[i * hs + 2];
      sum += std::sqrt(dx * dx + dy * dy + dz * dz);
      ++nseg;
    }
    mean_len = nseg ? sum / (double)nseg : 0.0;
  }
  const double per = std::max(16.0, 0.9 * (mean_len + 2 * rl + 2) * (2 * rl + 2) * (2 * rl + 2));
  unsigned long long cap = g->max_frag_desc ? g->max_frag_desc
                                            : (unsigned long long)(per * (double)std::max(V, 1ll));
  cap = std::min<unsigned long long>(cap, kCulledStart - 1ull);
  if (cap != g->list_cap || !g->lists) {
    VRT_CUDA(g, cudaStreamSynchronize(g->stream));
    dfree(g, g->lists);
    dfree(g, g->rec);
    dfree(g, g->rank);
    g->list_cap = 0;
    VRT_CUDA(g, dalloc(g, &g->lists, (size_t)cap));
    VRT_CUDA(g, dalloc(g, &g->rec, (size_t)cap));
    VRT_CUDA(g, dalloc(g, &g->rank, (size_t)cap));
    g->list_cap = cap;
  }
  {
    vrt_status s = size_exact_queue(g);
    if (s != VRT_OK) return s;
  }
  g->V = V;
  g->P = n_polylines;
  if (V > 0) {
    VRT_CUDA(g, cudaMemcpyAsync(g->flags, fl.data(), (size_t)V, cudaMemcpyHostToDevice, g->stream));
    vrt_status s = copy_vertices(g, 0, V, xyz, stride, on_device);
    if (s != VRT_OK) return s;
    if (g->order) {
      s = build_order(g, offsets, n_polylines);
      if (s != VRT_OK) return s;
    }
    VRT_CUDA(g, cudaStreamSynchronize(g->stream));  // fl is a host temporary
  }
  g->stage = 1;
  g->mips_valid = false;
  g->dirty_lo = 0;
  g->dirty_hi = V;
  return VRT_OK;
}

vrt_status vrt_update_vertices(vrt_grid g, int64_t first_vertex, int64_t n_vertices,
                               const float* xyz, int32_t stride, int32_t on_device) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (g->stage < 1) return fail(g, VRT_ERR_STATE, "vrt_upload_segments first");
  if (stride != 3 && stride != 4) return fail(g, VRT_ERR_INVALID_ARG, "stride must be 3 or 4");
  if (first_vertex < 0 || n_vertices < 0 || first_vertex + n_vertices > g->V)
    return fail(g, VRT_ERR_INVALID_ARG, "vertex range outside the uploaded set");
  if (n_vertices > 0 && !xyz) return fail(g, VRT_ERR_INVALID_ARG, "xyz is NULL");
  // the per-frame path checks coordinates on the device (ingest), for host and
  // device input alike; vrt_sync reports a bad one
  vrt_status s = copy_vertices(g, first_vertex, n_vertices, xyz, stride, on_device);
  if (s != VRT_OK) return s;
  if (n_vertices > 0) {  // these vertices and the neighbours whose clip normals they enter
    const long long lo = std::max<long long>(0, first_vertex - 1);
    const long long hi = std::min<long long>(g->V, first_vertex + n_vertices + 1);
    if (g->dirty_lo >= g->dirty_hi) {
      g->dirty_lo = lo;
      g->dirty_hi = hi;
    } else {
      g->dirty_lo = std::min(g->dirty_lo, lo);
      g->dirty_hi = std::max(g->dirty_hi, hi);
    }
  }
  g->stage = 1;
  g->mips_valid = false;
  return VRT_OK;
}

vrt_status vrt_voxelize(vrt_grid g) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (g->stage < 1) return fail(g, VRT_ERR_STATE, "vrt_upload_segments first");
  const size_t nv = (size_t)g->n * g->n * g->n;
  // clear the counters (everything after the error word)
  VRT_CUDA(g, cudaMemsetAsync((char*)g->st + sizeof(unsigned int), 0,
                              sizeof(DevStatus) - sizeof(unsigned int), g->stream));
  VRT_CUDA(g, cudaMemsetAsync(g->word, 0, nv * 4, g->stream));
  for (int i = 0; i < VRT_N_STAGES; ++i) g->ev_used[i] = false;
  stage_mark(g, ST_INGEST, 0);
  // the vertices that changed since the last ingest (all of them after an upload)
  g->launches += launch_ingest(g->raw, g->flags, g->dirty_lo, g->dirty_hi, g->pos, g->nrm, g->st,
                               g->stream);
  g->dirty_lo = g->dirty_hi = 0;
  stage_mark(g, ST_INGEST, 1);
  stage_mark(g, ST_PASS1, 0);
  g->launches += launch_pass1(g->pos, g->nrm, g->order, g->V, gdev(g), g->stream);
  g->launches += launch_brick_dist(gdev(g), g->btmp, g->bdist, g->stream);
  stage_mark(g, ST_PASS1, 1);
  VRT_CUDA(g, cudaGetLastError());
  g->stage = 2;
  g->mips_valid = false;
  return VRT_OK;
}

vrt_status vrt_build_mips(vrt_grid g) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (g->stage < 2) return fail(g, VRT_ERR_STATE, "vrt_voxelize first");
  if (!g->mips) VRT_CUDA(g, dalloc(g, (float**)&g->mips, (size_t)(g->lev_off[g->n_levels - 1] + 1)));
  stage_mark(g, ST_MIPS, 0);
  g->launches += launch_mips(gdev(g), g->mips, g->mips_fmt, g->lev_off, g->n_levels, g->stream);
  ++g->mips_id;
  stage_mark(g, ST_MIPS, 1);
  VRT_CUDA(g, cudaGetLastError());
  g->mips_valid = true;
  return VRT_OK;
}

vrt_status vrt_cull(vrt_grid g, const vrt_camera* cam, const vrt_render_params* p) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (!p) return fail(g, VRT_ERR_INVALID_ARG, "params is NULL");
  if (g->stage < 2) return fail(g, VRT_ERR_STATE, "vrt_voxelize first");
  if (p->cull < 0 || p->cull > 2) return fail(g, VRT_ERR_INVALID_ARG, "cull must be 0, 1 or 2");
  if (p->cull && !camera_ok(cam)) return fail(g, VRT_ERR_INVALID_ARG, "bad camera");
  if (p->cull && !(p->alpha > 0.0f && p->alpha <= 1.0f))
    return fail(g, VRT_ERR_INVALID_ARG, "alpha must be in (0, 1]");
  const size_t nv = (size_t)g->n * g->n * g->n;
  const GridDev d = gdev(g);
  // automatic: cull unless the last culled build kept more than 95% of the
  // occupied voxels (then culling costs more than it saves); look again every
  // 8 builds
  int cull = p->cull;
  if (cull == 2) {
    cull = g->auto_vis_frac < 0.0 || g->auto_vis_frac <= 0.95 || g->auto_skipped >= 8;
    g->auto_skipped = cull ? 0 : g->auto_skipped + 1;
  }
  // reset the list-build counters (scan tile counter .. end)
  const size_t off = offsetof(DevStatus, sum_count_field);
  VRT_CUDA(g, cudaMemsetAsync((char*)g->st + off, 0, sizeof(DevStatus) - off, g->stream));
  VRT_CUDA(g, cudaMemsetAsync((char*)g->st + offsetof(DevStatus, occupied_voxels), 0, sizeof(unsigned int), g->stream));
  VRT_CUDA(g, cudaMemsetAsync(g->tile_state, 0, (size_t)g->n_tiles * 8, g->stream));
  stage_mark(g, ST_CULL, 0);
  if (cull) {
    if (!g->eroded) VRT_CUDA(g, dalloc(g, &g->eroded, nv));
    if (!g->cdist) VRT_CUDA(g, dalloc(g, &g->cdist, nv / 64));
    if (!g->emean) VRT_CUDA(g, dalloc(g, &g->emean, nv / 64));
    // the exact-path queue is free between pass 1's exact decisions and pass 2:
    // the cull keeps its queue of occupied voxels there
    g->launches += launch_cull(d, host_cam(cam), p->alpha, g->eroded, g->btmp, g->cdist, g->emean,
                               g->cull_depth, reinterpret_cast<uint32_t*>(g->xq),
                               2ull * g->xq_cap, g->stream);
  } else {
    VRT_CUDA(g, cudaMemsetAsync(g->vis, 0xff, nv / 8, g->stream));
  }
  stage_mark(g, ST_CULL, 1);
  stage_mark(g, ST_SCAN, 0);
  g->launches += launch_scan(d, cull ? 0 : 1, g->tile_state, g->n_tiles, g->scan_stall,
                             g->scan_stall >= 0 ? kSpinLimitTest : 0, g->stream);
  g->launches += launch_finalize(d, g->stream);
  stage_mark(g, ST_SCAN, 1);
  stage_mark(g, ST_PASS2, 0);
  g->launches += launch_scatter(d, cull ? 1 : 0, nullptr, nullptr, g->stream);
  stage_mark(g, ST_PASS2, 1);
  VRT_CUDA(g, cudaGetLastError());
  g->culled = cull ? 1 : 0;
  ++g->build_id;
  g->stage = 3;
  return VRT_OK;
}

vrt_status vrt_trace(vrt_grid g, const vrt_camera* cam, const vrt_render_params* p, float* rgba,
                     int32_t* first_id, float* first_t) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (!p || !rgba) return fail(g, VRT_ERR_INVALID_ARG, "params or rgba_out is NULL");
  if (!camera_ok(cam)) return fail(g, VRT_ERR_INVALID_ARG, "bad camera");
  if (!(p->alpha > 0.0f && p->alpha <= 1.0f)) return fail(g, VRT_ERR_INVALID_ARG, "alpha must be in (0, 1]");
  if (p->ao_cones != 0 && p->ao_cones != 6) return fail(g, VRT_ERR_INVALID_ARG, "ao_cones must be 0 or 6");
  if (p->k != 0 && p->k != 1 && p->k != 8 && p->k != 16 && p->k != 32)
    return fail(g, VRT_ERR_INVALID_ARG, "k must be 0, 1, 8, 16 or 32");
  if (g->stage < 3) return fail(g, VRT_ERR_STATE, "vrt_cull first");
  if (p->ao_cones && !g->mips_valid) return fail(g, VRT_ERR_STATE, "vrt_build_mips first (ambient occlusion)");
  if (p->voxel_shading != 0 && p->voxel_shading != 1)
    return fail(g, VRT_ERR_INVALID_ARG, "voxel_shading must be 0 or 1");
  double light[3] = {0.0, 0.0, 0.0};
  if (p->voxel_shading) {
    const double l2 = (double)p->light[0] * p->light[0] + (double)p->light[1] * p->light[1] +
                      (double)p->light[2] * p->light[2];
    if (!(l2 > 0.0) || !std::isfinite(l2))
      return fail(g, VRT_ERR_INVALID_ARG, "light must be a finite non-zero direction");
    for (int k = 0; k < 3; ++k) light[k] = p->light[k] / std::sqrt(l2);
    if (!g->mips_valid) return fail(g, VRT_ERR_STATE, "vrt_build_mips first (voxel shading)");
  }
  int K;
  if (p->alpha >= 1.0f) {
    K = 1;
  } else if (p->k > 1) {
    K = p->k;
  } else {
    const double need = std::ceil(std::log(1e-4) / std::log(1.0 - (double)p->alpha));
    K = need <= 8 ? 8 : (need <= 16 ? 16 : 32);
  }
  const uint32_t npx = (uint32_t)cam->width * (uint32_t)cam->height;
  if (g->culled && npx > g->pq_cap) {
    VRT_CUDA(g, cudaStreamSynchronize(g->stream));
    dfree(g, g->pq[0]); dfree(g, g->pq[1]); dfree(g, g->resume);
    g->pq_cap = 0;
    VRT_CUDA(g, dalloc(g, &g->pq[0], npx));
    VRT_CUDA(g, dalloc(g, &g->pq[1], npx));
    VRT_CUDA(g, dalloc(g, &g->resume, 2 * (size_t)npx));
    g->pq_cap = npx;
  }
  const size_t nv = (size_t)g->n * g->n * g->n;
  ShadeArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  if (p->voxel_shading) {
    if (!g->shade) VRT_CUDA(g, dalloc(g, &g->shade, nv));
    if (!g->shade_mask) VRT_CUDA(g, dalloc(g, &g->shade_mask, nv / 32));
    sa.g = gdev(g);
    sa.mips = g->mips;
    sa.mips_fmt = g->mips_fmt;
    for (int l = 0; l < 11; ++l) sa.lev_off[l] = g->lev_off[l];
    sa.n_levels = g->n_levels;
    sa.ao = p->ao_cones ? 1 : 0;
    sa.lx = (float)light[0]; sa.ly = (float)light[1]; sa.lz = (float)light[2];
    sa.shade = g->shade;
    sa.mask = g->shade_mask;
    uint32_t lb[3];
    std::memcpy(lb, &sa.lx, 4); std::memcpy(lb + 1, &sa.ly, 4); std::memcpy(lb + 2, &sa.lz, 4);
    const uint64_t key[4] = {g->build_id, g->mips_id, ((uint64_t)lb[0] << 32) | lb[1],
                             ((uint64_t)lb[2] << 32) | (uint64_t)sa.ao};
    if (std::memcmp(key, g->shade_key, sizeof(key)) != 0) {
      stage_mark(g, ST_SHADE, 0);
      g->launches += launch_shade(sa, g->stream);
      stage_mark(g, ST_SHADE, 1);
      std::memcpy(g->shade_key, key, sizeof(key));
    }
    g->shade_valid = true;
  }
  TraceArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = gdev(g);
  make_camdev(host_cam(cam), a.cam);
  a.pos = g->pos; a.nrm = g->nrm;
  a.n_vert = (uint32_t)g->V;
  a.count = g->trace_counters;
  a.alpha = p->alpha; a.ao = p->voxel_shading ? 2 : (p->ao_cones ? 1 : 0);
  a.shade = p->voxel_shading ? g->shade : nullptr;
  a.mips = g->mips;
  a.mips_fmt = g->mips_fmt;
  for (int l = 0; l < 11; ++l) a.lev_off[l] = g->lev_off[l];
  a.n_levels = g->n_levels;
  a.rgba = reinterpret_cast<float4*>(rgba);
  a.first_id = first_id;
  a.first_t = first_t;
  a.need = g->need;
  a.vq_cap = g->vq_cap;
  a.pq_cap = g->pq_cap;
  a.vq = g->vq[0]; a.vq_cnt = &g->st->vq_cnt[0];
  a.pq = g->pq[0]; a.pq_cnt = &g->st->pq_cnt[0];
  a.resume = g->culled ? g->resume : nullptr;
  // Traces before the next-to-last repair round stop after a few queued
  // voxels (cheap, may need another round); the re-trace of the next-to-last
  // round queues without limit, so the last round always completes.
  a.max_queue = kMaxRepairRounds >= 2 ? kRayQueueLimit : 0xffffffffu;
  VRT_CUDA(g, cudaMemsetAsync((char*)g->st + offsetof(DevStatus, vq_cnt), 0,
                              4 * sizeof(unsigned int), g->stream));
  VRT_CUDA(g, cudaMemsetAsync((char*)g->st + offsetof(DevStatus, tr_next), 0,
                              sizeof(unsigned int) * (kMaxRepairRounds + 1), g->stream));
  a.work_next = &g->st->tr_next[0];
  a.short_list = g->short_list;
  a.ray_keys = g->ray_keys;
  a.key16 = g->key16;
  a.tile_w = g->tile_w;
  if (g->trace_counters) {  // touch bitmaps, cleared for this trace
    if (const vrt_status ts = size_touch_bitmaps(g)) return ts;
    VRT_CUDA(g, cudaMemsetAsync(g->touch_list, 0, g->touch_list_words * 4, g->stream));
    VRT_CUDA(g, cudaMemsetAsync(g->touch_vert, 0, g->touch_vert_words * 4, g->stream));
    VRT_CUDA(g, cudaMemsetAsync(g->touch_vox, 0, nv / 8, g->stream));
    a.touch_list = g->touch_list;
    a.touch_vert = g->touch_vert;
    a.touch_vox = g->touch_vox;
  }
  stage_mark(g, ST_TRACE, 0);
  g->launches += launch_trace(a, K, g->stream);
  stage_mark(g, ST_TRACE, 1);
  if (g->culled) {
    stage_mark(g, ST_REPAIR, 0);
    const GridDev d = gdev(g);
    for (int r = 0; r < kMaxRepairRounds; ++r) {
      const int ci = r & 1, nx = ci ^ 1;
      g->launches += launch_repair_alloc(d, g->vq[ci], &g->st->vq_cnt[ci], &g->st->pq_cnt[ci],
                                         g->vq_cap, g->stream);
      if (p->voxel_shading) {
        ShadeArgs sr = sa;
        sr.vq = g->vq[ci];
        sr.vq_cnt = &g->st->vq_cnt[ci];
        sr.vq_cap = g->vq_cap;
        g->launches += launch_shade_repair(sr, g->stream);
      }
      g->launches += launch_scatter(d, 2, g->need, &g->st->vq_cnt[ci], g->stream);
      g->launches += launch_repair_clear(d, g->need, g->vq[ci], &g->st->vq_cnt[ci], g->vq_cap, nx, g->stream);
      TraceArgs b = a;
      b.pix_list = g->pq[ci];
      b.pix_count = &g->st->pq_cnt[ci];
      b.vq = g->vq[nx]; b.vq_cnt = &g->st->vq_cnt[nx];
      b.pq = g->pq[nx]; b.pq_cnt = &g->st->pq_cnt[nx];
      b.max_queue = (r + 2 >= kMaxRepairRounds) ? 0xffffffffu : kRayQueueLimit;
      b.work_next = &g->st->tr_next[r + 1];
      g->launches += launch_trace(b, K, g->stream);
    }
    stage_mark(g, ST_REPAIR, 1);
  }
  if (g->trace_counters) {
    VRT_CUDA(g, cudaMemsetAsync((char*)g->st + offsetof(DevStatus, tr_u_entries), 0,
                                3 * sizeof(unsigned long long), g->stream));
    g->launches += launch_touch_count(g->touch_list, g->touch_list_words, g->touch_vert,
                                      g->touch_vert_words, g->touch_vox, nv / 32, g->st, g->stream);
  }
  VRT_CUDA(g, cudaGetLastError());
  return VRT_OK;
}

// For automatic culling: the visible share of the last culled list build.
static void note_visibility(vrt_grid g, const DevStatus& hs) {
  if (g->culled && hs.occupied_voxels) g->auto_vis_frac = (double)hs.visible_voxels / hs.occupied_voxels;
}

vrt_status vrt_sync(vrt_grid g) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  DevStatus hs;
  VRT_CUDA(g, cudaMemcpy(&hs, g->st, sizeof(hs), cudaMemcpyDeviceToHost));
  note_visibility(g, hs);
  uint32_t e = hs.err;
  if (g->culled && hs.vq_cnt[kMaxRepairRounds & 1] != 0) e |= kErrRepair;
  if (hs.err) VRT_CUDA(g, cudaMemset(g->st, 0, sizeof(unsigned int)));
  if (e & kErrRange) return fail(g, VRT_ERR_INVALID_ARG, "device coordinates out of range or not finite");
  if (e & kErrOverflow) return fail(g, VRT_ERR_OVERFLOW, "a 16-bit voxel field or the list capacity overflowed");
  if (e & kErrTimeout) return fail(g, VRT_ERR_TIMEOUT, "a bounded device wait gave up");
  if (e & kErrRepair) return fail(g, VRT_ERR_TIMEOUT, "culling repair did not converge");
  if (e & kErrBounds) return fail(g, VRT_ERR_BOUNDS, "index out of bounds");
  return VRT_OK;
}

vrt_status vrt_get_stats(vrt_grid g, vrt_stats* out) {
  if (!g || !out) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  DevStatus hs;
  VRT_CUDA(g, cudaMemcpy(&hs, g->st, sizeof(hs), cudaMemcpyDeviceToHost));
  note_visibility(g, hs);
  out->fragments = hs.F;
  out->fragments_listed = hs.listed;
  out->sum_occupancy = hs.sum_q;
  out->exact_decisions = hs.exact_decisions;
  out->occupied_voxels = hs.occupied_voxels;
  out->visible_voxels = hs.visible_voxels;
  out->repaired_voxels = hs.repaired_voxels;
  out->repair_rounds = hs.repair_rounds;
  out->max_count = hs.max_count;
  out->status_bits = hs.err;
  out->kernel_launches = g->launches;
  out->retraced_pixels = hs.retraced_pixels;
  out->trace_entries = hs.tr_entries;
  out->trace_capsule_tests = hs.tr_capsule;
  out->trace_voxels = hs.tr_voxels;
  out->trace_steps = hs.tr_steps;
  out->trace_wholewarp_voxels = hs.tr_ww_voxels;
  out->trace_wholewarp_entries = hs.tr_ww_entries;
  out->trace_hits = hs.tr_hits;
  for (int k = 0; k < 4; ++k) out->trace_cycles[k] = hs.tr_cycles[k];
  out->trace_unique_entries = hs.tr_u_entries;
  out->trace_unique_vertices = hs.tr_u_vertices;
  out->trace_unique_voxels = hs.tr_u_voxels;
  return VRT_OK;
}

vrt_status vrt_read_grid(vrt_grid g, uint32_t* words) {
  if (!g || !words) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  const int n = g->n;
  const size_t nv = (size_t)n * n * n;
  std::vector<uint32_t> w(nv);
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  VRT_CUDA(g, cudaMemcpy(w.data(), g->word, nv * 4, cudaMemcpyDeviceToHost));
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) words[((size_t)z * n + y) * n + x] = w[brick_index(x, y, z, g->log2nb)];
  return VRT_OK;
}

vrt_status vrt_read_lists(vrt_grid g, uint32_t* start, uint32_t* len, uint32_t* ids, uint64_t cap,
                          uint64_t* n_ids) {
  if (!g || !start || !len) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  if (g->stage < 3) return fail(g, VRT_ERR_STATE, "vrt_cull first");
  const int n = g->n;
  const size_t nv = (size_t)n * n * n;
  std::vector<uint32_t> w(nv), c(nv), vis(nv / 32);
  DevStatus hs;
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  VRT_CUDA(g, cudaMemcpy(w.data(), g->word, nv * 4, cudaMemcpyDeviceToHost));
  VRT_CUDA(g, cudaMemcpy(c.data(), g->cur, nv * 4, cudaMemcpyDeviceToHost));
  VRT_CUDA(g, cudaMemcpy(vis.data(), g->vis, nv / 8, cudaMemcpyDeviceToHost));
  VRT_CUDA(g, cudaMemcpy(&hs, g->st, sizeof(hs), cudaMemcpyDeviceToHost));
  note_visibility(g, hs);
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const uint32_t i = brick_index(x, y, z, g->log2nb);
        const size_t o = ((size_t)z * n + y) * n + x;
        const uint32_t cnt = w[i] & 0xffffu;
        if (cnt && ((vis[i >> 5] >> (i & 31)) & 1u)) { start[o] = c[i] - cnt; len[o] = cnt; }
        else { start[o] = 0; len[o] = 0; }
      }
  const uint64_t tot = std::min<uint64_t>(hs.list_tail, g->list_cap);
  if (n_ids) *n_ids = tot;
  if (ids && tot) VRT_CUDA(g, cudaMemcpy(ids, g->lists, std::min(tot, cap) * 4, cudaMemcpyDeviceToHost));
  return VRT_OK;
}

vrt_status vrt_read_mips(vrt_grid g, float* host, uint64_t n_floats) {
  if (!g || !host) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  if (!g->mips_valid) return fail(g, VRT_ERR_STATE, "vrt_build_mips first");
  const uint64_t tot = std::min<uint64_t>((uint64_t)g->lev_off[g->n_levels - 1] + 1, n_floats);
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  if (g->mips_fmt == kMipsF32) {
    VRT_CUDA(g, cudaMemcpy(host, g->mips, tot * 4, cudaMemcpyDeviceToHost));
    return VRT_OK;
  }
  std::vector<uint16_t> h(tot);
  VRT_CUDA(g, cudaMemcpy(h.data(), g->mips, tot * 2, cudaMemcpyDeviceToHost));
  for (uint64_t i = 0; i < tot; ++i) host[i] = g->mips_fmt == kMipsF16 ? half_to_float(h[i])
                                                                       : bf16_to_float(h[i]);
  return VRT_OK;
}

vrt_status vrt_read_shading(vrt_grid g, float* values, uint8_t* valid) {
  if (!g || !values) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  if (!g->shade_valid) return fail(g, VRT_ERR_STATE, "no trace has used voxel shading");
  const int n = g->n;
  const size_t nv = (size_t)n * n * n;
  std::vector<float> v(nv);
  std::vector<uint32_t> m(nv / 32);
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  VRT_CUDA(g, cudaMemcpy(v.data(), g->shade, nv * 4, cudaMemcpyDeviceToHost));
  VRT_CUDA(g, cudaMemcpy(m.data(), g->shade_mask, nv / 8, cudaMemcpyDeviceToHost));
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const uint32_t i = brick_index(x, y, z, g->log2nb);
        const size_t o = ((size_t)z * n + y) * n + x;
        const bool ok = (m[i >> 5] >> (i & 31)) & 1u;
        values[o] = ok ? v[i] : 0.0f;
        if (valid) valid[o] = ok ? 1 : 0;
      }
  return VRT_OK;
}

}  // extern "C"

// Allocate every buffer a frame with these parameters sizes lazily (the
// pyramid, shading field, cull fields, repair queues for this image size,
// instrumented-trace bitmaps), so that the frame's calls allocate nothing and
// can be captured into a CUDA graph. May synchronize the grid's stream.
vrt_status vrt::prepare_frame(vrt_grid g, const vrt_camera* cam, const vrt_render_params* p) {
  const size_t nv = (size_t)g->n * g->n * g->n;
  if ((p->ao_cones || p->voxel_shading) && !g->mips)
    VRT_CUDA(g, dalloc(g, (float**)&g->mips, (size_t)(g->lev_off[g->n_levels - 1] + 1)));
  if (p->voxel_shading && !g->shade) VRT_CUDA(g, dalloc(g, &g->shade, nv));
  if (p->voxel_shading && !g->shade_mask) VRT_CUDA(g, dalloc(g, &g->shade_mask, nv / 32));
  if (p->cull) {
    if (!g->eroded) VRT_CUDA(g, dalloc(g, &g->eroded, nv));
    if (!g->cdist) VRT_CUDA(g, dalloc(g, &g->cdist, nv / 64));
    if (!g->emean) VRT_CUDA(g, dalloc(g, &g->emean, nv / 64));
    const uint32_t npx = (uint32_t)cam->width * (uint32_t)cam->height;
    if (npx > g->pq_cap) {
      VRT_CUDA(g, cudaStreamSynchronize(g->stream));
      dfree(g, g->pq[0]); dfree(g, g->pq[1]); dfree(g, g->resume);
      g->pq_cap = 0;
      VRT_CUDA(g, dalloc(g, &g->pq[0], npx));
      VRT_CUDA(g, dalloc(g, &g->pq[1], npx));
      VRT_CUDA(g, dalloc(g, &g->resume, 2 * (size_t)npx));
      g->pq_cap = npx;
    }
  }
  if (g->trace_counters) {
    if (const vrt_status ts = size_touch_bitmaps(g)) return ts;
  }
  return VRT_OK;
}

extern "C" {

vrt_status vrt_frame(vrt_grid g, int64_t first_vertex, int64_t n_vertices, const float* xyz,
                     int32_t stride, int32_t on_device, const vrt_camera* cam,
                     const vrt_render_params* p, float* rgba, int32_t* first_id, float* first_t) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (!cam || !p || !rgba) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  auto chain = [&]() -> vrt_status {
    vrt_status r = VRT_OK;
    if (n_vertices > 0) r = vrt_update_vertices(g, first_vertex, n_vertices, xyz, stride, on_device);
    if (r == VRT_OK) r = vrt_voxelize(g);
    if (r == VRT_OK && (p->ao_cones || p->voxel_shading)) r = vrt_build_mips(g);
    if (r == VRT_OK) r = vrt_cull(g, cam, p);
    if (r == VRT_OK) r = vrt_trace(g, cam, p, rgba, first_id, first_t);
    return r;
  };
  if (!g->use_graph || g->stage < 1) return chain();
  // pageable host input cannot be captured (its copy is synchronous)
  if (n_vertices > 0 && !on_device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, xyz) != cudaSuccess || at.type == cudaMemoryTypeUnregistered) {
      cudaGetLastError();
      return chain();
    }
  }
  // every buffer the chain sizes lazily exists before the capture (no
  // allocation may happen inside one)
  if (const vrt_status ps = vrt::prepare_frame(g, cam, p)) return ps;
  if (!g->cap_stream) VRT_CUDA(g, cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = g->stream;
  g->stream = g->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  vrt_status r = VRT_OK;
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) {
    g->capturing = true;
    r = chain();
    g->capturing = false;
    e = cudaStreamEndCapture(g->stream, &graph);
  }
  g->stream = user;
  if (r != VRT_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    std::memset(g->shade_key, 0xff, sizeof(g->shade_key));  // the captured shading never ran
    if (r != VRT_OK) return r;
    return cuda_fail(g, e, "stream capture of the frame");
  }
  if (g->graph_exec) {  // same launch sequence as last frame: update the parameters in place
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(g->graph_exec, graph, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(g->graph_exec);
      g->graph_exec = nullptr;
    }
  }
  cudaError_t ie = cudaSuccess;
  if (!g->graph_exec) ie = cudaGraphInstantiate(&g->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    std::memset(g->shade_key, 0xff, sizeof(g->shade_key));
    return cuda_fail(g, ie, "cudaGraphInstantiate");
  }
  VRT_CUDA(g, cudaGraphLaunch(g->graph_exec, g->stream));
  return VRT_OK;
}

vrt_status vrt_tune_shapes(const vrt_grid_desc* base, const float* xyz, int32_t stride,
                           int64_t n_vertices, const int64_t* offsets, int64_t n_polylines,
                           const vrt_camera* cam, const vrt_render_params* p, const int32_t* sides,
                           int32_t n_sides, const int32_t* tiles, int32_t n_tiles, int32_t frames,
                           int32_t* best_side, int32_t* best_tile, float* ms_out) {
  if (!base || !xyz || !offsets || !cam || !p || !sides || n_sides <= 0 || !tiles || n_tiles <= 0 ||
      frames <= 0 || !best_side || !best_tile)
    return fail(nullptr, VRT_ERR_INVALID_ARG, "NULL argument or empty candidate list");
  if (stride != 3 && stride != 4) return fail(nullptr, VRT_ERR_INVALID_ARG, "stride must be 3 or 4");
  for (int32_t j = 0; j < n_tiles; ++j)
    if (tiles[j] != 2 && tiles[j] != 4 && tiles[j] != 8 && tiles[j] != 16)
      return fail(nullptr, VRT_ERR_INVALID_ARG, "tile widths must be 2, 4, 8 or 16");
  float best = INFINITY;
  *best_side = 0;
  *best_tile = 0;
  std::vector<float> scaled((size_t)n_vertices * 3);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  VRT_CUDA(nullptr, cudaEventCreate(&e0));
  VRT_CUDA(nullptr, cudaEventCreate(&e1));
  vrt_status result = VRT_OK;
  float* out = nullptr;
  const size_t npx = (size_t)cam->width * cam->height;
  if (cudaMalloc((void**)&out, npx * 4 * sizeof(float)) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return fail(nullptr, VRT_ERR_OOM, "output buffer");
  }
  for (int32_t i = 0; i < n_sides && result == VRT_OK; ++i) {
    // the same scene in a grid of side sides[i]: coordinates, radius and camera
    // scale with the side
    const double f = (double)sides[i] / (double)base->n;
    for (int64_t v = 0; v < n_vertices; ++v)
      for (int k = 0; k < 3; ++k) scaled[3 * v + k] = (float)(xyz[v * stride + k] * f);
    vrt_grid_desc d = *base;
    d.n = sides[i];
    d.radius = (float)(base->radius * f);
    vrt_camera c = *cam;
    for (int k = 0; k < 3; ++k) {
      c.eye[k] = (float)(cam->eye[k] * f);
      c.target[k] = (float)(cam->target[k] * f);
    }
    c.ortho_h = (float)(cam->ortho_h * f);
    vrt_grid g = nullptr;
    vrt_status r = vrt_create_grid(&d, nullptr, &g);
    if (r == VRT_OK) r = vrt_upload_segments(g, scaled.data(), 3, n_vertices, offsets, n_polylines, 0);
    for (int32_t j = 0; j < n_tiles; ++j) {
      float ms = INFINITY;
      vrt_status rj = r;
      if (rj == VRT_OK) rj = vrt_set_option(g, VRT_OPT_TRACE_TILE, tiles[j]);
      if (rj == VRT_OK) rj = vrt_frame(g, 0, 0, nullptr, 3, 0, &c, p, out, nullptr, nullptr);  // warm-up
      if (rj == VRT_OK) rj = vrt_sync(g);
      if (rj == VRT_OK) {
        cudaEventRecord(e0, nullptr);
        for (int32_t k = 0; k < frames && rj == VRT_OK; ++k)
          rj = vrt_frame(g, 0, 0, nullptr, 3, 0, &c, p, out, nullptr, nullptr);
        cudaEventRecord(e1, nullptr);
        cudaEventSynchronize(e1);
        if (rj == VRT_OK) rj = vrt_sync(g);
        if (rj == VRT_OK) {
          cudaEventElapsedTime(&ms, e0, e1);
          ms /= (float)frames;
        }
      }
      if (rj != VRT_OK) ms = INFINITY;  // a side that does not work (range, memory) is skipped
      if (ms_out) ms_out[(size_t)i * n_tiles + j] = ms;
      if (ms < best) {
        best = ms;
        *best_side = sides[i];
        *best_tile = tiles[j];
      }
    }
    if (g) vrt_destroy(g);
  }
  cudaFree(out);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*best_side == 0) return fail(nullptr, VRT_ERR_INVALID_ARG, "no candidate rendered the scene");
  return result;
}

vrt_status vrt_tune_grid_side(const vrt_grid_desc* base, const float* xyz, int32_t stride,
                              int64_t n_vertices, const int64_t* offsets, int64_t n_polylines,
                              const vrt_camera* cam, const vrt_render_params* p,
                              const int32_t* sides, int32_t n_sides, int32_t frames,
                              int32_t* best_side, float* ms_out) {
  const int32_t tile = 4;
  int32_t best_tile = 0;
  return vrt_tune_shapes(base, xyz, stride, n_vertices, offsets, n_polylines, cam, p, sides, n_sides,
                         &tile, 1, frames, best_side, &best_tile, ms_out);
}

vrt_status vrt_grid_device_bytes(vrt_grid g, uint64_t* bytes) {
  if (!g || !bytes) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  *bytes = g->dev_bytes;
  return VRT_OK;
}

vrt_status vrt_set_stream(vrt_grid g, void* cuda_stream) {
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  g->stream = (cudaStream_t)cuda_stream;
  return VRT_OK;
}

vrt_status vrt_set_option(vrt_grid g, int32_t option, int64_t value) {
  if (option == VRT_OPT_TEST_SCAN_STALL) {
    if (value < -1 || value >= (1ll << 30)) return fail(g, VRT_ERR_INVALID_ARG, "stall tile must be in [-1, 2^30)");
    if (!g) {
      set_noalloc_scan_stall(value);
      return VRT_OK;
    }
    g->scan_stall = (int)value;
    return VRT_OK;
  }
  if (!g) return fail(nullptr, VRT_ERR_INVALID_ARG, "grid is NULL");
  if (option == VRT_OPT_TRACE_SHORT_LIST) {
    if (value < 0 || value > (int64_t)kShortList)
      return fail(g, VRT_ERR_INVALID_ARG, "short-list limit must be in [0, 1024]");
    g->short_list = (uint32_t)value;
    return VRT_OK;
  }
  if (option == VRT_OPT_TRACE_TILE) {
    if (value != 2 && value != 4 && value != 8 && value != 16)
      return fail(g, VRT_ERR_INVALID_ARG, "trace tile width must be 2, 4, 8 or 16");
    g->tile_w = (int)value;
    return VRT_OK;
  }
  if (option == VRT_OPT_HIT_KEY) {
    if (value != VRT_HIT_KEY_DEPTH_ID && value != VRT_HIT_KEY_16_16)
      return fail(g, VRT_ERR_INVALID_ARG, "hit key must be VRT_HIT_KEY_DEPTH_ID or VRT_HIT_KEY_16_16");
    g->key16 = value == VRT_HIT_KEY_16_16;
    return VRT_OK;
  }
  if (option == VRT_OPT_TRACE_RAY_KEYS) {
    if (value < 1 || value > kRayKeys) return fail(g, VRT_ERR_INVALID_ARG, "ray key slots must be in [1, 32]");
    g->ray_keys = (uint32_t)value;
    return VRT_OK;
  }
  if (option == VRT_OPT_FORCE_EXACT) {
    g->force_exact = value ? 1 : 0;
    return g->V_alloc ? size_exact_queue(g) : VRT_OK;
  }
  if (option == VRT_OPT_TRACE_COUNTERS) {
    g->trace_counters = value ? 1 : 0;
    return VRT_OK;
  }
  if (option == VRT_OPT_CULL_DEPTH) {
    if (value < 0 || value > 1000000) return fail(g, VRT_ERR_INVALID_ARG, "cull depth must be in [0, 1e6]");
    g->cull_depth = (float)((double)value / 1000.0);
    return VRT_OK;
  }
  if (option == VRT_OPT_GRAPH) {
    g->use_graph = value != 0;
    return VRT_OK;
  }
  if (option == VRT_OPT_MIPS_FORMAT) {
    if (value != VRT_MIPS_F32 && value != VRT_MIPS_F16 && value != VRT_MIPS_BF16)
      return fail(g, VRT_ERR_INVALID_ARG, "mips format must be VRT_MIPS_F32, _F16 or _BF16");
    if ((int)value != g->mips_fmt) g->mips_valid = false;
    g->mips_fmt = (int)value;
    return VRT_OK;
  }
  if (option == VRT_OPT_STAGE_TIMING) {
    if (value && !g->ev[0][0])
      for (int i = 0; i < VRT_N_STAGES; ++i)
        for (int j = 0; j < 2; ++j) VRT_CUDA(g, cudaEventCreate(&g->ev[i][j]));
    g->timing = value != 0;
    return VRT_OK;
  }
  return fail(g, VRT_ERR_INVALID_ARG, "unknown option");
}

vrt_status vrt_get_stage_ms(vrt_grid g, float* ms, int32_t n) {
  if (!g || !ms || n < 0) return fail(g, VRT_ERR_INVALID_ARG, "NULL argument");
  VRT_CUDA(g, cudaStreamSynchronize(g->stream));
  for (int i = 0; i < n && i < VRT_N_STAGES; ++i) {
    ms[i] = -1.0f;
    if (g->timing && g->ev_used[i]) VRT_CUDA(g, cudaEventElapsedTime(&ms[i], g->ev[i][0], g->ev[i][1]));
  }
  return VRT_OK;
}

const char* vrt_last_error(vrt_grid g) { return g ? g->err.c_str() : g_create_error.c_str(); }

vrt_status vrt_destroy(vrt_grid g) {
  if (!g) return VRT_OK;
  cudaStreamSynchronize(g->stream);
  free_all(g);
  delete g;
  return VRT_OK;
}

}  // extern "C"
