// Serving: a request loop over resident line sets (the vrt_server_* calls of vrt.h).
//
// One scheduler thread owns the sets' grids and the stream slots. Submitting
// threads only copy their request into pinned host memory and queue it. The
// scheduler repeatedly (1) retires frames whose stream work has finished (a
// host callback on the slot's stream flags them), (2) issues the oldest queued
// request of every set that has no frame in flight, onto a free slot, making
// its set resident first (evicting least-recently-used idle sets while the HBM
// budget would be exceeded), and (3) sleeps until a submission or a finished
// frame wakes it. CUDA work is issued with the lock released. Optionally,
// frames of small sets (fewer segments than small_segments) are issued in
// batches: the oldest
// pending frame of each of up to max_batch idle small sets are captured into
// one CUDA graph -- a branch per set, each set's chain on its own stream, all
// joined at the end -- and launched at once on one slot, so their kernels run
// side by side and the host issues one launch for all of them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "launch.h"
#include "vrt.h"

extern thread_local std::string g_create_error;  // message returned by vrt_last_error(NULL)

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct ServerSet {
  vrt_grid_desc desc{};
  std::vector<float> xyz;        // host copy, 3 floats per vertex, kept current
  std::vector<int64_t> offsets;
  int64_t V = 0, P = 0;
  vrt_grid grid = nullptr;
  uint64_t bytes = 0;            // device bytes (measured once resident, else estimated)
  bool busy = false;             // a frame in flight
  uint64_t last_use = 0;
};

struct Request {
  int64_t id = 0;
  int32_t set = 0;
  int64_t first = 0, n = 0;
  float* upd = nullptr;          // pinned, 3 floats per vertex
  size_t upd_cap = 0;
  vrt_camera cam{};
  vrt_render_params p{};
  float* rgba = nullptr;
  int32_t* first_id = nullptr;
  float* first_t = nullptr;
  Clock::time_point t_submit, t_issue;
};

struct Slot {
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> branch;  // a batch's per-set streams (created at first use)
  cudaEvent_t fork = nullptr;        // a batch's fork point on `stream`
  std::vector<cudaEvent_t> join;     // a batch's per-branch ends
  bool busy = false;
  std::atomic<bool> done{false};
  Clock::time_point t_done;
  std::vector<Request> reqs;         // the frame, or the batch's frames, in flight
  struct vrt_server_s* server = nullptr;
};

}  // namespace

struct vrt_server_s {
  int device = 0;
  uint64_t budget = 0;
  uint64_t resident_bytes = 0;
  std::vector<std::unique_ptr<ServerSet>> sets;
  std::deque<Request> pending;
  std::vector<std::unique_ptr<Slot>> slots;
  std::deque<vrt_server_result> results;
  std::multimap<size_t, float*> pinned_free;  // capacity (floats) -> buffer
  std::vector<float*> pinned_all;
  std::mutex mu;
  std::condition_variable cv;     // wakes the scheduler
  std::condition_variable cv_done;  // wakes waiters in poll / destroy
  std::thread th;
  bool stop = false;
  int64_t next_id = 1;
  uint64_t submitted = 0, completed = 0;
  uint64_t tick = 0;
  int evictions = 0;
  int resident_sets = 0;
  int64_t small_segments = 0;  // sets with fewer segments are batched (<= 0: never)
  int max_batch = 16;
  uint64_t batches = 0, batched_frames = 0;
};

namespace {

// Failures of server calls report through vrt_last_error(NULL), whose message
// is kept per host thread.
vrt_status sfail(vrt_server, vrt_status st, const std::string& m) {
  g_create_error = m;
  return st;
}

// Footprint estimate of a set before it has been resident (its measured size
// replaces it afterwards): the grid's voxel arrays, vertex buffers, list and
// record capacity, exact queue, pyramid, cull and repair scratch at 1080p.
uint64_t estimate_bytes(const ServerSet& st) {
  const uint64_t n = (uint64_t)st.desc.n, nv = n * n * n, V = (uint64_t)std::max<int64_t>(st.V, 1);
  const double rl = st.desc.radius + 1.0 / 512.0;
  double mean_len = 1.0;
  {
    double sum = 0;
    int64_t cnt = 0;
    for (int64_t p = 0; p < st.P; ++p)
      for (int64_t i = st.offsets[p]; i + 1 < st.offsets[p + 1]; i += 64) {
        const float* a = &st.xyz[3 * i];
        const float* b = &st.xyz[3 * (i + 1)];
        sum += std::sqrt((double)(b[0] - a[0]) * (b[0] - a[0]) + (double)(b[1] - a[1]) * (b[1] - a[1]) +
                         (double)(b[2] - a[2]) * (b[2] - a[2]));
        ++cnt;
      }
    if (cnt) mean_len = sum / cnt;
  }
  const double per = std::max(16.0, 0.9 * (mean_len + 2 * rl + 2) * (2 * rl + 2) * (2 * rl + 2));
  const uint64_t cap = st.desc.max_fragments ? st.desc.max_fragments : (uint64_t)(per * V);
  const uint64_t xq = std::max<uint64_t>(4 * V, 1ull << 22);
  // words, cursors, marks, fields, pyramid; vertices; lists, records and ranks;
  // exact queue; cull scratch; voxel-space shading field and mask; pixel queues at 1080p
  return nv * 17 + nv / 4 + V * 45 + cap * 14 + xq * 8 + nv * 5 + nv * 4 + nv / 8 + 2073600ull * 40;
}

void CUDART_CB on_frame_done(void* arg) {
  Slot* sl = (Slot*)arg;
  sl->t_done = Clock::now();
  sl->done.store(true);
  std::lock_guard<std::mutex> lk(sl->server->mu);
  sl->server->cv.notify_all();
}

// Make set `k` resident: evict idle sets (least recently used first) while the
// budget would be exceeded, then create and upload it. Scheduler thread, called
// with the lock held; releases it around the CUDA calls. Returns false when it
// does not fit yet (busy sets hold the memory) or on an error (*st_out).
bool make_resident(vrt_server s, std::unique_lock<std::mutex>& lk, int k, vrt_status* st_out) {
  ServerSet& st = *s->sets[k];
  *st_out = VRT_OK;
  if (st.grid) return true;
  if (!st.bytes) st.bytes = estimate_bytes(st);
  while (s->resident_bytes + st.bytes > s->budget) {
    int victim = -1;
    for (size_t i = 0; i < s->sets.size(); ++i) {
      const ServerSet& o = *s->sets[i];
      if (o.grid && !o.busy && (victim < 0 || o.last_use < s->sets[victim]->last_use)) victim = (int)i;
    }
    if (victim < 0) {
      if (s->resident_bytes == 0) break;  // alone: try, its measured size decides
      return false;                       // else wait for busy sets
    }
    ServerSet& v = *s->sets[victim];
    vrt_grid vg = v.grid;
    v.grid = nullptr;
    s->resident_bytes -= v.bytes;
    --s->resident_sets;
    ++s->evictions;
    lk.unlock();
    vrt_destroy(vg);
    lk.lock();
  }
  s->resident_bytes += st.bytes;  // reserved while it is created
  ++s->resident_sets;
  lk.unlock();
  vrt_grid g = nullptr;
  vrt_status r = vrt_create_grid(&st.desc, nullptr, &g);
  if (r == VRT_OK) r = vrt_upload_segments(g, st.xyz.data(), 3, st.V, st.offsets.data(), st.P, 0);
  if (r != VRT_OK && g) {
    vrt_destroy(g);
    g = nullptr;
  }
  uint64_t b = 0;
  if (r == VRT_OK) vrt_grid_device_bytes(g, &b);
  lk.lock();
  if (r == VRT_OK) {  // the measured size replaces the estimate
    s->resident_bytes += b - st.bytes;
    st.bytes = b;
    if (b > s->budget) {  // alone it exceeds the budget
      lk.unlock();
      vrt_destroy(g);
      lk.lock();
      r = VRT_ERR_OOM;
    }
  }
  if (r != VRT_OK) {
    s->resident_bytes -= st.bytes;
    --s->resident_sets;
    *st_out = r;
    return false;
  }
  st.grid = g;
  return true;
}

// Evict idle sets (least recently used first) while the resident sets hold
// more than the budget (buffers sized by a frame can grow a set). Lock held;
// released around the CUDA calls.
void trim(vrt_server s, std::unique_lock<std::mutex>& lk) {
  while (s->resident_bytes > s->budget) {
    int victim = -1;
    for (size_t i = 0; i < s->sets.size(); ++i) {
      const ServerSet& o = *s->sets[i];
      if (o.grid && !o.busy && (victim < 0 || o.last_use < s->sets[victim]->last_use)) victim = (int)i;
    }
    if (victim < 0) return;
    ServerSet& v = *s->sets[victim];
    vrt_grid vg = v.grid;
    v.grid = nullptr;
    s->resident_bytes -= v.bytes;
    --s->resident_sets;
    ++s->evictions;
    lk.unlock();
    vrt_destroy(vg);
    lk.lock();
  }
}

// The calls of one frame of `rq` on its set's grid, on stream `stream`.
vrt_status frame_chain(ServerSet& st, Request& rq, cudaStream_t stream) {
  vrt_grid g = st.grid;
  vrt_status r = vrt_set_stream(g, stream);
  if (r == VRT_OK && rq.n > 0) {
    // the host copy follows every issued update (for uploads after an eviction)
    std::memcpy(&st.xyz[3 * rq.first], rq.upd, sizeof(float) * 3 * (size_t)rq.n);
    r = vrt_update_vertices(g, rq.first, rq.n, rq.upd, 3, 0);
  }
  if (r == VRT_OK) r = vrt_voxelize(g);
  if (r == VRT_OK && (rq.p.ao_cones || rq.p.voxel_shading)) r = vrt_build_mips(g);
  if (r == VRT_OK) r = vrt_cull(g, &rq.cam, &rq.p);
  if (r == VRT_OK) r = vrt_trace(g, &rq.cam, &rq.p, rq.rgba, rq.first_id, rq.first_t);
  return r;
}

// Issue one frame of `rq` on slot `sl` (scheduler thread, lock released).
vrt_status issue(vrt_server s, Slot& sl, Request& rq) {
  vrt_status r = frame_chain(*s->sets[rq.set], rq, sl.stream);
  if (r == VRT_OK && cudaLaunchHostFunc(sl.stream, on_frame_done, &sl) != cudaSuccess)
    r = VRT_ERR_CUDA;
  return r;
}

// Issue the frames of `sl.reqs` (distinct resident sets) as one CUDA graph on
// slot `sl`: capture on the slot's stream, fork one branch stream per frame,
// run each frame's chain on its branch, join them back, launch the graph once
// (scheduler thread, lock released). On failure nothing has reached the device
// (the capture is discarded); *captured says whether the grids' host state
// already moved on (their sets must then be uploaded again).
vrt_status issue_batch(vrt_server s, Slot& sl, bool* captured) {
  const size_t k = sl.reqs.size();
  *captured = false;
  // buffers the frames size lazily, before the capture (no allocation inside)
  for (Request& rq : sl.reqs) {
    ServerSet& st = *s->sets[rq.set];
    vrt_status r = vrt_set_stream(st.grid, sl.stream);
    if (r == VRT_OK) r = vrt::prepare_frame(st.grid, &rq.cam, &rq.p);
    if (r != VRT_OK) return r;
  }
  while (sl.branch.size() < k) {
    cudaStream_t b = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) return VRT_ERR_CUDA;
    sl.branch.push_back(b);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return VRT_ERR_CUDA;
    sl.join.push_back(e);
  }
  if (!sl.fork && cudaEventCreateWithFlags(&sl.fork, cudaEventDisableTiming) != cudaSuccess)
    return VRT_ERR_CUDA;
  if (cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return VRT_ERR_CUDA;
  *captured = true;
  vrt_status r = cudaEventRecord(sl.fork, sl.stream) == cudaSuccess ? VRT_OK : VRT_ERR_CUDA;
  for (size_t i = 0; i < k && r == VRT_OK; ++i) {
    if (cudaStreamWaitEvent(sl.branch[i], sl.fork, 0) != cudaSuccess) { r = VRT_ERR_CUDA; break; }
    r = frame_chain(*s->sets[sl.reqs[i].set], sl.reqs[i], sl.branch[i]);
    if (r == VRT_OK && (cudaEventRecord(sl.join[i], sl.branch[i]) != cudaSuccess ||
                        cudaStreamWaitEvent(sl.stream, sl.join[i], 0) != cudaSuccess))
      r = VRT_ERR_CUDA;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(sl.stream, &graph);
  // later calls on these grids (vrt_sync when the batch retires) use the slot's stream
  for (Request& rq : sl.reqs) vrt_set_stream(s->sets[rq.set]->grid, sl.stream);
  if (r == VRT_OK && ec != cudaSuccess) r = VRT_ERR_CUDA;
  cudaGraphExec_t exec = nullptr;
  if (r == VRT_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) r = VRT_ERR_CUDA;
  if (graph) cudaGraphDestroy(graph);
  if (r == VRT_OK && cudaGraphLaunch(exec, sl.stream) != cudaSuccess) r = VRT_ERR_CUDA;
  if (exec) cudaGraphExecDestroy(exec);  // the launched graph still runs to its end
  if (r != VRT_OK) {
    cudaGetLastError();
    return r;
  }
  *captured = false;  // it ran: the grids' state is that of the frames
  if (cudaLaunchHostFunc(sl.stream, on_frame_done, &sl) != cudaSuccess) return VRT_ERR_CUDA;
  return VRT_OK;
}

void finish(vrt_server s, const Request& rq, int32_t status, Clock::time_point t_done) {  // lock held
  vrt_server_result res;
  res.request_id = rq.id;
  res.set_id = rq.set;
  res.status = status;
  res.latency_ms = ms_between(rq.t_submit, t_done);
  res.queue_ms = ms_between(rq.t_submit, rq.t_issue);
  s->results.push_back(res);
  if (rq.upd) s->pinned_free.emplace(rq.upd_cap, rq.upd);
  ++s->completed;
  s->cv_done.notify_all();
}

// Evict set k's grid (its host copy stays): used when a batch capture failed
// after the grid's host-side state had moved on. Lock held, released around
// the CUDA calls.
void drop_grid(vrt_server s, std::unique_lock<std::mutex>& lk, int k) {
  ServerSet& v = *s->sets[k];
  if (!v.grid) return;
  vrt_grid vg = v.grid;
  v.grid = nullptr;
  s->resident_bytes -= v.bytes;
  --s->resident_sets;
  lk.unlock();
  vrt_destroy(vg);
  lk.lock();
}

// Issue a batch of small-set frames on `sl` if at least two are ready: the
// oldest pending request of each idle, unblocked set with fewer than
// small_segments segments, up to max_batch, each made resident. Returns false
// (having issued nothing) when fewer than two qualify. Lock held; released
// around the CUDA calls.
bool issue_small_batch(vrt_server s, std::unique_lock<std::mutex>& lk, Slot& sl,
                       std::vector<char>& blocked) {
  std::vector<char> seen(s->sets.size(), 0);
  std::vector<size_t> pick;
  for (size_t i = 0; i < s->pending.size() && (int)pick.size() < s->max_batch; ++i) {
    const int k = s->pending[i].set;
    if (seen[k]) continue;
    seen[k] = 1;
    const ServerSet& st = *s->sets[k];
    if (st.busy || blocked[k] || st.V - st.P >= s->small_segments) continue;
    pick.push_back(i);
  }
  if (pick.size() < 2) return false;
  // take them out of the queue (highest index first keeps the others valid)
  std::vector<Request> reqs;
  for (size_t j = pick.size(); j-- > 0;) {
    reqs.push_back(s->pending[pick[j]]);
    s->pending.erase(s->pending.begin() + (long)pick[j]);
  }
  std::reverse(reqs.begin(), reqs.end());
  sl.busy = true;
  sl.done.store(false);
  sl.reqs.clear();
  for (Request& rq : reqs) {
    ServerSet& st = *s->sets[rq.set];
    st.busy = true;
    st.last_use = ++s->tick;
    vrt_status r = VRT_OK;
    const bool ok = make_resident(s, lk, rq.set, &r);
    if (ok) {
      sl.reqs.push_back(rq);
    } else if (r == VRT_OK) {  // no room yet: back to the queue's front, try later
      st.busy = false;
      s->pending.push_front(rq);
      blocked[rq.set] = 1;
    } else {
      st.busy = false;
      rq.t_issue = Clock::now();
      finish(s, rq, r, Clock::now());
    }
  }
  if (sl.reqs.empty()) {
    sl.busy = false;
    return true;  // the picks were handled (queued again or failed)
  }
  const Clock::time_point t_issue = Clock::now();
  for (Request& rq : sl.reqs) rq.t_issue = t_issue;
  lk.unlock();
  bool captured = false;
  vrt_status r = sl.reqs.size() >= 2 ? issue_batch(s, sl, &captured) : issue(s, sl, sl.reqs[0]);
  if (r != VRT_OK) cudaStreamSynchronize(sl.stream);
  lk.lock();
  if (r == VRT_OK) {
    if (sl.reqs.size() >= 2) {
      ++s->batches;
      s->batched_frames += sl.reqs.size();
    }
    return true;
  }
  for (Request& rq : sl.reqs) {  // nothing of the failed batch reached the device
    if (captured) drop_grid(s, lk, rq.set);
    else if (s->sets[rq.set]->grid) {
      lk.unlock();
      vrt_sync(s->sets[rq.set]->grid);
      lk.lock();
    }
    s->sets[rq.set]->busy = false;
    finish(s, rq, r, Clock::now());
  }
  sl.reqs.clear();
  sl.busy = false;
  return true;
}

void scheduler(vrt_server s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // (1) retire finished frames (a slot holds one frame or a batch)
    for (auto& slp : s->slots) {
      Slot& sl = *slp;
      if (!sl.busy || !sl.done.load()) continue;
      for (Request& rq : sl.reqs) {
        ServerSet& st = *s->sets[rq.set];
        lk.unlock();
        const vrt_status status = vrt_sync(st.grid);  // the frame's device status
        uint64_t b = 0;
        vrt_grid_device_bytes(st.grid, &b);
        lk.lock();
        s->resident_bytes += b - st.bytes;  // lazily sized buffers may have grown
        st.bytes = b;
        st.busy = false;
        finish(s, rq, status, sl.t_done);
      }
      sl.reqs.clear();
      sl.busy = false;
      sl.done.store(false);
    }
    trim(s, lk);
    // (2) issue: the oldest queued request of each idle set, while slots are free
    bool issued = false;
    std::vector<char> blocked(s->sets.size(), 0);  // no room for the set this round
    for (;;) {
      Slot* free_slot = nullptr;
      for (auto& slp : s->slots)
        if (!slp->busy) { free_slot = slp.get(); break; }
      if (!free_slot) break;
      if (s->small_segments > 0 && issue_small_batch(s, lk, *free_slot, blocked)) {
        issued = true;
        continue;
      }
      // the first request that is the oldest of its set, whose set is idle and not blocked
      std::vector<char> seen(s->sets.size(), 0);
      size_t pick = s->pending.size();
      for (size_t i = 0; i < s->pending.size(); ++i) {
        const int k = s->pending[i].set;
        if (seen[k]) continue;
        seen[k] = 1;
        if (!s->sets[k]->busy && !blocked[k]) { pick = i; break; }
      }
      if (pick == s->pending.size()) break;
      Request rq = s->pending[pick];
      s->pending.erase(s->pending.begin() + (long)pick);
      ServerSet& st = *s->sets[rq.set];
      st.busy = true;
      st.last_use = ++s->tick;
      free_slot->busy = true;
      free_slot->done.store(false);
      vrt_status r = VRT_OK;
      const bool ok = make_resident(s, lk, rq.set, &r);
      if (!ok && r == VRT_OK) {  // no room yet: back in place, try again later
        st.busy = false;
        free_slot->busy = false;
        s->pending.insert(s->pending.begin() + (long)pick, rq);
        blocked[rq.set] = 1;
        continue;
      }
      if (ok) {
        rq.t_issue = Clock::now();
        free_slot->reqs.assign(1, rq);
        lk.unlock();
        r = issue(s, *free_slot, free_slot->reqs[0]);
        lk.lock();
        if (r != VRT_OK) free_slot->reqs.clear();
      }
      if (r != VRT_OK) {
        // Part of the frame may already be on the slot's stream (the update
        // copy from rq.upd, voxelization, ...): wait for it before the pinned
        // buffer returns to the pool and the set can run on another slot.
        if (ok) {
          lk.unlock();
          cudaStreamSynchronize(free_slot->stream);
          vrt_sync(st.grid);  // drop a device status the partial frame may have left
          lk.lock();
        }
        st.busy = false;
        free_slot->busy = false;
        rq.t_issue = Clock::now();
        finish(s, rq, r, Clock::now());
      }
      issued = true;
    }
    bool inflight = false;
    for (auto& slp : s->slots) inflight = inflight || slp->busy;
    if (s->stop && s->pending.empty() && !inflight) break;
    if (!issued) s->cv.wait_for(lk, std::chrono::milliseconds(2));
  }
}

}  // namespace

extern "C" {

vrt_status vrt_server_create(const vrt_server_desc* desc, vrt_server* out) {
  if (!out || !desc) return sfail(nullptr, VRT_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (desc->max_inflight < 0) return sfail(nullptr, VRT_ERR_INVALID_ARG, "max_inflight must be >= 0");
  if (desc->max_batch < 0) return sfail(nullptr, VRT_ERR_INVALID_ARG, "max_batch must be >= 0");
  vrt_server s = new (std::nothrow) vrt_server_s();
  if (!s) return sfail(nullptr, VRT_ERR_OOM, "host allocation failed");
  s->device = desc->device;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(s->device) != cudaSuccess) {
    delete s;
    return sfail(nullptr, VRT_ERR_INVALID_ARG, "bad device");
  }
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  s->budget = desc->hbm_budget ? desc->hbm_budget : (uint64_t)(0.8 * (double)fr);
  s->small_segments = desc->small_segments;
  s->max_batch = desc->max_batch == 0 ? 16 : std::min(64, std::max(2, desc->max_batch));
  const int slots = desc->max_inflight ? desc->max_inflight : 4;
  for (int i = 0; i < slots; ++i) {
    auto sl = std::make_unique<Slot>();
    sl->server = s;
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& o : s->slots) cudaStreamDestroy(o->stream);
      delete s;
      cudaSetDevice(prev);
      return sfail(nullptr, VRT_ERR_CUDA, "cudaStreamCreate failed");
    }
    s->slots.push_back(std::move(sl));
  }
  cudaSetDevice(prev);
  s->th = std::thread(scheduler, s);
  *out = s;
  return VRT_OK;
}

vrt_status vrt_server_add_set(vrt_server s, const vrt_grid_desc* grid, const float* xyz,
                              int32_t stride, int64_t n_vertices, const int64_t* offsets,
                              int64_t n_polylines, int32_t* set_id) {
  if (!s || !grid || !offsets || !set_id || (n_vertices > 0 && !xyz))
    return sfail(s, VRT_ERR_INVALID_ARG, "NULL argument");
  if (stride != 3 && stride != 4) return sfail(s, VRT_ERR_INVALID_ARG, "stride must be 3 or 4");
  if (n_vertices < 0 || n_polylines < 0 || offsets[0] != 0 || offsets[n_polylines] != n_vertices)
    return sfail(s, VRT_ERR_INVALID_ARG, "offsets must start at 0 and end at n_vertices");
  auto st = std::make_unique<ServerSet>();
  st->desc = *grid;
  st->V = n_vertices;
  st->P = n_polylines;
  st->offsets.assign(offsets, offsets + n_polylines + 1);
  st->xyz.resize(3 * (size_t)n_vertices);
  for (int64_t i = 0; i < n_vertices; ++i)
    for (int k = 0; k < 3; ++k) {
      const float x = xyz[i * stride + k];
      if (!(x >= -256.0f && x < 768.0f))
        return sfail(s, VRT_ERR_INVALID_ARG, "coordinates must be finite and in [-256, 768)");
      st->xyz[3 * i + k] = x;
    }
  std::lock_guard<std::mutex> lk(s->mu);
  st->bytes = 0;
  s->sets.push_back(std::move(st));
  *set_id = (int32_t)s->sets.size() - 1;
  return VRT_OK;
}

vrt_status vrt_server_submit(vrt_server s, int32_t set_id, int64_t first_vertex,
                             int64_t n_vertices, const float* xyz, int32_t stride,
                             const vrt_camera* cam, const vrt_render_params* p, float* rgba_out,
                             int32_t* first_id_out, float* first_t_out, int64_t* request_id) {
  const Clock::time_point t0 = Clock::now();
  if (!s || !cam || !p || !rgba_out || !request_id) return sfail(s, VRT_ERR_INVALID_ARG, "NULL argument");
  if (stride != 3 && stride != 4) return sfail(s, VRT_ERR_INVALID_ARG, "stride must be 3 or 4");
  // the checks vrt_cull and vrt_trace make, so that a bad request fails here
  // and never reaches a stream
  if (const char* why = vrt::frame_args_error(cam, p)) return sfail(s, VRT_ERR_INVALID_ARG, why);
  Request rq;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return sfail(s, VRT_ERR_STATE, "server is shutting down");
    if (set_id < 0 || set_id >= (int32_t)s->sets.size())
      return sfail(s, VRT_ERR_INVALID_ARG, "unknown set");
    const ServerSet& st = *s->sets[set_id];
    if (first_vertex < 0 || n_vertices < 0 || first_vertex + n_vertices > st.V || (n_vertices > 0 && !xyz))
      return sfail(s, VRT_ERR_INVALID_ARG, "vertex range outside the set");
    if (n_vertices > 0) {  // a pooled pinned buffer large enough, if any
      auto it = s->pinned_free.lower_bound(3 * (size_t)n_vertices);
      if (it != s->pinned_free.end()) {
        rq.upd_cap = it->first;
        rq.upd = it->second;
        s->pinned_free.erase(it);
      }
    }
  }
  if (n_vertices > 0) {
    if (!rq.upd) {
      rq.upd_cap = 3 * (size_t)n_vertices;
      int prev = 0;
      cudaGetDevice(&prev);
      cudaSetDevice(s->device);
      void* h = nullptr;
      const cudaError_t e = cudaMallocHost(&h, rq.upd_cap * sizeof(float));
      cudaSetDevice(prev);
      if (e != cudaSuccess) return sfail(s, VRT_ERR_OOM, "cudaMallocHost failed");
      rq.upd = (float*)h;
      std::lock_guard<std::mutex> lk(s->mu);
      s->pinned_all.push_back(rq.upd);
    }
    for (int64_t i = 0; i < n_vertices; ++i)
      for (int k = 0; k < 3; ++k) rq.upd[3 * i + k] = xyz[i * stride + k];
  }
  rq.set = set_id;
  rq.first = first_vertex;
  rq.n = n_vertices;
  rq.cam = *cam;
  rq.p = *p;
  rq.rgba = rgba_out;
  rq.first_id = first_id_out;
  rq.first_t = first_t_out;
  rq.t_submit = t0;
  std::lock_guard<std::mutex> lk(s->mu);
  rq.id = s->next_id++;
  *request_id = rq.id;
  s->pending.push_back(rq);
  ++s->submitted;
  s->cv.notify_all();
  return VRT_OK;
}

vrt_status vrt_server_poll(vrt_server s, vrt_server_result* out, int32_t cap, int32_t* n_out,
                           int32_t wait) {
  if (!s || !n_out || (cap > 0 && !out)) return sfail(s, VRT_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (wait) s->cv_done.wait(lk, [&] { return s->completed == s->submitted; });
  int32_t n = 0;
  while (n < cap && !s->results.empty()) {
    out[n++] = s->results.front();
    s->results.pop_front();
  }
  *n_out = n;
  return VRT_OK;
}

vrt_status vrt_server_get_stats(vrt_server s, vrt_server_stats* out) {
  if (!s || !out) return sfail(s, VRT_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->hbm_budget = s->budget;
  out->resident_bytes = s->resident_bytes;
  out->completed = s->completed;
  out->evictions = s->evictions;
  out->pending = (int32_t)s->pending.size();
  int inflight = 0;
  for (auto& sl : s->slots) inflight += sl->busy ? 1 : 0;
  out->inflight = inflight;
  out->resident_sets = s->resident_sets;
  out->batches = s->batches;
  out->batched_frames = s->batched_frames;
  return VRT_OK;
}

vrt_status vrt_server_destroy(vrt_server s) {
  if (!s) return sfail(nullptr, VRT_ERR_INVALID_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto& st : s->sets)
    if (st->grid) vrt_destroy(st->grid);
  for (auto& sl : s->slots) {
    cudaStreamDestroy(sl->stream);
    for (cudaStream_t b : sl->branch) cudaStreamDestroy(b);
    for (cudaEvent_t e : sl->join) cudaEventDestroy(e);
    if (sl->fork) cudaEventDestroy(sl->fork);
  }
  for (float* p : s->pinned_all) cudaFreeHost(p);
  cudaSetDevice(prev);
  delete s;
  return VRT_OK;
}

}  // extern "C"
