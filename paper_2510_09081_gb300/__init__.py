"""GB300 (sm_103a) voxel ray tracing of dynamic line sets.

Python binding of ``libvrt.so`` (C ABI: ``include/vrt.h``), after Kraaijeveld et
al., "Real-Time Rendering of Dynamic Line Sets using Voxel Ray Tracing" (arXiv
2510.09081). The functions carry the names of the C entry points and only
marshal arguments: every step of a frame (ingest, voxelization, mips, culling,
scan, list scatter, ray tracing) runs in the library's CUDA kernels. Device
buffers are torch CUDA tensors; there is no CPU fallback -- without the built
library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvrt.so")
_lib = None

OK, ERR_INVALID_ARG, ERR_OOM, ERR_OVERFLOW, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_BOUNDS = range(8)
STATUS_NAMES = ["OK", "INVALID_ARG", "OOM", "OVERFLOW", "CUDA", "TIMEOUT", "STATE", "BOUNDS"]
OPT_FORCE_EXACT = 1
OPT_STAGE_TIMING = 2
OPT_TRACE_COUNTERS = 3
OPT_MIPS_FORMAT = 4
OPT_GRAPH = 5
OPT_CULL_DEPTH = 6
OPT_TEST_SCAN_STALL = 7
OPT_TRACE_SHORT_LIST = 8
OPT_TRACE_RAY_KEYS = 9
OPT_HIT_KEY = 10
OPT_TRACE_TILE = 11
HIT_KEY_DEPTH_ID, HIT_KEY_16_16 = 0, 1
NOALLOC_GAVE_UP, NOALLOC_WRAPPED = 1, 2   # status bits of scan_counts_noalloc
MIPS_F32, MIPS_F16, MIPS_BF16 = 0, 1, 2
STAGES = ["ingest", "pass1", "mips", "cull", "scan", "pass2", "trace", "repair", "shade"]

# Exported symbols of the C ABI (include/vrt.h)
SYMBOLS = ["vrt_create_grid", "vrt_upload_segments", "vrt_update_vertices", "vrt_voxelize",
           "vrt_build_mips", "vrt_cull", "vrt_trace", "vrt_sync", "vrt_get_stats",
           "vrt_read_grid", "vrt_read_lists", "vrt_read_mips", "vrt_read_shading", "vrt_set_option",
           "vrt_get_stage_ms", "vrt_scan_counts_noalloc", "vrt_last_error", "vrt_destroy",
           "vrt_grid_device_bytes", "vrt_set_stream", "vrt_server_create", "vrt_server_add_set",
           "vrt_server_submit", "vrt_server_poll", "vrt_server_get_stats", "vrt_server_destroy",
           "vrt_frame", "vrt_tune_grid_side", "vrt_tune_shapes"]


class VrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("radius", ctypes.c_float), ("r_min", ctypes.c_float),
                ("occ_scale", ctypes.c_int32), ("max_fragments", ctypes.c_uint64)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_inflight", ctypes.c_int32),
                ("device", ctypes.c_int32), ("small_segments", ctypes.c_int32),
                ("max_batch", ctypes.c_int32)]


class ServerResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("set_id", ctypes.c_int32),
                ("status", ctypes.c_int32), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("resident_sets", ctypes.c_int32),
                ("evictions", ctypes.c_int32), ("pending", ctypes.c_int32),
                ("inflight", ctypes.c_int32), ("batches", ctypes.c_uint64),
                ("batched_frames", ctypes.c_uint64)]


class CameraC(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("ortho", ctypes.c_int32),
                ("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fovy_deg", ctypes.c_float),
                ("ortho_h", ctypes.c_float)]


class RenderParamsC(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("ao_cones", ctypes.c_int32), ("cull", ctypes.c_int32),
                ("k", ctypes.c_int32), ("voxel_shading", ctypes.c_int32), ("light", ctypes.c_float * 3)]


class StatsC(ctypes.Structure):
    _fields_ = [("fragments", ctypes.c_uint64), ("fragments_listed", ctypes.c_uint64),
                ("sum_occupancy", ctypes.c_uint64), ("exact_decisions", ctypes.c_uint64),
                ("occupied_voxels", ctypes.c_uint32), ("visible_voxels", ctypes.c_uint32),
                ("repaired_voxels", ctypes.c_uint32), ("repair_rounds", ctypes.c_uint32),
                ("max_count", ctypes.c_uint32), ("status_bits", ctypes.c_uint32),
                ("kernel_launches", ctypes.c_uint64), ("retraced_pixels", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("trace_entries", ctypes.c_uint64),
                ("trace_capsule_tests", ctypes.c_uint64), ("trace_voxels", ctypes.c_uint64),
                ("trace_steps", ctypes.c_uint64), ("trace_wholewarp_voxels", ctypes.c_uint64),
                ("trace_wholewarp_entries", ctypes.c_uint64), ("trace_hits", ctypes.c_uint64),
                ("trace_cycles", ctypes.c_uint64 * 4), ("trace_unique_entries", ctypes.c_uint64),
                ("trace_unique_vertices", ctypes.c_uint64), ("trace_unique_voxels", ctypes.c_uint64)]


def load():
    """Load libvrt.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise VrtError(ERR_STATE, f"{LIB_PATH} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "vrt_create_grid": [ctypes.POINTER(GridDesc), P, ctypes.POINTER(P)],
        "vrt_upload_segments": [P, P, i32, i64, P, i64, i32],
        "vrt_update_vertices": [P, i64, i64, P, i32, i32],
        "vrt_voxelize": [P],
        "vrt_build_mips": [P],
        "vrt_cull": [P, ctypes.POINTER(CameraC), ctypes.POINTER(RenderParamsC)],
        "vrt_trace": [P, ctypes.POINTER(CameraC), ctypes.POINTER(RenderParamsC), P, P, P],
        "vrt_sync": [P],
        "vrt_get_stats": [P, ctypes.POINTER(StatsC)],
        "vrt_read_grid": [P, P],
        "vrt_read_lists": [P, P, P, P, u64, ctypes.POINTER(u64)],
        "vrt_read_mips": [P, P, u64],
        "vrt_read_shading": [P, P, P],
        "vrt_set_option": [P, i32, i64],
        "vrt_get_stage_ms": [P, P, i32],
        "vrt_scan_counts_noalloc": [P, P, P, u64, P, P, P],
        "vrt_destroy": [P],
        "vrt_grid_device_bytes": [P, ctypes.POINTER(u64)],
        "vrt_frame": [P, i64, i64, P, i32, i32, ctypes.POINTER(CameraC),
                      ctypes.POINTER(RenderParamsC), P, P, P],
        "vrt_tune_grid_side": [ctypes.POINTER(GridDesc), P, i32, i64, P, i64,
                               ctypes.POINTER(CameraC), ctypes.POINTER(RenderParamsC), P, i32, i32,
                               ctypes.POINTER(i32), P],
        "vrt_tune_shapes": [ctypes.POINTER(GridDesc), P, i32, i64, P, i64,
                            ctypes.POINTER(CameraC), ctypes.POINTER(RenderParamsC), P, i32, P, i32,
                            i32, ctypes.POINTER(i32), ctypes.POINTER(i32), P],
        "vrt_set_stream": [P, P],
        "vrt_server_create": [ctypes.POINTER(ServerDesc), ctypes.POINTER(P)],
        "vrt_server_add_set": [P, ctypes.POINTER(GridDesc), P, i32, i64, P, i64,
                               ctypes.POINTER(i32)],
        "vrt_server_submit": [P, i32, i64, i64, P, i32, ctypes.POINTER(CameraC),
                              ctypes.POINTER(RenderParamsC), P, P, P, ctypes.POINTER(i64)],
        "vrt_server_poll": [P, ctypes.POINTER(ServerResult), i32, ctypes.POINTER(i32), i32],
        "vrt_server_get_stats": [P, ctypes.POINTER(ServerStats)],
        "vrt_server_destroy": [P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.vrt_last_error.argtypes = [P]
    lib.vrt_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status, g=None):
    if status != OK:
        msg = load().vrt_last_error(g)
        raise VrtError(status, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ptr(x):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _is_device(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def camera_c(cam) -> CameraC:
    c = CameraC()
    c.width, c.height, c.ortho = int(cam.width), int(cam.height), int(cam.ortho)
    c.eye[:] = [float(v) for v in cam.eye]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.fovy_deg = float(getattr(cam, "fovy_deg", 45.0))
    c.ortho_h = float(getattr(cam, "ortho_h", 0.0))
    return c


def params_c(alpha=1.0, ao_cones=0, cull=0, k=0, voxel_shading=0, light=(0.0, 0.0, 1.0)) -> RenderParamsC:
    p = RenderParamsC(alpha=float(alpha), ao_cones=int(ao_cones), cull=int(cull), k=int(k),
                      voxel_shading=int(voxel_shading))
    p.light[:] = [float(v) for v in light]
    return p


# ------------------------------------------------------------ C entry points
def create_grid(n, radius, r_min=0.5, occ_scale=32, max_fragments=0, stream=None):
    lib = load()
    d = GridDesc(n=int(n), radius=float(radius), r_min=float(r_min), occ_scale=int(occ_scale),
                 max_fragments=int(max_fragments))
    h = ctypes.c_void_p()
    _check(lib.vrt_create_grid(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)))
    return h


def upload_segments(g, xyz, offsets):
    """xyz: float32 [V, 3|4] numpy array (host) or torch CUDA tensor (device);
    offsets: int64 [P + 1] (host)."""
    off = np.ascontiguousarray(np.asarray(offsets), dtype=np.int64)
    dev = _is_device(xyz)
    if not dev:
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    else:
        assert xyz.is_contiguous() and str(xyz.dtype) == "torch.float32"
    V = int(xyz.shape[0])
    stride = int(xyz.shape[1]) if V else 3
    _check(load().vrt_upload_segments(g, _ptr(xyz), stride, V, off.ctypes.data, off.shape[0] - 1,
                                      int(dev)), g)


def update_vertices(g, first_vertex, xyz):
    dev = _is_device(xyz)
    if not dev:
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    V = int(xyz.shape[0])
    stride = int(xyz.shape[1]) if V else 3
    _check(load().vrt_update_vertices(g, int(first_vertex), V, _ptr(xyz), stride, int(dev)), g)


def voxelize(g):
    _check(load().vrt_voxelize(g), g)


def build_mips(g):
    _check(load().vrt_build_mips(g), g)


def cull(g, cam, params):
    c = cam if isinstance(cam, CameraC) else camera_c(cam)
    _check(load().vrt_cull(g, ctypes.byref(c), ctypes.byref(params)), g)


def trace(g, cam, params, rgba, first_id=None, first_t=None):
    """rgba: torch float32 CUDA tensor [H, W, 4]; first_id int32 [H, W];
    first_t float32 [H, W] (both optional)."""
    c = cam if isinstance(cam, CameraC) else camera_c(cam)
    _check(load().vrt_trace(g, ctypes.byref(c), ctypes.byref(params), _ptr(rgba), _ptr(first_id),
                            _ptr(first_t)), g)


def sync(g):
    _check(load().vrt_sync(g), g)


def get_stats(g) -> dict:
    s = StatsC()
    _check(load().vrt_get_stats(g, ctypes.byref(s)), g)
    out = {}
    for k, _ in StatsC._fields_:
        v = getattr(s, k)
        out[k] = [int(x) for x in v] if k == "trace_cycles" else int(v)
    return out


def read_grid(g, n):
    out = np.zeros(n ** 3, np.uint32)
    _check(load().vrt_read_grid(g, out.ctypes.data), g)
    return out


def read_lists(g, n, cap=None):
    start = np.zeros(n ** 3, np.uint32)
    ln = np.zeros(n ** 3, np.uint32)
    tot = ctypes.c_uint64(0)
    _check(load().vrt_read_lists(g, start.ctypes.data, ln.ctypes.data, None, 0, ctypes.byref(tot)), g)
    ids = np.zeros(max(int(tot.value), 1), np.uint32)
    _check(load().vrt_read_lists(g, start.ctypes.data, ln.ctypes.data, ids.ctypes.data,
                                 ids.shape[0], ctypes.byref(tot)), g)
    return start, ln, ids[:int(tot.value)]


def read_shading(g, n):
    """The voxel-space shading field of the last shaded trace, [z, y, x], and
    the mask of voxels it computed."""
    vals = np.zeros((n, n, n), np.float32)
    valid = np.zeros((n, n, n), np.uint8)
    _check(load().vrt_read_shading(g, vals.ctypes.data, valid.ctypes.data), g)
    return vals, valid.astype(bool)


def read_mips(g, n):
    sizes, m = [], n
    while m >= 1:
        sizes.append(m)
        m //= 2
    tot = sum(s ** 3 for s in sizes)
    out = np.zeros(tot, np.float32)
    _check(load().vrt_read_mips(g, out.ctypes.data, tot), g)
    levels, o = [], 0
    for s in sizes:
        levels.append(out[o:o + s ** 3].reshape(s, s, s))
        o += s ** 3
    return levels


def set_option(g, option, value):
    _check(load().vrt_set_option(g, int(option), int(value)), g)


def get_stage_ms(g) -> dict:
    ms = np.zeros(len(STAGES), np.float32)
    _check(load().vrt_get_stage_ms(g, ms.ctypes.data, len(STAGES)), g)
    return {k: float(v) for k, v in zip(STAGES, ms) if v >= 0}


def scan_counts_noalloc(words, offsets, marks=None, total=None, status=None, stream=None,
                        n_voxels=None):
    """Exclusive scan of packed-word counts without any device allocation
    (vrt_scan_counts_noalloc). All arguments are torch CUDA tensors."""
    n = int(words.numel()) if n_voxels is None else int(n_voxels)
    # the C call cannot see the tensors' sizes: n must fit every buffer it touches
    if n > words.numel() or n > offsets.numel():
        raise VrtError(ERR_INVALID_ARG, f"n_voxels {n} exceeds words ({words.numel()}) "
                                        f"or offsets ({offsets.numel()})")
    if marks is not None and marks.numel() * 32 < n:
        raise VrtError(ERR_INVALID_ARG, f"marks hold {marks.numel() * 32} bits, n_voxels is {n}")
    for name, t in (("words", words), ("offsets", offsets), ("marks", marks), ("total", total),
                    ("status", status)):
        if t is not None and (t.element_size() != 4 or not t.is_contiguous() or not t.is_cuda):
            raise VrtError(ERR_INVALID_ARG, f"{name} must be a contiguous 32-bit CUDA tensor")
    _check(load().vrt_scan_counts_noalloc(_ptr(words), _ptr(marks), _ptr(offsets), n,
                                          _ptr(total), _ptr(status), _stream_ptr(stream)))


def destroy(g):
    if g:
        _check(load().vrt_destroy(g))


# --------------------------------------------------------------- convenience
class Renderer:
    """One line set on one grid, with torch output buffers; ``frame`` runs
    voxelize -> (mips) -> cull -> trace on the device."""

    def __init__(self, n, radius, r_min=0.5, occ_scale=32, max_fragments=0, stream=None):
        self.n = int(n)
        self.h = create_grid(n, radius, r_min, occ_scale, max_fragments, stream)
        self._bufs = None

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, xyz, offsets):
        upload_segments(self.h, xyz, offsets)

    def update(self, first_vertex, xyz):
        update_vertices(self.h, first_vertex, xyz)

    def buffers(self, width, height):
        import torch
        if self._bufs is None or self._bufs[0].shape[:2] != (height, width):
            self._bufs = (torch.empty((height, width, 4), dtype=torch.float32, device="cuda"),
                          torch.empty((height, width), dtype=torch.int32, device="cuda"),
                          torch.empty((height, width), dtype=torch.float32, device="cuda"))
        return self._bufs

    def frame(self, cam, alpha=1.0, ao_cones=0, cull_on=0, k=0, voxelize_first=True,
              voxel_shading=0, light=(0.0, 0.0, 1.0)):
        p = params_c(alpha, ao_cones, cull_on, k, voxel_shading, light)
        c = camera_c(cam)
        rgba, fid, ft = self.buffers(c.width, c.height)
        if voxelize_first:
            voxelize(self.h)
            if ao_cones or voxel_shading:
                build_mips(self.h)
        cull(self.h, c, p)
        trace(self.h, c, p, rgba, fid, ft)
        return rgba, fid, ft

    def trace_only(self, cam, alpha=1.0, ao_cones=0, k=0, voxel_shading=0, light=(0.0, 0.0, 1.0)):
        """A frame of a static scene: trace with the lists (and voxel-space
        field) of the last build."""
        p = params_c(alpha, ao_cones, 0, k, voxel_shading, light)
        c = camera_c(cam)
        rgba, fid, ft = self.buffers(c.width, c.height)
        trace(self.h, c, p, rgba, fid, ft)
        return rgba, fid, ft


def grid_device_bytes(g) -> int:
    out = ctypes.c_uint64(0)
    _check(load().vrt_grid_device_bytes(g, ctypes.byref(out)), g)
    return int(out.value)


# ------------------------------------------------------------------- serving
class Server:
    """The library's request loop over resident line sets (vrt.h, "serving"):
    ``submit`` queues a frame of a registered set and returns at once; ``poll``
    returns finished requests with their status and latency."""

    def __init__(self, hbm_budget=0, max_inflight=4, device=0, small_segments=0, max_batch=0):
        desc = ServerDesc(hbm_budget=int(hbm_budget), max_inflight=int(max_inflight),
                          device=int(device), small_segments=int(small_segments),
                          max_batch=int(max_batch))
        h = ctypes.c_void_p()
        _check(load().vrt_server_create(ctypes.byref(desc), ctypes.byref(h)))
        self.h = h

    def add_set(self, xyz, offsets, n, radius, r_min=0.5, occ_scale=32, max_fragments=0) -> int:
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        desc = GridDesc(n=int(n), radius=float(radius), r_min=float(r_min),
                        occ_scale=int(occ_scale), max_fragments=int(max_fragments))
        sid = ctypes.c_int32(0)
        _check(load().vrt_server_add_set(self.h, ctypes.byref(desc), _ptr(xyz), int(xyz.shape[1]),
                                         int(xyz.shape[0]), _ptr(offsets), int(offsets.shape[0] - 1),
                                         ctypes.byref(sid)))
        return int(sid.value)

    def submit(self, set_id, cam, rgba, alpha=1.0, ao_cones=0, cull_on=0, first_id=None,
               first_t=None, first_vertex=0, update=None, voxel_shading=0,
               light=(0.0, 0.0, 1.0), k=0) -> int:
        """rgba (and first_id / first_t) are device tensors that must stay alive
        until the request completes; update: host float32 [k, 3] for vertices
        first_vertex .. first_vertex + k - 1."""
        c = camera_c(cam)
        p = params_c(alpha, ao_cones, cull_on, k, voxel_shading, light)
        if update is None:
            upd, n_upd, stride = None, 0, 3
        else:
            upd = np.ascontiguousarray(update, dtype=np.float32)
            n_upd, stride = int(upd.shape[0]), int(upd.shape[1])
        rid = ctypes.c_int64(0)
        _check(load().vrt_server_submit(self.h, int(set_id), int(first_vertex), n_upd,
                                        _ptr(upd) if upd is not None else None, stride,
                                        ctypes.byref(c), ctypes.byref(p), _ptr(rgba),
                                        _ptr(first_id) if first_id is not None else None,
                                        _ptr(first_t) if first_t is not None else None,
                                        ctypes.byref(rid)))
        return int(rid.value)

    def poll(self, wait=False, cap=4096):
        buf = (ServerResult * cap)()
        n = ctypes.c_int32(0)
        out = []
        while True:
            _check(load().vrt_server_poll(self.h, buf, cap, ctypes.byref(n), int(bool(wait))))
            out += [dict(request_id=buf[i].request_id, set_id=buf[i].set_id, status=buf[i].status,
                         latency_ms=buf[i].latency_ms, queue_ms=buf[i].queue_ms)
                    for i in range(n.value)]
            if n.value < cap:
                return out
            wait = False

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().vrt_server_get_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            _check(load().vrt_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def frame(g, cam_c, params, rgba, first_id=None, first_t=None, first_vertex=0, update=None):
    """vrt_frame: update (optional) + voxelize + mips (AO or voxel shading) + cull + trace."""
    if update is None:
        upd, n, stride, dev = None, 0, 3, 0
    else:
        dev = _is_device(update)
        if hasattr(update, "data_ptr"):  # torch tensor (device, or pinned host memory: captured)
            if str(update.dtype) != "torch.float32" or not update.is_contiguous():
                raise ValueError("update must be a contiguous float32 tensor")
            upd = update
        else:
            upd = np.ascontiguousarray(update, dtype=np.float32)
        n, stride = int(upd.shape[0]), int(upd.shape[1])
    _check(load().vrt_frame(g, int(first_vertex), n, _ptr(upd) if upd is not None else None, stride,
                            int(dev), ctypes.byref(cam_c), ctypes.byref(params), _ptr(rgba),
                            _ptr(first_id) if first_id is not None else None,
                            _ptr(first_t) if first_t is not None else None), g)


def tune_grid_side(xyz, offsets, n, radius, cam, sides, alpha=1.0, ao_cones=0, cull_on=0, frames=3):
    """vrt_tune_grid_side: (best side, {side: mean ms})."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    desc = GridDesc(n=int(n), radius=float(radius), r_min=0.5, occ_scale=32, max_fragments=0)
    sides_a = np.ascontiguousarray(sides, dtype=np.int32)
    ms = np.zeros(sides_a.shape[0], np.float32)
    best = ctypes.c_int32(0)
    _check(load().vrt_tune_grid_side(ctypes.byref(desc), _ptr(xyz), int(xyz.shape[1]), int(xyz.shape[0]),
                                     _ptr(offsets), int(offsets.shape[0] - 1), ctypes.byref(camera_c(cam)),
                                     ctypes.byref(params_c(alpha, ao_cones, cull_on, 0)), _ptr(sides_a),
                                     int(sides_a.shape[0]), int(frames), ctypes.byref(best), _ptr(ms)))
    return int(best.value), {int(k): float(v) for k, v in zip(sides_a, ms)}


def tune_shapes(xyz, offsets, n, radius, cam, sides, tiles=(2, 4, 8, 16), alpha=1.0, ao_cones=0,
                cull_on=0, frames=3):
    """vrt_tune_shapes: ((best side, best tile width), {(side, tile): mean ms})."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    desc = GridDesc(n=int(n), radius=float(radius), r_min=0.5, occ_scale=32, max_fragments=0)
    sides_a = np.ascontiguousarray(sides, dtype=np.int32)
    tiles_a = np.ascontiguousarray(tiles, dtype=np.int32)
    ms = np.zeros(sides_a.shape[0] * tiles_a.shape[0], np.float32)
    bs, bt = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().vrt_tune_shapes(ctypes.byref(desc), _ptr(xyz), int(xyz.shape[1]), int(xyz.shape[0]),
                                  _ptr(offsets), int(offsets.shape[0] - 1), ctypes.byref(camera_c(cam)),
                                  ctypes.byref(params_c(alpha, ao_cones, cull_on, 0)), _ptr(sides_a),
                                  int(sides_a.shape[0]), _ptr(tiles_a), int(tiles_a.shape[0]),
                                  int(frames), ctypes.byref(bs), ctypes.byref(bt), _ptr(ms)))
    grid = {(int(a), int(b)): float(ms[i * tiles_a.shape[0] + j])
            for i, a in enumerate(sides_a) for j, b in enumerate(tiles_a)}
    return (int(bs.value), int(bt.value)), grid
