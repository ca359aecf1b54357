"""CPU oracle for the voxel ray-tracing hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. The product path (``paper_2510_09081_gb300``) never
does, and this package imports nothing from it.

The oracle is plain fp64 / exact-integer C++ (``oracle.cpp``) behind ctypes. See
that file's header for what each function restates from the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Parity bands for an fp32 implementation, in the units of the quantity they
# bound:
#   tie:   two depths closer than tie_abs + tie_rel * t may come out in either order
#   graze: |discriminant| / r^2 below graze_rel may flip hit <-> miss
#   pos:   hit points within pos_abs + pos_rel * t of a clip plane or the grid
#          boundary may be accepted or rejected
DEFAULT_BANDS = dict(tie_rel=2e-6, tie_abs=2e-5, graze_rel=1e-3, pos_abs=2e-5, pos_rel=4e-7)


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host C++ compiler (no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Cam(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("ortho", ctypes.c_int32),
                ("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fovy_deg", ctypes.c_float),
                ("ortho_h", ctypes.c_float)]


class _Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("ao_cones", ctypes.c_int32),
                ("tie_rel", ctypes.c_double), ("tie_abs", ctypes.c_double),
                ("graze_rel", ctypes.c_double), ("pos_abs", ctypes.c_double),
                ("pos_rel", ctypes.c_double), ("voxel_shading", ctypes.c_int32),
                ("light", ctypes.c_float * 3)]


def _prm(alpha, ao_cones, bands, voxel_shading, light):
    b = dict(DEFAULT_BANDS)
    if bands:
        b.update(bands)
    prm = _Params(alpha=float(alpha), ao_cones=int(ao_cones), voxel_shading=int(voxel_shading), **b)
    prm.light[:] = [float(v) for v in light]
    return prm


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    lib.or_create.restype = P
    lib.or_create.argtypes = [P, i32, i64, P, i64, i32, f32, f32, i32, i32, ctypes.POINTER(i32)]
    lib.or_destroy.argtypes = [P]
    lib.or_build_lists.restype = i64
    lib.or_build_lists.argtypes = [P]
    lib.or_ambiguous.restype = i64
    lib.or_ambiguous.argtypes = [P]
    lib.or_get_lists.argtypes = [P] * 7
    lib.or_get_vertices.argtypes = [P] * 6
    lib.or_build_mips.restype = i64
    lib.or_build_mips.argtypes = [P, P]
    lib.or_ao.restype = f64
    lib.or_ao.argtypes = [P, P]
    lib.or_voxel_shade.restype = f64
    lib.or_voxel_shade.argtypes = [P, i64, i64, i64, i32, P]
    lib.or_render.restype = i32
    lib.or_render.argtypes = [P, ctypes.POINTER(_Cam), ctypes.POINTER(_Params), i32, i64, i64,
                              P, P, P, P, P, P]
    lib.or_voxel_fragments.restype = i64
    lib.or_voxel_fragments.argtypes = [P, i64, i64, i64, P, i64, P]
    lib.or_render_pixels.restype = i32
    lib.or_render_pixels.argtypes = [P, ctypes.POINTER(_Cam), ctypes.POINTER(_Params), i32, P, i64,
                                     P, P, P, P, P, P]
    lib.or_seg_box_within.restype = i32
    lib.or_seg_box_within.argtypes = [P, P, P, i64, i64]
    lib.or_clipped_capsule_sdf.restype = f64
    lib.or_clipped_capsule_sdf.argtypes = [P, P, P, P, P, i32, i32, f64]
    lib.or_capsule_occupancy.restype = f64
    lib.or_capsule_occupancy.argtypes = [P, P, P, P, P, i32, i32, f64, f64]
    lib.or_line_capsule_entry.restype = f64
    lib.or_line_capsule_entry.argtypes = [P, P, P, P, f64]
    lib.or_camera_ray.argtypes = [ctypes.POINTER(_Cam), i32, i32, P, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cam(cam) -> _Cam:
    c = _Cam()
    c.width, c.height, c.ortho = int(cam.width), int(cam.height), int(cam.ortho)
    c.eye[:] = [float(x) for x in cam.eye]
    c.target[:] = [float(x) for x in cam.target]
    c.up[:] = [float(x) for x in cam.up]
    c.fovy_deg = float(cam.fovy_deg)
    c.ortho_h = float(cam.ortho_h)
    return c


class OracleError(RuntimeError):
    pass


class Oracle:
    """One line set on one grid. ``xyz`` float32 [V, 3] (or [V, 4]; the 4th
    component is ignored), ``offsets`` int64 [P + 1]."""

    def __init__(self, xyz, offsets, n, radius, r_min=0.5, occ_scale=32, nthreads=None):
        lib = _load()
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        stride = self.xyz.shape[1] if self.xyz.ndim == 2 else 3
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n = int(n)
        self.V = int(self.xyz.shape[0])
        self.P = int(self.offsets.shape[0] - 1)
        self.nthreads = int(nthreads or os.cpu_count() or 1)
        st = ctypes.c_int32(0)
        self._h = lib.or_create(_ptr(self.xyz), stride, self.V, _ptr(self.offsets), self.P,
                                self.n, float(radius), float(r_min), int(occ_scale),
                                self.nthreads, ctypes.byref(st))
        self.status = int(st.value)
        self._F = None
        if self.status != 0:
            lib.or_destroy(self._h)
            self._h = None
            raise OracleError(f"oracle rejected the input (status {self.status})")

    @classmethod
    def from_lineset(cls, ls, **kw):
        return cls(ls.xyz, ls.offsets, ls.n, ls.radius, **kw)

    def close(self):
        if self._h is not None:
            _load().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- lists
    def build_lists(self) -> int:
        if self._F is None:
            self._F = int(_load().or_build_lists(self._h))
        return self._F

    def lists(self):
        F = self.build_lists()
        nv = self.n ** 3
        count = np.zeros(nv, np.uint32)
        occ_nom = np.zeros(nv, np.uint32)
        occ_lo = np.zeros(nv, np.uint32)
        occ_hi = np.zeros(nv, np.uint32)
        start = np.zeros(nv + 1, np.uint64)
        ids = np.zeros(max(F, 1), np.uint32)
        _load().or_get_lists(self._h, _ptr(count), _ptr(occ_nom), _ptr(occ_lo), _ptr(occ_hi),
                             _ptr(start), _ptr(ids))
        return dict(count=count, occ_nom=occ_nom, occ_lo=occ_lo, occ_hi=occ_hi, start=start,
                    ids=ids[:F], F=F, ambiguous=int(_load().or_ambiguous(self._h)))

    def vertices(self):
        V = self.V
        pos = np.zeros((V, 3)); nrm = np.zeros((V, 3))
        en = np.zeros(V, np.uint8); first = np.zeros(V, np.uint8); last = np.zeros(V, np.uint8)
        _load().or_get_vertices(self._h, _ptr(pos), _ptr(nrm), _ptr(en), _ptr(first), _ptr(last))
        return dict(pos=pos, nrm=nrm, en=en, first=first, last=last)

    # ----------------------------------------------------------------- mips
    def mips(self):
        lib = _load()
        total = 0
        m = self.n
        while m >= 1:
            total += m ** 3
            m //= 2
        out = np.zeros(total)
        lib.or_build_mips(self._h, _ptr(out))
        levels, off, m = [], 0, self.n
        while m >= 1:
            levels.append(out[off:off + m ** 3].reshape(m, m, m))
            off += m ** 3
            m //= 2
        return levels

    def ao(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        return float(_load().or_ao(self._h, _ptr(p)))

    def voxel_shade(self, x, y, z, light, ao_cones=0):
        """Voxel-space shading value at the centre of voxel (x, y, z) (Sec. 3.4):
        AO (when ao_cones) times 1/2 + 1/2 * shadow transmittance toward light."""
        lt = np.ascontiguousarray(light, dtype=np.float32)
        return float(_load().or_voxel_shade(self._h, int(x), int(y), int(z), int(ao_cones), _ptr(lt)))

    # --------------------------------------------------------------- render
    def render(self, cam, alpha=1.0, ao_cones=0, brute=False, pix_begin=0, pix_end=None,
               bands=None, voxel_shading=0, light=(0.0, 0.0, 1.0)):
        lib = _load()
        prm = _prm(alpha, ao_cones, bands, voxel_shading, light)
        c = _cam(cam)
        npx = cam.width * cam.height
        pix_end = npx if pix_end is None else pix_end
        n = pix_end - pix_begin
        rgba = np.zeros((n, 4), np.float32)
        rgba_alt = np.zeros((n, 4), np.float32)
        fid = np.zeros(n, np.int32)
        fid_alt = np.zeros(n, np.int32)
        ft = np.zeros(n, np.float32)
        ex = np.zeros(n, np.uint8)
        lib.or_render(self._h, ctypes.byref(c), ctypes.byref(prm), int(bool(brute)),
                      int(pix_begin), int(pix_end), _ptr(rgba), _ptr(rgba_alt), _ptr(fid),
                      _ptr(fid_alt), _ptr(ft), _ptr(ex))
        return dict(rgba=rgba, rgba_alt=rgba_alt, first_id=fid, first_id_alt=fid_alt,
                    first_t=ft, exempt=ex)


    # ------------------------------------------------------- sampled checks
    def voxel_fragments(self, x, y, z):
        """Segments listed in voxel (x, y, z) (increasing ids) and its occupancy
        code sums (nominal, lowest, highest), by brute force over every segment."""
        lib = _load()
        occ = np.zeros(3, np.uint64)
        n = int(lib.or_voxel_fragments(self._h, int(x), int(y), int(z), None, 0, _ptr(occ)))
        ids = np.zeros(max(n, 1), np.uint32)
        lib.or_voxel_fragments(self._h, int(x), int(y), int(z), _ptr(ids), n, _ptr(occ))
        return ids[:n], tuple(int(v) for v in occ)

    def render_pixels(self, cam, pix, alpha=1.0, ao_cones=0, brute=False, bands=None,
                      voxel_shading=0, light=(0.0, 0.0, 1.0)):
        """Render the listed pixels (row-major indices); outputs as render()."""
        lib = _load()
        prm = _prm(alpha, ao_cones, bands, voxel_shading, light)
        c = _cam(cam)
        pix = np.ascontiguousarray(pix, np.int64)
        n = pix.shape[0]
        rgba = np.zeros((n, 4), np.float32)
        rgba_alt = np.zeros((n, 4), np.float32)
        fid = np.zeros(n, np.int32)
        fid_alt = np.zeros(n, np.int32)
        ft = np.zeros(n, np.float32)
        ex = np.zeros(n, np.uint8)
        lib.or_render_pixels(self._h, ctypes.byref(c), ctypes.byref(prm), int(bool(brute)),
                             _ptr(pix), n, _ptr(rgba), _ptr(rgba_alt), _ptr(fid), _ptr(fid_alt),
                             _ptr(ft), _ptr(ex))
        return dict(rgba=rgba, rgba_alt=rgba_alt, first_id=fid, first_id_alt=fid_alt,
                    first_t=ft, exempt=ex)


# ------------------------------------------------------------ single functions
def seg_box_within(A, B, lo, S, R) -> bool:
    A = np.ascontiguousarray(A, np.int64); B = np.ascontiguousarray(B, np.int64)
    lo = np.ascontiguousarray(lo, np.int64)
    return bool(_load().or_seg_box_within(_ptr(A), _ptr(B), _ptr(lo), int(S), int(R)))


def _d3(v):
    return np.ascontiguousarray(v, np.float64)


def clipped_capsule_sdf(p, v0, v1, n0=(0, 0, 0), n1=(0, 0, 0), en0=0, en1=0, r=0.5) -> float:
    a = [_d3(x) for x in (p, v0, v1, n0, n1)]
    return float(_load().or_clipped_capsule_sdf(*[_ptr(x) for x in a], int(en0), int(en1),
                                                float(r)))


def capsule_occupancy(p, v0, v1, n0=(0, 0, 0), n1=(0, 0, 0), en0=0, en1=0, r=0.5,
                      r_min=0.5) -> float:
    a = [_d3(x) for x in (p, v0, v1, n0, n1)]
    return float(_load().or_capsule_occupancy(*[_ptr(x) for x in a], int(en0), int(en1),
                                              float(r), float(r_min)))


def line_capsule_entry(o, d, a, b, r) -> float:
    v = [_d3(x) for x in (o, d, a, b)]
    return float(_load().or_line_capsule_entry(*[_ptr(x) for x in v], float(r)))


def camera_ray(cam, px, py):
    o = np.zeros(3); d = np.zeros(3)
    c = _cam(cam)
    _load().or_camera_ray(ctypes.byref(c), int(px), int(py), _ptr(o), _ptr(d))
    return o, d
