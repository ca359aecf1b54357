"""Seeded synthetic line sets and cameras shaped like the paper's workloads.

This module only draws inputs: polyline vertices (float32, voxel units), polyline
offsets (int64) and camera descriptions. It holds none of the rendering method's
arithmetic (no snapping, voxelization, intersection or shading), so the CUDA path
and the CPU oracle can both consume it without sharing any of the method.

The paper's datasets (HCP tractograms, flow streamlines; Table 1) are not
available, so these generators stand in for them with the shapes the workloads
describe:

* ``tiny_walks``  -- random-walk polylines in a 64^3 grid (opaque, orthographic).
* ``bundles``     -- tractography-like bundles of streamlines around cubic-spline
                     centerlines inside an ellipsoid, with a per-frame replacement
                     of a contiguous block of streamlines (interactive filtering).
* ``abc_pathlines`` -- RK4 lines in a time-varying ABC flow, every vertex moving
                     each frame.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20251009


@dataclasses.dataclass
class LineSet:
    xyz: np.ndarray        # float32 [V, 3]
    offsets: np.ndarray    # int64 [P + 1]; polyline p owns vertices offsets[p]..offsets[p+1]-1
    n: int                 # grid side
    radius: float          # tube radius in voxels

    @property
    def n_vertices(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_polylines(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_segments(self) -> int:
        lens = np.diff(self.offsets)
        return int(np.maximum(lens - 1, 0).sum())


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    ortho: int
    eye: tuple
    target: tuple
    up: tuple
    fovy_deg: float = 45.0
    ortho_h: float = 0.0


@dataclasses.dataclass
class RenderParams:
    alpha: float = 1.0
    ao_cones: int = 0
    cull: int = 0
    k: int = 0          # 0 = choose from alpha


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _random_perp(rng, u):
    """Random unit vectors perpendicular to the rows of u."""
    w = rng.normal(size=u.shape)
    w -= (w * u).sum(-1, keepdims=True) * u
    return _unit(w)


# ----------------------------------------------------------------------------
# Config: tiny opaque random walks
# ----------------------------------------------------------------------------
def tiny_walks(n_lines=2000, n_verts=50, n=64, radius=0.4, step=0.5,
               turn_deg=10.0, seed=SEED_BASE + 0, lo=1.0, hi=None,
               start_lo=8.0, start_hi=None) -> LineSet:
    """Random walks: step ``step`` voxels, turn ~N(0, turn_deg) about a random
    perpendicular axis, starts uniform in [start_lo, start_hi]^3, reflected at
    [lo, hi] on every axis."""
    rng = np.random.default_rng(seed)
    hi = float(n - 1) if hi is None else hi
    start_hi = float(n - 8) if start_hi is None else start_hi
    p = rng.uniform(start_lo, start_hi, size=(n_lines, 3))
    u = _unit(rng.normal(size=(n_lines, 3)))
    out = np.empty((n_lines, n_verts, 3), dtype=np.float64)
    out[:, 0] = p
    for s in range(1, n_verts):
        w = _random_perp(rng, u)
        th = np.deg2rad(rng.normal(0.0, turn_deg, size=(n_lines, 1)))
        u = _unit(u * np.cos(th) + np.cross(w, u) * np.sin(th))
        p = p + step * u
        for k in range(3):
            below = p[:, k] < lo
            p[below, k] = 2 * lo - p[below, k]
            u[below, k] = -u[below, k]
            above = p[:, k] > hi
            p[above, k] = 2 * hi - p[above, k]
            u[above, k] = -u[above, k]
        out[:, s] = p
    xyz = out.reshape(-1, 3).astype(np.float32)
    offsets = np.arange(0, n_lines * n_verts + 1, n_verts, dtype=np.int64)
    return LineSet(xyz=xyz, offsets=offsets, n=n, radius=radius)


def walk_set(n_segments, n, radius=0.4, verts_range=(20, 200), seed=SEED_BASE + 3,
             step=0.5, turn_deg=10.0) -> LineSet:
    """Random walks (as tiny_walks) of uniformly random length in verts_range,
    about n_segments segments in all, starting anywhere in the grid's interior."""
    rng = np.random.default_rng(seed)
    lo, hi = verts_range
    lens = []
    segs = 0
    while segs < n_segments:
        L = int(rng.integers(lo, hi + 1))
        L = min(L, n_segments - segs + 1)
        if L < 2:
            break
        lens.append(L)
        segs += L - 1
    lens = np.asarray(lens, dtype=np.int64)
    full = tiny_walks(n_lines=lens.shape[0], n_verts=int(lens.max()), n=n, radius=radius, step=step,
                      turn_deg=turn_deg, seed=seed + 1, start_lo=2.0, start_hi=float(n - 2))
    keep = np.arange(int(lens.max()))[None, :] < lens[:, None]
    xyz = full.xyz.reshape(lens.shape[0], int(lens.max()), 3)[keep]
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return LineSet(xyz=np.ascontiguousarray(xyz, np.float32), offsets=offsets, n=n, radius=radius)


def tiny_walks_camera(n=64, width=256, height=256) -> Camera:
    c = n / 2.0
    return Camera(width=width, height=height, ortho=1,
                  eye=(c, c, -1.0), target=(c, c, float(n)), up=(0.0, 1.0, 0.0),
                  ortho_h=float(n))


# ----------------------------------------------------------------------------
# Config: tractography-like bundles (dynamic: a block of streamlines replaced
# per frame)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class _Bundle:
    ctrl: np.ndarray     # [5, 3]
    width: float


def _ellipsoid_point(rng, center, axes, scale=1.0):
    while True:
        q = rng.uniform(-1.0, 1.0, size=3)
        if (q * q).sum() <= 1.0:
            return center + scale * q * axes


def _make_bundles(rng, n_bundles, center, axes):
    out = []
    for _ in range(n_bundles):
        while True:
            s = _ellipsoid_point(rng, center, axes, 0.9)
            e = _ellipsoid_point(rng, center, axes, 0.9)
            if np.linalg.norm(e - s) >= 80.0:
                break
        ctrl = [s]
        for k in (1, 2, 3):
            m = s + (e - s) * (k / 4.0) + rng.normal(0.0, 20.0, size=3)
            q = (m - center) / axes
            rr = math.sqrt((q * q).sum())
            if rr > 0.9:
                m = center + q / rr * 0.9 * axes
            ctrl.append(m)
        ctrl.append(e)
        out.append(_Bundle(ctrl=np.array(ctrl), width=float(rng.uniform(2.0, 6.0))))
    return out


def _catmull_rom(ctrl, u):
    """Uniform cubic Catmull-Rom spline through ``ctrl`` (K points) at u in [0,1].
    Returns positions and tangents (d/du)."""
    k = ctrl.shape[0]
    pts = np.concatenate([2 * ctrl[:1] - ctrl[1:2], ctrl, 2 * ctrl[-1:] - ctrl[-2:-1]], 0)
    x = np.clip(u, 0.0, 1.0) * (k - 1)
    seg = np.minimum(x.astype(np.int64), k - 2)
    f = (x - seg)[..., None]
    p0, p1, p2, p3 = pts[seg], pts[seg + 1], pts[seg + 2], pts[seg + 3]
    f2, f3 = f * f, f * f * f
    pos = 0.5 * ((2 * p1) + (-p0 + p2) * f + (2 * p0 - 5 * p1 + 4 * p2 - p3) * f2
                 + (-p0 + 3 * p1 - 3 * p2 + p3) * f3)
    der = 0.5 * ((-p0 + p2) + 2 * (2 * p0 - 5 * p1 + 4 * p2 - p3) * f
                 + 3 * (-p0 + 3 * p1 - 3 * p2 + p3) * f2) * (k - 1)
    return pos, der


def _bundle_streamlines(rng, b: _Bundle, n_lines, n_verts, n):
    t0 = rng.uniform(0.0, 0.05, size=(n_lines, 1))
    t1 = rng.uniform(0.95, 1.0, size=(n_lines, 1))
    u = t0 + (t1 - t0) * np.linspace(0.0, 1.0, n_verts)[None, :]
    pos, der = _catmull_rom(b.ctrl, u)
    tan = _unit(der)
    ref = np.zeros(3)
    ref[np.argmin(np.abs(tan.reshape(-1, 3).mean(0)))] = 1.0
    n1 = _unit(np.cross(tan, ref))
    n2 = np.cross(tan, n1)
    sig = b.width / 2.0
    off = rng.normal(0.0, sig, size=(n_lines, 1, 2))
    # smooth low-amplitude noise along the line
    amp = 0.15 * sig
    ph = rng.uniform(0, 2 * np.pi, size=(n_lines, 1, 2))
    fr = rng.uniform(1.0, 4.0, size=(n_lines, 1, 2))
    s = np.linspace(0.0, 1.0, n_verts)[None, :, None]
    off = off + amp * np.sin(2 * np.pi * fr * s + ph)
    p = pos + off[..., :1] * n1 + off[..., 1:] * n2
    return np.clip(p, 1.0, n - 1.0)


@dataclasses.dataclass
class BundleSet:
    lineset: LineSet
    bundles: list
    line_bundle: np.ndarray    # [P] bundle index of each streamline
    n_verts: int
    seed: int


def bundles(n_lines=100_000, n_verts=100, n_bundles=30, n=256, radius=0.35,
            seed=SEED_BASE + 1) -> BundleSet:
    rng = np.random.default_rng(seed)
    scale = n / 256.0
    center = np.array([128.0, 128.0, 128.0]) * scale
    axes = np.array([110.0, 90.0, 100.0]) * scale
    bl = _make_bundles(rng, n_bundles, center, axes)
    line_bundle = (np.arange(n_lines) * n_bundles) // n_lines
    xyz = np.empty((n_lines, n_verts, 3), dtype=np.float32)
    for bi, b in enumerate(bl):
        idx = np.nonzero(line_bundle == bi)[0]
        if idx.size:
            xyz[idx] = _bundle_streamlines(rng, b, idx.size, n_verts, n)
    offsets = np.arange(0, n_lines * n_verts + 1, n_verts, dtype=np.int64)
    ls = LineSet(xyz=xyz.reshape(-1, 3), offsets=offsets, n=n, radius=radius)
    return BundleSet(lineset=ls, bundles=bl, line_bundle=line_bundle, n_verts=n_verts, seed=seed)


def bundles_update(bs: BundleSet, frame: int, fraction=0.05):
    """Replacement streamlines for one frame of interactive filtering: a
    contiguous block of ``fraction`` of the streamlines, redrawn from the same
    bundles with a frame-dependent seed. Returns (first_vertex, xyz [k, 3])."""
    p = bs.lineset.n_polylines
    k = max(1, int(round(p * fraction)))
    first = (frame * k) % p
    if first + k > p:
        first = p - k
    rng = np.random.default_rng(bs.seed * 1000 + 7 + frame)
    out = np.empty((k, bs.n_verts, 3), dtype=np.float32)
    lb = bs.line_bundle[first:first + k]
    for bi in np.unique(lb):
        idx = np.nonzero(lb == bi)[0]
        out[idx] = _bundle_streamlines(rng, bs.bundles[bi], idx.size, bs.n_verts, bs.lineset.n)
    return first * bs.n_verts, out.reshape(-1, 3)


def bundles_camera(n=256, width=1920, height=1080, seed=SEED_BASE + 1, radius=300.0,
                   elevation_deg=20.0) -> Camera:
    rng = np.random.default_rng(seed + 99)
    th = rng.uniform(0.0, 2 * np.pi)
    el = np.deg2rad(elevation_deg)
    c = np.array([n / 2.0] * 3)
    rad = radius * n / 256.0
    eye = c + rad * np.array([np.cos(el) * np.cos(th), np.cos(el) * np.sin(th), np.sin(el)])
    return Camera(width=width, height=height, ortho=0, eye=tuple(map(float, eye)),
                  target=tuple(map(float, c)), up=(0.0, 0.0, 1.0), fovy_deg=45.0)


# ----------------------------------------------------------------------------
# Config: unsteady ABC-flow pathlines (every vertex changes each frame)
# ----------------------------------------------------------------------------
ABC = (math.sqrt(3.0), math.sqrt(2.0), 1.0)


def _abc_velocity(x, phase, xp):
    a, b, c = ABC
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    u = a * xp.sin(Z + phase) + c * xp.cos(Y + phase)
    v = b * xp.sin(X + phase) + a * xp.cos(Z + phase)
    w = c * xp.sin(Y + phase) + b * xp.cos(X + phase)
    return xp.stack([u, v, w], -1)


def abc_pathlines(n_particles=1_000_000, n_verts=32, n=512, radius=0.25, frame=0,
                  seed=SEED_BASE + 2, xp=np, device=None):
    """Lines traced by RK4 through the ABC flow with phase 0.1*frame; the domain
    [0, 2pi)^3 maps to [0, n)^3. Seeds are uniform in the central [n/8, 7n/8]^3.
    The step is chosen so that the mean segment length is about one voxel.
    ``xp`` may be numpy or torch (with ``device``) for large sets."""
    rng = np.random.default_rng(seed)
    seeds = rng.uniform(n / 8.0, 7.0 * n / 8.0, size=(n_particles, 3))
    to_flow = 2 * np.pi / n
    phase = 0.1 * frame
    dt = 1.0 * to_flow / 2.2  # mean |u| of the ABC field is about 2.2
    if xp is np:
        x = seeds * to_flow
        out = np.empty((n_particles, n_verts, 3), dtype=np.float32)
        out[:, 0] = seeds
        for s in range(1, n_verts):
            k1 = _abc_velocity(x, phase, np)
            k2 = _abc_velocity(x + 0.5 * dt * k1, phase, np)
            k3 = _abc_velocity(x + 0.5 * dt * k2, phase, np)
            k4 = _abc_velocity(x + dt * k3, phase, np)
            x = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            out[:, s] = x / to_flow
        xyz = np.clip(out, 0.5, n - 0.5).reshape(-1, 3)
    else:
        torch = xp
        x = torch.as_tensor(seeds * to_flow, dtype=torch.float64, device=device)
        out = torch.empty((n_particles, n_verts, 3), dtype=torch.float32, device=device)
        out[:, 0] = (x / to_flow).float()
        for s in range(1, n_verts):
            k1 = _abc_velocity(x, phase, torch)
            k2 = _abc_velocity(x + 0.5 * dt * k1, phase, torch)
            k3 = _abc_velocity(x + 0.5 * dt * k2, phase, torch)
            k4 = _abc_velocity(x + dt * k3, phase, torch)
            x = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            out[:, s] = (x / to_flow).float()
        xyz = out.clamp_(0.5, n - 0.5).reshape(-1, 3)
    offsets = np.arange(0, n_particles * n_verts + 1, n_verts, dtype=np.int64)
    return LineSet(xyz=xyz, offsets=offsets, n=n, radius=radius)


def abc_camera(n=512, frame=0, width=1920, height=1080) -> Camera:
    c = n / 2.0
    a = 0.01 * frame
    d = np.array([math.cos(a), math.sin(a), 0.2])
    d /= np.linalg.norm(d)
    return Camera(width=width, height=height, ortho=0, eye=(c, c, c),
                  target=tuple(map(float, np.array([c, c, c]) + 10.0 * d)),
                  up=(0.0, 0.0, 1.0), fovy_deg=45.0)


# ----------------------------------------------------------------------------
# Small structured sets for tests
# ----------------------------------------------------------------------------
def random_polylines(n_lines, n_verts_range, n, radius, seed, step=(0.2, 3.0),
                     margin=1.0):
    """Polylines of random length with random steps, kept inside [margin, n-margin]."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(n_verts_range[0], n_verts_range[1] + 1, size=n_lines)
    pts = []
    for L in lens:
        p = rng.uniform(margin, n - margin, size=3)
        line = [p.copy()]
        for _ in range(int(L) - 1):
            d = _unit(rng.normal(size=3)) * rng.uniform(*step)
            p = np.clip(p + d, margin, n - margin)
            line.append(p.copy())
        pts.append(np.array(line).reshape(-1, 3))
    xyz = np.concatenate(pts, 0).astype(np.float32) if pts else np.zeros((0, 3), np.float32)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return LineSet(xyz=xyz, offsets=offsets, n=n, radius=radius)
