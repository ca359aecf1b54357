"""Pins for the CPU oracle: each checks it against something other than itself
(exact rational brute force, closed forms from the paper's definitions,
invariants the paper states), so that a dropped term, a wrong sign or index, or
a transposed operand in the oracle fails one of them."""
from fractions import Fraction as Fr
import itertools
import math

import numpy as np
import pytest

import oracle
from gen.linesets import Camera, LineSet, random_polylines, tiny_walks, tiny_walks_camera

U = 16384  # oracle units per voxel


# ----------------------------------------------------------------------------
# exact segment-box predicate
# ----------------------------------------------------------------------------
def _min_dist2_exact(A, B, lo, hi):
    """Exact min over t in [0,1] of the squared distance from A + t(B - A) to
    the box [lo, hi] (Fractions). The distance is convex and piecewise
    quadratic in t with kinks where a coordinate crosses a face plane."""
    A = [Fr(int(x)) for x in A]
    D = [Fr(int(b)) - a for a, b in zip(A, B)]
    lo = [int(x) for x in lo]
    hi = [int(x) for x in hi]
    kinks = {Fr(0), Fr(1)}
    for k in range(3):
        if D[k] != 0:
            for plane in (lo[k], hi[k]):
                t = (Fr(plane) - A[k]) / D[k]
                if 0 < t < 1:
                    kinks.add(t)
    ks = sorted(kinks)

    def f(t):
        s = Fr(0)
        for k in range(3):
            x = A[k] + t * D[k]
            e = lo[k] - x if x < lo[k] else (x - hi[k] if x > hi[k] else 0)
            s += e * e
        return s

    best = min(f(t) for t in ks)
    for a, b in zip(ks[:-1], ks[1:]):
        m = (a + b) / 2
        # quadratic on this piece: sum over axes outside at m of (A + tD - plane)^2
        qa = qb = Fr(0)
        for k in range(3):
            x = A[k] + m * D[k]
            if x < lo[k] or x > hi[k]:
                pl = lo[k] if x < lo[k] else hi[k]
                w = A[k] - pl
                qa += D[k] * D[k]
                qb += 2 * w * D[k]
        if qa > 0:
            ts = -qb / (2 * qa)
            if a < ts < b:
                best = min(best, f(ts))
    return best


def test_predicate_matches_rational_brute_force():
    rng = np.random.default_rng(1)
    S = 8
    n_true = 0
    for trial in range(3000):
        A = rng.integers(-12, 20, size=3)
        B = A + rng.integers(-10, 11, size=3)
        if trial % 5 == 0:
            B = A.copy()  # degenerate segments
        lo = rng.integers(-2, 6, size=3)
        R = int(rng.integers(1, 9))
        exact = _min_dist2_exact(A, B, lo, lo + S) <= R * R
        got = oracle.seg_box_within(A, B, lo, S, R)
        assert got == exact, (A, B, lo, R)
        n_true += exact
    assert 300 < n_true < 2700  # both outcomes well represented


def test_predicate_exact_ties():
    """Segments whose distance to the box is exactly R are listed (closed sets),
    one unit further they are not: face, edge and corner contacts."""
    S, R = 100, 30
    lo = np.array([0, 0, 0])
    cases = [
        # face contact: parallel to x at y = -R
        ((-50, -R, 50), (150, -R, 50)),
        # edge contact: along z, distance to edge (x=S, y=S) exactly R (3-4-5)
        ((S + 18, S + 24, -40), (S + 18, S + 24, 140)),
        # corner contact: starts at (S,S,S) + (10,20,20), |(10,20,20)| = R, and
        # runs away from the box
        ((S + 10, S + 20, S + 20), (S + 20, S + 40, S + 40)),
    ]
    for A, B in cases:
        A, B = np.array(A), np.array(B)
        assert _min_dist2_exact(A, B, lo, lo + S) == R * R
        assert oracle.seg_box_within(A, B, lo, S, R)
        assert not oracle.seg_box_within(A, B, lo, S, R - 1)


def _lists_of(o):
    L = o.lists()
    n = o.n
    out = {}
    for v in np.nonzero(L["count"])[0]:
        s, e = int(L["start"][v]), int(L["start"][v + 1])
        z, y, x = v // (n * n), (v // n) % n, v % n
        out[(int(x), int(y), int(z))] = list(map(int, L["ids"][s:e]))
    return out, L


def _single(a, b, n=16, r=0.4):
    xyz = np.array([a, b], np.float32)
    return oracle.Oracle(xyz, np.array([0, 2]), n, r)


def test_hand_case_offset_axis_segment():
    """Segment along x at y = z = 1.3, r = 0.4: rows (j,k) = (1,1), (0,1), (1,0)
    are within 0.3 of it, the diagonal row (0,0) is at sqrt(0.18) = 0.424 > 0.4
    (and above the list radius 0.4 + 2^-9)."""
    o = _single((2.25, 1.3, 1.3), (6.75, 1.3, 1.3))
    lists, _ = _lists_of(o)
    rows = {(y, z) for (x, y, z) in lists}
    assert rows == {(1, 1), (0, 1), (1, 0)}
    xs = {x for (x, y, z) in lists}
    # x extent [2.25 - 0.4, 6.75 + 0.4] touches voxels 1..7
    assert xs == set(range(1, 8))


def test_hand_case_segment_on_edge():
    """Segment lying on the edge y = z = 1 lists all four rows around it."""
    o = _single((2.5, 1.0, 1.0), (5.5, 1.0, 1.0))
    lists, _ = _lists_of(o)
    rows = {(y, z) for (x, y, z) in lists}
    assert rows == {(0, 0), (0, 1), (1, 0), (1, 1)}


def _fp64_seg_box_dist(a, b, lo):
    """Segment-box distance by golden-section search on the convex function."""
    a, b, lo = map(np.asarray, (a, b, lo))

    def f(t):
        p = a + t * (b - a)
        e = np.maximum(0, np.maximum(lo - p, p - (lo + 1)))
        return float(np.sqrt((e * e).sum()))

    lo_t, hi_t = 0.0, 1.0
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        m1 = hi_t - g * (hi_t - lo_t)
        m2 = lo_t + g * (hi_t - lo_t)
        if f(m1) <= f(m2):
            hi_t = m2
        else:
            lo_t = m1
    return min(f(0.0), f(1.0), f(0.5 * (lo_t + hi_t)))


def test_lists_are_exactly_the_voxels_within_list_radius():
    """Listed voxels are within r + 2^-9 of the segment, every other voxel of the
    segment's neighbourhood is not (fp64 search, away from near-ties), and lists
    come out sorted by segment id."""
    ls = random_polylines(6, (2, 6), 16, 0.45, seed=3)
    o = oracle.Oracle.from_lineset(ls)
    lists, L = _lists_of(o)
    vt = o.vertices()
    pos = vt["pos"]
    rl = round(0.45 * U) / U + 2 ** -9
    member = {}
    for vox, ids in lists.items():
        assert ids == sorted(ids)
        for i in ids:
            member[(i, vox)] = True
    checked = 0
    for i in range(ls.n_vertices - 1):
        if vt["last"][i]:
            continue
        a, b = pos[i], pos[i + 1]
        lo = np.floor(np.minimum(a, b) - 2).astype(int)
        hi = np.floor(np.maximum(a, b) + 2).astype(int)
        for x, y, z in itertools.product(*[range(max(0, lo[k]), min(16, hi[k] + 1)) for k in range(3)]):
            d = _fp64_seg_box_dist(a, b, (x, y, z))
            if abs(d - rl) < 1e-7:
                continue
            assert ((i, (x, y, z)) in member) == (d <= rl), (i, (x, y, z), d)
            checked += 1
    assert checked > 1000


def test_lists_brute_force_over_whole_grid():
    """On an 16^3 grid, the voxels listing each segment equal the voxels whose
    exact rational distance to the segment is within the list radius, over all
    4096 voxels (not just the oracle's candidate box)."""
    ls = random_polylines(2, (2, 3), 16, 0.6, seed=11)
    o = oracle.Oracle.from_lineset(ls)
    lists, _ = _lists_of(o)
    X = np.rint(ls.xyz.astype(np.float64) * U).astype(np.int64)
    RL = round(0.6 * U) + 32
    for i in range(ls.n_vertices - 1):
        if i + 1 in ls.offsets[1:-1] or i == ls.n_vertices - 1:
            continue
        if any(i == e - 1 for e in ls.offsets[1:]):
            continue
        want = set()
        for x, y, z in itertools.product(range(16), repeat=3):
            lo = np.array([x, y, z]) * U
            # cheap exact reject: AABB gap
            gap = np.maximum(0, np.maximum(lo - np.maximum(X[i], X[i + 1]),
                                           np.minimum(X[i], X[i + 1]) - (lo + U)))
            if (gap.astype(object) ** 2).sum() > RL * RL:
                continue
            if _min_dist2_exact(X[i], X[i + 1], lo, lo + U) <= RL * RL:
                want.add((x, y, z))
        got = {v for v, ids in lists.items() if i in ids}
        assert got and got == want


def test_every_point_within_r_lies_in_a_listing_voxel():
    """Conservativeness (Sec. 3.1): any point within r of a segment lies in a
    voxel that lists the segment."""
    ls = random_polylines(20, (2, 8), 32, 0.35, seed=5)
    o = oracle.Oracle.from_lineset(ls)
    lists, _ = _lists_of(o)
    pos = o.vertices()["pos"]
    last = o.vertices()["last"]
    r = round(0.35 * U) / U
    rng = np.random.default_rng(0)
    n = 0
    for i in range(ls.n_vertices - 1):
        if last[i]:
            continue
        for _ in range(200):
            t = rng.uniform()
            q = pos[i] + t * (pos[i + 1] - pos[i])
            off = rng.normal(size=3)
            off *= r * rng.uniform() ** (1 / 3) / np.linalg.norm(off)
            p = q + off
            v = tuple(int(c) for c in np.floor(p))
            if min(v) < 0 or max(v) >= 32:
                continue
            assert i in lists.get(v, []), (i, p)
            n += 1
    assert n > 10000


def test_snap_and_normals():
    """Vertices are snapped to the 2^-14 grid (round half to even); clip normals
    are the unit central difference at interior vertices and disabled at
    polyline ends and where the central difference vanishes."""
    xyz = np.array([[1.00003, 2.0, 3.0], [2.0, 2.0, 3.0], [3.0, 4.0, 3.0],
                    [5.0, 5.0, 5.0], [6.0, 5.0, 5.0], [5.0, 5.0, 5.0], [4.0, 4.0, 4.0]],
                   np.float32)
    off = np.array([0, 3, 7])
    o = oracle.Oracle(xyz, off, 16, 0.3)
    v = o.vertices()
    want = np.rint(xyz.astype(np.float64) * U) / U
    assert np.array_equal(v["pos"], want)
    assert list(v["first"]) == [1, 0, 0, 1, 0, 0, 0]
    assert list(v["last"]) == [0, 0, 1, 0, 0, 0, 1]
    assert list(v["en"]) == [0, 1, 0, 0, 0, 1, 0]  # vertex 4: v5 - v3 = 0 -> disabled
    d = want[2] - want[0]
    assert np.allclose(v["nrm"][1], d / np.linalg.norm(d), atol=1e-15)


# ----------------------------------------------------------------------------
# Alg. 2 / Alg. 3
# ----------------------------------------------------------------------------
def test_sdf_closed_forms():
    v0, v1 = (0, 0, 0), (2, 0, 0)
    # on the axis: -r
    assert oracle.clipped_capsule_sdf((1, 0, 0), v0, v1, r=0.4) == pytest.approx(-0.4)
    # beside the body at distance 1: 1 - r
    assert oracle.clipped_capsule_sdf((1.5, 0.6, 0.8), v0, v1, r=0.4) == pytest.approx(0.6)
    # beyond the end cap (unclipped): distance to v1 minus r
    assert oracle.clipped_capsule_sdf((2.3, 0.4, 0), v0, v1, r=0.4) == pytest.approx(0.1)
    # behind v0 with the plane n0 = +x enabled: the plane term wins
    s = oracle.clipped_capsule_sdf((-0.3, 0, 0), v0, v1, n0=(1, 0, 0), en0=1, r=0.4)
    assert s == pytest.approx(0.3)
    # plane disabled: round cap
    s = oracle.clipped_capsule_sdf((-0.3, 0, 0), v0, v1, n0=(1, 0, 0), en0=0, r=0.4)
    assert s == pytest.approx(-0.1)
    # beyond v1 with n1 = +x enabled: plane term p.n1 - v1.n1
    s = oracle.clipped_capsule_sdf((2.2, 0.1, 0), v0, v1, n1=(1, 0, 0), en1=1, r=0.4)
    assert s == pytest.approx(0.2)
    # a tilted plane at v1 (45 degrees) cuts the cap: point on the axis past v1
    n = np.array([1, 1, 0]) / math.sqrt(2)
    s = oracle.clipped_capsule_sdf((2.1, 0, 0), v0, v1, n1=n, en1=1, r=0.4)
    assert s == pytest.approx(max(0.1 - 0.4, 0.1 / math.sqrt(2)))


def test_occupancy_closed_forms():
    v0, v1 = (0, 0, 0), (4, 0, 0)
    # on the axis, r < r_min: sdf = -r_min, occ = clamp(0.5 + 0.5) * (r/r_min)^2
    assert oracle.capsule_occupancy((2, 0, 0), v0, v1, r=0.4, r_min=0.5) == pytest.approx(0.64)
    # r = 0.25, one voxel off-axis: sdf = 1 - 0.5 -> occupancy 0
    assert oracle.capsule_occupancy((2, 1, 0), v0, v1, r=0.25, r_min=0.5) == 0.0
    # r >= r_min: no correction; on the axis occupancy saturates at 1
    assert oracle.capsule_occupancy((2, 0, 0), v0, v1, r=0.75, r_min=0.5) == pytest.approx(1.0)
    # half a voxel off-axis with r = r_min: sdf = 0 -> 0.5
    assert oracle.capsule_occupancy((2, 0.5, 0), v0, v1, r=0.5, r_min=0.5) == pytest.approx(0.5)
    # 0.7 off-axis, r = 0.6: sdf = 0.1 -> 0.4
    assert oracle.capsule_occupancy((2, 0, 0.7), v0, v1, r=0.6, r_min=0.5) == pytest.approx(0.4)


def test_occupancy_sums_over_listed_voxels():
    """Per-voxel occupancy codes are the sum of round(Q * Alg3(centre)) over the
    segments listed in that voxel (Q = 32), recomputed here from the closed
    form for a single straight segment (no clip planes)."""
    a, b = np.array([3.25, 4.5, 5.75]), np.array([9.5, 6.25, 5.0])
    o = _single(tuple(a), tuple(b), n=16, r=0.4)
    lists, L = _lists_of(o)
    assert lists
    for (x, y, z), ids in lists.items():
        p = np.array([x + 0.5, y + 0.5, z + 0.5])
        d = b - a
        h = np.clip(np.dot(p - a, d) / np.dot(d, d), 0, 1)
        sdf = np.linalg.norm(p - a - h * d) - 0.5
        occ = np.clip(0.5 - sdf, 0, 1) * (round(0.4 * U) / U / 0.5) ** 2
        q = math.floor(32 * occ + 0.5)
        v = (z * 16 + y) * 16 + x
        assert L["occ_lo"][v] <= q <= L["occ_hi"][v]


# ----------------------------------------------------------------------------
# rays
# ----------------------------------------------------------------------------
def test_line_capsule_closed_forms():
    a, b, r = (0, 0, 0), (2, 0, 0), 0.5
    # perpendicular through the axis from distance 3: t = 3 - r
    assert oracle.line_capsule_entry((1, 3, 0), (0, -1, 0), a, b, r) == pytest.approx(2.5)
    # perpendicular, offset 0.3 from the axis: t = 3 - sqrt(r^2 - 0.09)
    assert oracle.line_capsule_entry((1, 3, 0.3), (0, -1, 0), a, b, r) == pytest.approx(2.6)
    # along the axis: cap at t = 5 - r
    assert oracle.line_capsule_entry((-5, 0, 0), (1, 0, 0), a, b, r) == pytest.approx(4.5)
    # parallel, offset 0.3: cap sphere at t = 5 - 0.4
    assert oracle.line_capsule_entry((-5, 0.3, 0), (1, 0, 0), a, b, r) == pytest.approx(4.6)
    # from the other end (direction is normalised inside)
    assert oracle.line_capsule_entry((7, 0, 0.3), (-2, 0, 0), a, b, r) == pytest.approx(4.6)
    # miss
    assert oracle.line_capsule_entry((1, 3, 0.6), (0, -1, 0), a, b, r) == math.inf
    # origin inside: the entry lies behind the origin
    assert oracle.line_capsule_entry((1, 0.1, 0), (0, 1, 0), a, b, r) < 0
    # degenerate segment = sphere
    assert oracle.line_capsule_entry((0, 0, -4), (0, 0, 1), a, a, r) == pytest.approx(3.5)
    # oblique ray hitting the body: closed form for the infinite cylinder
    d = np.array([0.0, -1.0, 1.0]) / math.sqrt(2)
    o = np.array([1.0, 2.0, -2.0])
    t = oracle.line_capsule_entry(o, d, a, b, r)
    p = o + t * d
    assert math.hypot(p[1], p[2]) == pytest.approx(r)
    assert 0 < p[0] < 2


def test_camera_rays():
    cam = Camera(width=1, height=1, ortho=0, eye=(1, 2, 3), target=(1, 2, 10), up=(0, 1, 0))
    o, d = oracle.camera_ray(cam, 0, 0)
    assert np.allclose(o, (1, 2, 3)) and np.allclose(d, (0, 0, 1))
    cam = Camera(width=4, height=2, ortho=0, eye=(0, 0, 0), target=(0, 0, 1), up=(0, 1, 0),
                 fovy_deg=90.0)
    o, d = oracle.camera_ray(cam, 3, 0)  # right-most column, top row
    # right = f x up = (-1, 0, 0); x: (2*3.5/4 - 1) * tan45 * 2 = 1.5; y: (1 - 0.5) = 0.5
    want = np.array([-1.5, 0.5, 1.0]); want /= np.linalg.norm(want)
    assert np.allclose(d, want)
    cam = tiny_walks_camera()
    o, d = oracle.camera_ray(cam, 0, 0)
    assert np.allclose(d, (0, 0, 1))
    assert np.allclose(o, (32 + (0.5 - 0.5 / 256) * 64, 32 + (0.5 - 0.5 / 256) * 64, -1))


def _ortho_down(x0, y0, z0=10.0, n=16):
    """1x1 orthographic camera whose single ray starts at (x0, y0, z0), looking -z."""
    return Camera(width=1, height=1, ortho=1, eye=(x0, y0, z0), target=(x0, y0, z0 - 1),
                  up=(0, 1, 0), ortho_h=1.0)


def test_clip_planes_at_a_right_angle_joint():
    """Polyline (4,4,4) -> (6,4,4) -> (6,6,4), r = 0.4: the joint plane has
    normal (1,1,0)/sqrt(2). A ray from above just past the plane on segment 1's
    side hits segment 1 at the top of its tube; on segment 0's side, segment 0."""
    xyz = np.array([[4, 4, 4], [6, 4, 4], [6, 6, 4]], np.float32)
    o = oracle.Oracle(xyz, np.array([0, 3]), 16, 0.4)
    r = round(0.4 * U) / U
    out = o.render(_ortho_down(6.1, 4.05), alpha=1.0)
    assert out["first_id"][0] == 1
    assert out["first_t"][0] == pytest.approx(10 - 4 - math.sqrt(r * r - 0.01), abs=1e-6)
    out = o.render(_ortho_down(5.9, 3.95), alpha=1.0)
    assert out["first_id"][0] == 0
    assert out["first_t"][0] == pytest.approx(10 - 4 - math.sqrt(r * r - 0.0025), abs=1e-6)
    # colour = |tangent|: segment 1 runs along y
    out = o.render(_ortho_down(6.1, 4.05), alpha=1.0)
    assert np.allclose(out["rgba"][0], (0, 1, 0, 1))


def test_compositing_closed_form_and_order():
    """Four parallel x-segments stacked under the ray: C = c (1 - (1-a)^4) and
    A = 1 - (1-a)^4 for colour c = (1,0,0); for two colours the nearer one is
    weighted by alpha and the farther by alpha (1 - alpha)."""
    a = 0.3
    xyz = np.array([[2, 8, z, ] for z in (1, 1, 3, 3, 5, 5, 7, 7)], np.float32)
    xyz[1::2, 0] = 12
    o = oracle.Oracle(xyz, np.array([0, 2, 4, 6, 8]), 16, 0.4)
    out = o.render(_ortho_down(7.0, 8.0), alpha=a)
    A = 1 - (1 - a) ** 4
    assert np.allclose(out["rgba"][0], (A, 0, 0, A), atol=1e-6)
    # front segment along y (green), back along x (red)
    xyz = np.array([[2, 8, 1], [12, 8, 1], [7, 3, 5], [7, 13, 5]], np.float32)
    o = oracle.Oracle(xyz, np.array([0, 2, 4]), 16, 0.4)
    out = o.render(_ortho_down(7.0, 8.0), alpha=a)
    assert np.allclose(out["rgba"][0], (a * (1 - a), a, 0, 1 - (1 - a) ** 2), atol=1e-6)
    assert out["first_id"][0] == 2


def test_list_based_render_equals_brute_force():
    """Sec. 3.5 conservativeness: tracing through the per-voxel lists finds
    exactly the hits a brute-force test of all segments finds."""
    ls = tiny_walks(n_lines=120, n_verts=30, seed=77)
    o = oracle.Oracle.from_lineset(ls)
    cam = Camera(width=48, height=40, ortho=0, eye=(80.0, 70.0, 40.0), target=(32, 32, 32),
                 up=(0, 0, 1), fovy_deg=40.0)
    for alpha in (1.0, 0.3):
        a = o.render(cam, alpha=alpha)
        b = o.render(cam, alpha=alpha, brute=True)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        assert (a["first_id"] >= 0).sum() > 300


def test_ground_truth_order_from_brute_force_hits():
    """Transparent colour equals compositing all hits sorted by depth: built here
    from per-segment entries of the brute-force oracle pieces (line entry, grid
    and clip tests) on a sparse scene."""
    ls = random_polylines(8, (2, 4), 16, 0.5, seed=21, step=(2.0, 5.0))
    o = oracle.Oracle.from_lineset(ls)
    v = o.vertices()
    cam = Camera(width=12, height=12, ortho=0, eye=(30.0, 25.0, 20.0), target=(8, 8, 8),
                 up=(0, 0, 1), fovy_deg=35.0)
    out = o.render(cam, alpha=0.4)
    r = round(0.5 * U) / U
    for p in range(cam.width * cam.height):
        if out["exempt"][p]:
            continue
        org, d = oracle.camera_ray(cam, p % cam.width, p // cam.width)
        hits = []
        for i in range(ls.n_vertices - 1):
            if v["last"][i]:
                continue
            t = oracle.line_capsule_entry(org, d, v["pos"][i], v["pos"][i + 1], r)
            if not (t >= 0 and math.isfinite(t)):
                continue
            P = org + t * d
            if (P < 0).any() or (P > 16).any():
                continue
            if v["en"][i] and np.dot(P - v["pos"][i], v["nrm"][i]) < 0:
                continue
            if v["en"][i + 1] and np.dot(P - v["pos"][i + 1], v["nrm"][i + 1]) > 0:
                continue
            dd = v["pos"][i + 1] - v["pos"][i]
            hits.append((t, i, np.abs(dd) / np.linalg.norm(dd)))
        hits.sort(key=lambda h: (h[0], h[1]))
        C, T = np.zeros(3), 1.0
        for t, i, c in hits:
            C += T * 0.4 * c
            T *= 0.6
        assert np.allclose(out["rgba"][p], (*C, 1 - T), atol=1e-6)


# ----------------------------------------------------------------------------
# mips and ambient occlusion
# ----------------------------------------------------------------------------
def _full_grid(n=16):
    """Lines along x through every voxel centre row, r = 0.75: every voxel centre
    is on an axis, so every voxel's occupancy saturates."""
    ys, zs = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    a = np.stack([np.full(ys.size, 0.25), ys.ravel(), zs.ravel()], 1)
    b = np.stack([np.full(ys.size, n - 0.25), ys.ravel(), zs.ravel()], 1)
    xyz = np.stack([a, b], 1).reshape(-1, 3).astype(np.float32)
    return oracle.Oracle(xyz, np.arange(0, xyz.shape[0] + 1, 2), n, 0.75)


def test_mips_uniform_and_mass_preserving():
    o = _full_grid(16)
    lv = o.mips()
    assert len(lv) == 5
    for l in lv:
        assert np.all(l == 1.0)
    ls = random_polylines(10, (3, 8), 16, 0.4, seed=9)
    o = oracle.Oracle.from_lineset(ls)
    lv = o.mips()
    s0 = lv[0].sum()
    assert s0 > 0
    for k, l in enumerate(lv):
        assert l.sum() * 8 ** k == pytest.approx(s0, rel=1e-12)
        assert l.max() <= 1.0


def test_ao_empty_and_full():
    """No occupancy: AO = 1. Full occupancy: each cone's first sample is 1, the
    accumulated occlusion saturates and AO = 0 (Sec. 3.4 cones)."""
    o = oracle.Oracle(np.array([[1, 1, 1], [1.5, 1, 1]], np.float32), np.array([0, 2]), 16, 0.1)
    assert o.ao((12.0, 12.0, 12.0)) == 1.0
    o = _full_grid(16)
    assert o.ao((8.0, 8.0, 8.0)) == pytest.approx(0.0, abs=1e-12)


def test_ao_single_wall():
    """A full half-space (x < 8) seen from x = 9: the -x cone samples it, the
    others are partly covered; AO is strictly between 0 and 1 and symmetric in
    y and z."""
    o = _full_grid(16)
    full = o.mips()
    n = 16
    ys, zs = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    a = np.stack([np.full(ys.size, 0.25), ys.ravel(), zs.ravel()], 1)
    b = np.stack([np.full(ys.size, 7.75), ys.ravel(), zs.ravel()], 1)
    xyz = np.stack([a, b], 1).reshape(-1, 3).astype(np.float32)
    o = oracle.Oracle(xyz, np.arange(0, xyz.shape[0] + 1, 2), n, 0.75)
    ao = o.ao((9.0, 8.0, 8.0))
    assert 0.0 < ao < 1.0
    # the wall is symmetric about y = 8 and z = 8
    assert o.ao((9.0, 9.3, 8.0)) == pytest.approx(o.ao((9.0, 6.7, 8.0)), abs=1e-12)
    assert o.ao((9.0, 8.0, 9.3)) == pytest.approx(o.ao((9.0, 8.0, 6.7)), abs=1e-12)
    # further from the wall is less occluded
    assert o.ao((13.0, 8.0, 8.0)) > ao
    assert full[0].sum() > 0


# ----------------------------------------------------------------------------
# voxel-space shading (Sec. 3.4, Shading)
# ----------------------------------------------------------------------------
AXES = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def _column_shadow(occ0, x, y, z, L):
    """Transmittance from the centre of voxel (x, y, z) toward an axis light L:
    with L along an axis every sample sits on a texel centre k voxels away, so
    S is the product of (1 - occupancy) over the voxels strictly beyond this one
    up to the grid boundary."""
    n = occ0.shape[0]
    S = 1.0
    k = 1
    while True:
        u = (x + k * L[0], y + k * L[1], z + k * L[2])
        if not all(0 <= c < n for c in u):
            break
        S *= 1.0 - occ0[u[2], u[1], u[0]]
        k += 1
    return S


def test_voxel_shadow_closed_form_along_axes():
    ls = tiny_walks(n_lines=150, n_verts=40, n=16, radius=0.6, seed=41)
    o = oracle.Oracle.from_lineset(ls)
    occ0 = o.mips()[0]
    assert 0.05 < (occ0 > 0).mean() < 0.9
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(60):
        x, y, z = (int(v) for v in rng.integers(0, 16, 3))
        for L in AXES:
            S = _column_shadow(occ0, x, y, z, L)
            assert o.voxel_shade(x, y, z, L) == pytest.approx(0.5 + 0.5 * S, abs=1e-12)
            checked += S < 0.999
    assert checked > 50  # most columns are shadowed by something
    # with ambient occlusion: the cone AO at the voxel centre times the same term
    for _ in range(10):
        x, y, z = (int(v) for v in rng.integers(0, 16, 3))
        S = _column_shadow(occ0, x, y, z, (0, 0, -1))
        ao = o.ao((x + 0.5, y + 0.5, z + 0.5))
        assert o.voxel_shade(x, y, z, (0, 0, -1), ao_cones=6) == pytest.approx(ao * (0.5 + 0.5 * S),
                                                                               abs=1e-12)


def test_voxel_shadow_empty_full_and_boundary():
    """Empty grid: no shadow (1). Full grid: the first sample, one voxel toward
    the light, is fully occupied (1/2), except where that sample's texels are
    all outside the grid (1); any unnormalized light direction gives the same."""
    o = oracle.Oracle(np.array([[1, 1, 1], [1.5, 1, 1]], np.float32), np.array([0, 2]), 16, 0.1)
    assert o.voxel_shade(10, 10, 10, (0.3, -0.2, 0.9)) == 1.0
    o = _full_grid(16)
    assert o.voxel_shade(7, 7, 7, (0.3, -0.2, 0.9)) == pytest.approx(0.5, abs=1e-12)
    assert o.voxel_shade(14, 3, 3, (1, 0, 0)) == pytest.approx(0.5, abs=1e-12)
    assert o.voxel_shade(15, 3, 3, (1, 0, 0)) == pytest.approx(1.0, abs=1e-12)
    assert o.voxel_shade(15, 3, 3, (-2, 0, 0)) == pytest.approx(0.5, abs=1e-12)
    assert o.voxel_shade(0, 3, 3, (-1, 0, 0)) == pytest.approx(1.0, abs=1e-12)


def test_render_samples_the_voxel_shading_at_the_hit():
    """A tube along x whose top passes through the centre of voxel (5, 8, 4),
    seen from above through that centre: the opaque hit lies on the centre, so
    the colour is the tangent colour (1, 0, 0) times that voxel's shading; a hit
    on the face between two voxel centres gets the mean of the two."""
    r = 0.5
    zc = 4.5 - r
    xyz = np.array([[2.0, 8.5, zc], [12.0, 8.5, zc], [2.0, 3.5, 1.5], [5.0, 3.5, 13.5]], np.float32)
    o = oracle.Oracle(xyz, np.array([0, 2, 4]), 16, r)
    light = (0.0, 0.0, -1.0)  # below: through the tube itself
    out = o.render(_ortho_down(5.5, 8.5), alpha=1.0, voxel_shading=1, light=light)
    assert out["first_id"][0] == 0
    assert out["first_t"][0] == pytest.approx(10 - 4.5, abs=1e-6)
    sh = o.voxel_shade(5, 8, 4, light)
    assert sh < 0.9  # the tube shadows the centre
    assert np.allclose(out["rgba"][0], (sh, 0, 0, 1), atol=1e-6)
    # the top of the end ball at x = 12 lies on the face between voxels 11 and
    # 12, whose columns below differ (tube body vs end cap)
    out = o.render(_ortho_down(12.0, 8.5), alpha=1.0, voxel_shading=1, light=light)
    assert out["first_t"][0] == pytest.approx(10 - 4.5, abs=1e-6)
    s11, s12 = o.voxel_shade(11, 8, 4, light), o.voxel_shade(12, 8, 4, light)
    assert abs(s11 - s12) > 0.01
    assert np.allclose(out["rgba"][0], (0.5 * (s11 + s12), 0, 0, 1), atol=1e-6)
    # the light from above: nothing above the tube, the centre is unshadowed
    out = o.render(_ortho_down(5.5, 8.5), alpha=1.0, voxel_shading=1, light=(0, 0, 1))
    assert np.allclose(out["rgba"][0], (1, 0, 0, 1), atol=1e-6)
    # without voxel shading the same pixel is the plain tangent colour
    assert np.allclose(o.render(_ortho_down(5.5, 8.5), alpha=1.0)["rgba"][0], (1, 0, 0, 1))


# ------------------------------------------------------------- sampled queries
def test_voxel_fragments_equal_the_list_build():
    # the per-voxel brute-force query (for sets too large for a full build)
    # against the full list build on a small set
    ls = tiny_walks(n_lines=120, n_verts=30, seed=11)
    o = oracle.Oracle.from_lineset(ls)
    L = o.lists()
    n = ls.n
    rng = np.random.default_rng(3)
    occupied = np.nonzero(L["count"])[0]
    sample = np.concatenate([rng.choice(occupied, 40, replace=False), rng.integers(0, n ** 3, 10)])
    for v in sample:
        x, y, z = int(v % n), int((v // n) % n), int(v // (n * n))
        ids, (qn, ql, qh) = o.voxel_fragments(x, y, z)
        want = L["ids"][L["start"][v]:L["start"][v + 1]]
        assert np.array_equal(ids, want), (x, y, z)
        assert (qn, ql, qh) == (L["occ_nom"][v], L["occ_lo"][v], L["occ_hi"][v])


@pytest.mark.parametrize("brute", [False, True])
def test_render_pixels_equal_render(brute):
    ls = tiny_walks(n_lines=200, n_verts=30, seed=12)
    cam = tiny_walks_camera(width=40, height=30)
    o = oracle.Oracle.from_lineset(ls)
    full = o.render(cam, alpha=0.4, brute=brute)
    pix = np.random.default_rng(5).choice(40 * 30, 60, replace=False)
    part = o.render_pixels(cam, pix, alpha=0.4, brute=brute)
    for k in ("rgba", "rgba_alt", "first_id", "first_id_alt", "first_t", "exempt"):
        assert np.array_equal(part[k], full[k][pix]), k
