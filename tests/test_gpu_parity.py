"""Parity of the CUDA path (through the C ABI) with the CPU oracle, on seeded
synthetic line sets that span many bricks, tiles and a ragged image edge.
Tolerances are stated in tests/parity.py."""
import itertools

import numpy as np
import pytest

import oracle
import paper_2510_09081_gb300 as vrt
from gen.linesets import (Camera, LineSet, random_polylines, tiny_walks, tiny_walks_camera)
from parity import RGBA_TOL, check_lists, check_words, compare_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def gpu_grid(ls, force_exact=False, occ_scale=32, max_fragments=0):
    r = vrt.Renderer(ls.n, ls.radius, occ_scale=occ_scale, max_fragments=max_fragments)
    r.upload(ls.xyz, ls.offsets)
    if force_exact:
        vrt.set_option(r.h, vrt.OPT_FORCE_EXACT, 1)
    return r


def gpu_lists(ls, cull=0, cam=None, **kw):
    r = gpu_grid(ls, **kw)
    vrt.voxelize(r.h)
    if cam is None:
        cam = tiny_walks_camera(ls.n, 16, 16)
    vrt.cull(r.h, vrt.camera_c(cam), vrt.params_c(cull=cull))
    vrt.sync(r.h)
    words = vrt.read_grid(r.h, ls.n)
    start, ln, ids = vrt.read_lists(r.h, ls.n)
    st = vrt.get_stats(r.h)
    r.close()
    return words, (start, ln, ids), st


def gpu_image(r, cam, alpha=1.0, ao=0, cull=0, k=0, voxelize=True):
    rgba, fid, ft = r.frame(cam, alpha=alpha, ao_cones=ao, cull_on=cull, k=k,
                            voxelize_first=voxelize)
    vrt.sync(r.h)
    return rgba.cpu().numpy(), fid.cpu().numpy(), ft.cpu().numpy()


def assert_image(res, max_exempt_frac=0.01):
    assert res["col_bad"] == 0, res
    assert res["id_bad"] == 0, res
    assert res["exempt_colour"] <= max_exempt_frac * res["n"], res
    assert res["exempt_id"] <= max_exempt_frac * res["n"], res
    # depth of the first hit: fp32 vs fp64; grazing entries are ill-conditioned
    assert res["max_t_rel"] < 2e-4, res


# ----------------------------------------------------------------- lists
def test_tiny_walks_words_and_lists():
    ls = tiny_walks()
    o = oracle.Oracle.from_lineset(ls)
    L = o.lists()
    words, lists, st = gpu_lists(ls)
    check_words(words, L)
    check_lists(*lists, L)
    assert st["fragments"] == L["F"]
    assert st["fragments_listed"] == L["F"]
    assert st["status_bits"] == 0


def _edge_case_set():
    """Degenerate segments, one-vertex and empty polylines, lines crossing and
    running outside the grid, long segments, vertices on voxel faces."""
    rng = np.random.default_rng(5)
    pts, offs = [], [0]

    def add(line):
        line = np.asarray(line, np.float32).reshape(-1, 3)
        pts.append(line)
        offs.append(offs[-1] + line.shape[0])

    add([[5, 5, 5], [5, 5, 5], [7, 5, 5]])                 # degenerate first segment
    add([[10, 10, 10]])                                    # one vertex: no segment
    add(np.zeros((0, 3)))                                  # empty polyline
    add([[-3, 8, 8], [12, 9, 7], [35, 10, 9]])             # enters and leaves the grid
    add([[1, 1, 1], [30, 29, 28]])                          # long diagonal
    add([[8, 8, 8], [9, 8, 8], [9, 9, 8], [9, 9, 9]])       # on voxel faces / edges
    add([[20.5, 20.5, 3], [20.5, 20.5, 28]])                # axis-parallel through centres
    add([[16, 16, 16], [16.0001, 16, 16], [16, 16, 16]])    # tiny zig-zag
    for _ in range(40):
        n = int(rng.integers(2, 8))
        p = rng.uniform(-2, 34, size=3)
        line = [p]
        for _ in range(n - 1):
            p = p + rng.normal(size=3) * rng.uniform(0.0, 6.0)
            line.append(p)
        add(np.array(line))
    xyz = np.concatenate(pts, 0)
    return LineSet(xyz=xyz, offsets=np.array(offs, np.int64), n=32, radius=0.45)


@pytest.mark.parametrize("force_exact", [False, True])
def test_edge_case_lists(force_exact):
    ls = _edge_case_set()
    L = oracle.Oracle.from_lineset(ls).lists()
    words, lists, st = gpu_lists(ls, force_exact=force_exact)
    check_words(words, L)
    check_lists(*lists, L)
    if force_exact:
        assert st["exact_decisions"] > st["fragments"]


@pytest.mark.parametrize("radius", [0.05, 0.4, 1.3])
def test_random_polylines_lists(radius):
    ls = random_polylines(300, (2, 30), 32, radius, seed=int(radius * 100))
    L = oracle.Oracle.from_lineset(ls).lists()
    words, lists, _ = gpu_lists(ls)
    check_words(words, L)
    check_lists(*lists, L)


def test_filter_and_exact_paths_agree_on_ties():
    """Segments placed exactly at the list radius from voxel faces, edges and
    corners (on the 2^-14 lattice) exercise the exact fallback."""
    R = round(0.4 * 16384) + 32
    u = 1.0 / 16384
    lines = []
    for k in range(30):
        base = np.array([4.0 + k % 5 * 5, 4.0 + (k // 5) * 4, 6.0])
        off = R * u
        lines.append([base + [0, -off, 0.5], base + [3, -off, 0.5]])          # face tie
        d = off / np.sqrt(2)
        lines.append([base + [-d, -d, -3], base + [-d, -d, 3]])                # near edge
        lines.append([base + [0.5, 1 + off, 0.2], base + [0.5, 1 + off, 0.8]])  # face tie
    xyz = np.array(lines, np.float32).reshape(-1, 3)
    ls = LineSet(xyz=xyz, offsets=np.arange(0, xyz.shape[0] + 1, 2), n=32, radius=0.4)
    L = oracle.Oracle.from_lineset(ls).lists()
    w0, l0, st0 = gpu_lists(ls)
    w1, l1, _ = gpu_lists(ls, force_exact=True)
    check_lists(*l0, L)
    check_lists(*l1, L)
    assert st0["exact_decisions"] > 0


# ----------------------------------------------------------------- images
def _persp_cam(n=64, w=157, h=93):
    return Camera(width=w, height=h, ortho=0, eye=(n * 1.6, n * 1.3, n * 0.9),
                  target=(n / 2, n / 2, n / 2), up=(0, 0, 1), fovy_deg=45.0)


def test_tiny_walks_opaque_ortho():
    ls = tiny_walks()
    o = oracle.Oracle.from_lineset(ls)
    cam = tiny_walks_camera()
    ref = o.render(cam, alpha=1.0)
    r = gpu_grid(ls)
    res = compare_image(*gpu_image(r, cam), ref)
    r.close()
    assert res["hits"] > 50000
    assert_image(res)


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.3, 0.1])
def test_perspective_images(alpha):
    ls = tiny_walks(n_lines=600, n_verts=40, seed=123)
    o = oracle.Oracle.from_lineset(ls)
    cam = _persp_cam()
    ref = o.render(cam, alpha=alpha)
    r = gpu_grid(ls)
    res = compare_image(*gpu_image(r, cam, alpha=alpha), ref)
    r.close()
    assert res["hits"] > 2000
    assert_image(res)


def test_k_buffer_size_does_not_change_the_image():
    ls = tiny_walks(n_lines=600, n_verts=40, seed=123)
    cam = _persp_cam()
    r = gpu_grid(ls)
    outs = [gpu_image(r, cam, alpha=0.2, k=k) for k in (8, 16, 32)]
    r.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("alpha", [1.0, 0.3])
def test_culling_never_changes_the_image(alpha):
    ls = tiny_walks(n_lines=3000, n_verts=60, seed=9)
    cam = _persp_cam(w=211, h=117)
    r = gpu_grid(ls)
    off = gpu_image(r, cam, alpha=alpha, cull=0)
    on = gpu_image(r, cam, alpha=alpha, cull=1)
    st = vrt.get_stats(r.h)
    r.close()
    for a, b in zip(off, on):
        assert np.array_equal(a, b)
    assert st["visible_voxels"] < st["occupied_voxels"]


def test_automatic_culling():
    # cull = 2: the image is that of cull = 0 in every frame; a set the cull
    # keeps almost entirely stops being culled after its first culled frame
    ls = tiny_walks(n_lines=3000, n_verts=60, seed=9)
    cam = _persp_cam(w=211, h=117)
    r = gpu_grid(ls)
    off = gpu_image(r, cam, alpha=0.3, cull=0)
    vis = []
    for f in range(4):
        img = gpu_image(r, cam, alpha=0.3, cull=2)
        st = vrt.get_stats(r.h)
        vis.append((st["visible_voxels"], st["occupied_voxels"]))
        for a, b in zip(off, img):
            assert np.array_equal(a, b)
    r.close()
    frac = vis[0][0] / vis[0][1]
    if frac > 0.95:   # kept almost everything: later builds skip the cull
        assert all(v == o for v, o in vis[1:])
    else:             # culling pays: every build culls
        assert all(v < o for v, o in vis)
    # a sparse set in front of the camera keeps everything visible
    sp = tiny_walks(n_lines=40, n_verts=30, seed=10)
    r = gpu_grid(sp)
    gpu_image(r, cam, alpha=0.3, cull=2)
    st0 = vrt.get_stats(r.h)
    gpu_image(r, cam, alpha=0.3, cull=2)
    st1 = vrt.get_stats(r.h)
    r.close()
    assert st0["visible_voxels"] / st0["occupied_voxels"] > 0.95
    assert st1["visible_voxels"] == st1["occupied_voxels"]


def test_mips_match_oracle():
    ls = tiny_walks(n_lines=800, n_verts=50, n=64, seed=3)
    o = oracle.Oracle.from_lineset(ls)
    L = o.lists()
    ref = o.mips()
    r = gpu_grid(ls)
    vrt.voxelize(r.h)
    vrt.build_mips(r.h)
    got = vrt.read_mips(r.h, 64)
    r.close()
    # a near-tie occupancy code may differ by one step: bound its effect per level
    bound = ((L["occ_hi"].astype(np.float64) - L["occ_lo"]) / 32.0).reshape(64, 64, 64)
    for lvl, (g, f) in enumerate(zip(got, ref)):
        assert g.shape == f.shape
        assert np.all(np.abs(g - f) <= bound + 1e-6), lvl
        m = bound.shape[0] // 2
        if m >= 1:
            bound = bound.reshape(m, 2, m, 2, m, 2).mean(axis=(1, 3, 5))


@pytest.mark.parametrize("alpha", [1.0, 0.4])
def test_ambient_occlusion_images(alpha):
    ls = tiny_walks(n_lines=1500, n_verts=60, n=32, radius=0.6, seed=17, start_lo=4.0,
                    start_hi=28.0)
    o = oracle.Oracle.from_lineset(ls)
    cam = Camera(width=96, height=80, ortho=0, eye=(16.0, 16.0, 16.0), target=(40.0, 30.0, 20.0),
                 up=(0, 0, 1), fovy_deg=60.0)
    ref = o.render(cam, alpha=alpha, ao_cones=6)
    r = gpu_grid(ls)
    res = compare_image(*gpu_image(r, cam, alpha=alpha, ao=6, cull=1), ref)
    r.close()
    assert res["hits"] > 1000
    assert_image(res, max_exempt_frac=0.02)


# --------------------------------------- reduced-precision pyramid (FP16/BF16)
# Each level is averaged in fp32 from its stored children and rounded once, so
# level l of the stored pyramid lies within (l + 1) half-ulps of 1 (2^-12 for
# fp16, 2^-9 for bf16; all texels are in [0, 1]) of the fp64 pyramid, beyond
# the fp32 near-tie allowance. An AO sample is a convex combination of texels,
# a cone's factor a product of four (1 - sample) terms in [0, 1] and AO their
# mean, so a texel error e moves AO, and the composited colour, by at most 4 e.
HALF_ULP = {vrt.MIPS_F16: 2.0 ** -12, vrt.MIPS_BF16: 2.0 ** -9}


def _abc_small():
    # the ABC flow at 1/64 of the benchmark's lines in a 128^3 grid: partial
    # occlusion, so AO samples are neither 0 nor 1 and texels are not short
    # binary fractions
    from gen.linesets import abc_pathlines, abc_camera
    return (abc_pathlines(n_particles=15_625, n=128, frame=0),
            abc_camera(n=128, frame=0, width=320, height=180))


@pytest.mark.parametrize("fmt", [vrt.MIPS_F16, vrt.MIPS_BF16])
def test_reduced_precision_mips_match_oracle(fmt):
    ls, _ = _abc_small()
    n = ls.n
    o = oracle.Oracle.from_lineset(ls)
    L = o.lists()
    ref = o.mips()
    r = gpu_grid(ls)
    vrt.set_option(r.h, vrt.OPT_MIPS_FORMAT, fmt)
    vrt.voxelize(r.h)
    vrt.build_mips(r.h)
    got = vrt.read_mips(r.h, n)
    r.close()
    bound = ((L["occ_hi"].astype(np.float64) - L["occ_lo"]) / 32.0).reshape(n, n, n)
    worst = []
    for lvl, (g, f) in enumerate(zip(got, ref)):
        err = np.abs(g - f) - bound
        worst.append(float(err.max()))
        assert err.max() <= (lvl + 1) * HALF_ULP[fmt] + 1e-6, (lvl, float(err.max()))
        m = bound.shape[0] // 2
        if m >= 1:
            bound = bound.reshape(m, 2, m, 2, m, 2).mean(axis=(1, 3, 5))
    assert max(worst) > 0.0  # the rounding is exercised
    print(f"fmt {fmt}: max texel error per level {['%.1e' % w for w in worst]}")


@pytest.mark.parametrize("fmt", [vrt.MIPS_F32, vrt.MIPS_F16, vrt.MIPS_BF16])
def test_reduced_precision_ao_images(fmt):
    ls, cam = _abc_small()
    o = oracle.Oracle.from_lineset(ls)
    pix = np.random.default_rng(9).choice(cam.width * cam.height, 1500, replace=False)
    ref = o.render_pixels(cam, pix, alpha=1.0, ao_cones=6)
    r = gpu_grid(ls)
    vrt.set_option(r.h, vrt.OPT_MIPS_FORMAT, fmt)
    rgba, fid, ft = gpu_image(r, cam, alpha=1.0, ao=6, cull=1)
    r.close()
    rgba, fid, ft = rgba.reshape(-1, 4)[pix], fid.reshape(-1)[pix], ft.reshape(-1)[pix]
    levels = 6  # cone samples read levels 0..5 (diameter <= 2 * 9.5 * tan(half angle) < 32)
    tol = RGBA_TOL + (4 * levels * HALF_ULP[fmt] if fmt != vrt.MIPS_F32 else 0.0)
    res = compare_image(rgba, fid, ft, ref, tol=tol)
    assert res["hits"] > 1000
    assert_image(res, max_exempt_frac=0.02)
    # the error actually seen, against the primary fp64 result
    ok = ((ref["exempt"] & 1) == 0) & (fid >= 0)
    d = np.abs(rgba - ref["rgba"]).max(1)[ok]
    print(f"fmt {fmt}: RGBA error vs fp64 oracle over {ok.sum()} hit pixels: "
          f"mean {d.mean():.2e} max {d.max():.2e} (bound {tol:.1e})")


# ------------------------------------------------------------ dynamic data
def test_update_vertices_equals_fresh_upload():
    ls = tiny_walks(n_lines=500, n_verts=50, seed=1)
    ls2 = tiny_walks(n_lines=500, n_verts=50, seed=2)
    new = ls.xyz.copy()
    new[5000:9000] = ls2.xyz[5000:9000]
    r = gpu_grid(ls)
    vrt.voxelize(r.h)
    vrt.update_vertices(r.h, 5000, torch.from_numpy(ls2.xyz[5000:9000]).cuda())
    vrt.voxelize(r.h)
    vrt.sync(r.h)
    w_upd = vrt.read_grid(r.h, 64)
    # only the updated vertices and their neighbours are ingested again: the
    # frame equals one from a fresh upload of the new vertices, bitwise
    cam = _persp_cam()
    img_upd = gpu_image(r, cam, alpha=0.3, voxelize=False)
    r.close()
    fresh = LineSet(xyz=new, offsets=ls.offsets, n=64, radius=ls.radius)
    r2 = gpu_grid(fresh)
    img_fresh = gpu_image(r2, cam, alpha=0.3)
    r2.close()
    for a, b in zip(img_upd, img_fresh):
        assert np.array_equal(a, b)
    L = oracle.Oracle.from_lineset(fresh).lists()
    check_words(w_upd, L)


def test_device_stride4_upload_matches_host():
    ls = tiny_walks(n_lines=300, n_verts=30, seed=4)
    x4 = np.concatenate([ls.xyz, np.full((ls.n_vertices, 1), 7.0, np.float32)], 1)
    r = vrt.Renderer(64, ls.radius)
    r.upload(torch.from_numpy(x4).cuda(), ls.offsets)
    vrt.voxelize(r.h)
    vrt.sync(r.h)
    w = vrt.read_grid(r.h, 64)
    r.close()
    check_words(w, oracle.Oracle.from_lineset(ls).lists())


# ------------------------------------------------------------------ errors
def test_error_reporting():
    ls = tiny_walks(n_lines=50, n_verts=20, seed=6)
    bad = ls.xyz.copy()
    bad[3, 1] = 900.0
    r = vrt.Renderer(64, 0.4)
    with pytest.raises(vrt.VrtError) as e:
        r.upload(bad, ls.offsets)
    assert e.value.status == vrt.ERR_INVALID_ARG
    # device input out of range: reported at sync
    r.upload(torch.from_numpy(bad).cuda(), ls.offsets)
    vrt.voxelize(r.h)
    with pytest.raises(vrt.VrtError) as e:
        vrt.sync(r.h)
    assert e.value.status == vrt.ERR_INVALID_ARG
    vrt.sync(r.h)  # cleared
    # a host update out of range: checked on the device, reported at sync
    r.upload(ls.xyz, ls.offsets)
    vrt.update_vertices(r.h, 0, np.ascontiguousarray(bad[:10]))
    vrt.voxelize(r.h)
    with pytest.raises(vrt.VrtError) as e:
        vrt.sync(r.h)
    assert e.value.status == vrt.ERR_INVALID_ARG
    vrt.sync(r.h)  # cleared
    # trace before the list build
    r.upload(ls.xyz, ls.offsets)
    rgba = torch.zeros((4, 4, 4), device="cuda")
    with pytest.raises(vrt.VrtError) as e:
        vrt.trace(r.h, tiny_walks_camera(64, 4, 4), vrt.params_c(), rgba)
    assert e.value.status == vrt.ERR_STATE
    r.close()


def test_overflow_is_detected():
    # occupancy field: 2000 coincident segments at scale 65535 wrap 16 bits
    xyz = np.tile(np.array([[10.5, 10.5, 10.2], [10.5, 10.5, 10.8]], np.float32), (2000, 1))
    ls = LineSet(xyz=xyz, offsets=np.arange(0, 4001, 2), n=32, radius=0.5)
    r = gpu_grid(ls, occ_scale=65535)
    vrt.voxelize(r.h)
    vrt.cull(r.h, vrt.camera_c(tiny_walks_camera(32, 8, 8)), vrt.params_c())
    with pytest.raises(vrt.VrtError) as e:
        vrt.sync(r.h)
    assert e.value.status == vrt.ERR_OVERFLOW
    r.close()
    # list capacity
    ls = tiny_walks(n_lines=100, n_verts=20, seed=8)
    r = gpu_grid(ls, max_fragments=1000)
    vrt.voxelize(r.h)
    vrt.cull(r.h, vrt.camera_c(tiny_walks_camera(64, 8, 8)), vrt.params_c())
    with pytest.raises(vrt.VrtError) as e:
        vrt.sync(r.h)
    assert e.value.status == vrt.ERR_OVERFLOW
    r.close()


# ------------------------------------------------ voxel-space shading (Sec. 3.4)
LIGHT = (0.3, -0.5, 0.8)


def _dilate(m):
    """Voxels within one step (26-neighbourhood) of a set voxel."""
    n = m.shape[0]
    p = np.pad(m, 1)
    out = np.zeros_like(m)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out |= p[dz:dz + n, dy:dy + n, dx:dx + n]
    return out


def _shadow_spread(spread, x, y, z, light):
    """Bound on how far the shadow transmittance from the centre of (x, y, z)
    can move when the level-0 texels move within `spread` ([z, y, x]): each
    sample is a convex combination of texels, so it moves by at most the
    weighted spread of its texels, and a product of factors in [0, 1] by at
    most the sum of its factors' moves."""
    n = spread.shape[0]
    L = np.asarray(light, np.float64) / np.linalg.norm(light)
    P = np.array([x, y, z], np.float64) + 0.5
    k = np.arange(1, int(np.sqrt(3.0) * (n + 1)) + 3, dtype=np.float64)[:, None]
    q = P + k * L
    inside = np.all((q >= -0.5) & (q <= n + 0.5), axis=1)
    q = q[:np.argmin(inside) if not inside.all() else len(q)]  # the march ends at the first outside
    u = q - 0.5
    b = np.floor(u).astype(np.int64)
    f = u - b
    tot = 0.0
    for d in itertools.product((0, 1), repeat=3):
        c = b + np.array(d)
        ok = np.all((c >= 0) & (c < n), axis=1)
        w = np.prod(np.where(np.array(d)[None, :] == 1, f, 1.0 - f), axis=1)
        cc = np.clip(c, 0, n - 1)
        tot += float((w * ok * spread[cc[:, 2], cc[:, 1], cc[:, 0]]).sum())
    return tot


def test_voxel_shading_field_matches_oracle():
    ls, cam = _abc_small()
    n = ls.n
    o = oracle.Oracle.from_lineset(ls)
    L = o.lists()
    # a near-tie occupancy code may come out one step either way in fp32
    spread = ((L["occ_hi"].astype(np.float64) - L["occ_lo"]) / 32.0).reshape(n, n, n)
    r = gpu_grid(ls)
    fields = {}
    for ao in (0, 6):
        r.frame(cam, alpha=0.4, ao_cones=ao, cull_on=1, voxel_shading=1, light=LIGHT)
        vrt.sync(r.h)
        fields[ao] = vrt.read_shading(r.h, n)
    start, ln, _ = vrt.read_lists(r.h, n)
    st = vrt.get_stats(r.h)
    r.close()
    listed = (ln > 0).reshape(n, n, n)
    assert listed.sum() < st["occupied_voxels"]  # the cull dropped voxels
    for ao in (0, 6):
        assert np.array_equal(fields[ao][1], _dilate(listed))
    vals0, valid = fields[0]
    vals6 = fields[6][0]
    idx = np.argwhere(valid)
    rng = np.random.default_rng(4)
    pick = idx[rng.choice(idx.shape[0], min(400, idx.shape[0]), replace=False)]
    worst, worst_ao, widened = 0.0, 0.0, 0
    for z, y, x in pick:
        # shadow only: 1/2 + S/2, within the early stop (5e-5), fp32 rounding
        # and the near-tie bound
        ref = o.voxel_shade(x, y, z, LIGHT, ao_cones=0)
        b = 0.5 * _shadow_spread(spread, x, y, z, LIGHT)
        widened += b > 0
        err = abs(float(vals0[z, y, x]) - ref)
        assert err <= 2e-4 + b, (x, y, z, float(vals0[z, y, x]), ref, b)
        if b == 0:
            worst = max(worst, err)
        # with AO: the ratio is the cone AO at the voxel centre (tolerance of
        # the per-hit AO images)
        ao_ref = o.ao((x + 0.5, y + 0.5, z + 0.5))
        e_ao = abs(float(vals6[z, y, x]) / float(vals0[z, y, x]) - ao_ref)
        assert e_ao <= RGBA_TOL, (x, y, z, e_ao)
        worst_ao = max(worst_ao, e_ao)
    assert vals0[valid].min() < 0.6 and vals0[valid].max() > 0.99  # shadows and light both occur
    ao_seen = vals6[valid] / vals0[valid]
    assert ao_seen.min() < 0.3 and ao_seen.max() > 0.7  # AO is partial, neither 0 nor 1
    print(f"voxel shading field: {len(pick)} voxels, shadow worst error {worst:.2e} where no "
          f"near-tie code is read ({widened} with a widened bound), AO worst error {worst_ao:.2e}")


@pytest.mark.parametrize("alpha", [1.0, 0.4])
def test_voxel_shading_images(alpha):
    ls, cam = _abc_small()
    o = oracle.Oracle.from_lineset(ls)
    pix = np.random.default_rng(11).choice(cam.width * cam.height, 1500, replace=False)
    ref = o.render_pixels(cam, pix, alpha=alpha, ao_cones=6, voxel_shading=1, light=LIGHT)
    r = gpu_grid(ls)
    rgba, fid, ft = gpu_image_vs(r, cam, alpha)
    per_hit = gpu_image(r, cam, alpha=alpha, ao=6, cull=1)[0]
    r.close()
    res = compare_image(rgba.reshape(-1, 4)[pix], fid.reshape(-1)[pix], ft.reshape(-1)[pix], ref)
    assert res["hits"] > 1000
    assert_image(res, max_exempt_frac=0.02)
    # the field (AO at voxel centres, and the shadow) is not the per-hit AO
    assert np.abs(rgba - per_hit).max() > 0.05
    ok = ((ref["exempt"] & 1) == 0) & (fid.reshape(-1)[pix] >= 0)
    d = np.abs(rgba.reshape(-1, 4)[pix] - ref["rgba"]).max(1)[ok]
    print(f"voxel shading alpha {alpha}: RGBA error vs fp64 oracle over {ok.sum()} hit pixels: "
          f"mean {d.mean():.2e} max {d.max():.2e}")


def gpu_image_vs(r, cam, alpha, light=LIGHT, cull=1, ao=6):
    rgba, fid, ft = r.frame(cam, alpha=alpha, ao_cones=ao, cull_on=cull, voxel_shading=1, light=light)
    vrt.sync(r.h)
    return rgba.cpu().numpy().copy(), fid.cpu().numpy().copy(), ft.cpu().numpy().copy()


@pytest.mark.parametrize("alpha", [1.0, 0.3])
def test_voxel_shading_culling_never_changes_the_image(alpha):
    # culling lists fewer voxels, so fewer get shaded; every voxel a hit
    # samples is still computed (repair rounds extend the field), and with the
    # same values, so the images are equal bitwise
    ls = tiny_walks(n_lines=3000, n_verts=60, seed=9)
    cam = _persp_cam(w=211, h=117)
    r = gpu_grid(ls)
    off = gpu_image_vs(r, cam, alpha, light=(-0.2, 0.9, 0.4), cull=0, ao=6)
    on = gpu_image_vs(r, cam, alpha, light=(-0.2, 0.9, 0.4), cull=1, ao=6)
    # a much lower cull threshold: voxels rays reach are culled, listed and
    # shaded by the repair rounds
    vrt.set_option(r.h, vrt.OPT_CULL_DEPTH, 300)
    rep = gpu_image_vs(r, cam, alpha, light=(-0.2, 0.9, 0.4), cull=1, ao=6)
    st = vrt.get_stats(r.h)
    r.close()
    for a, b, c in zip(off, on, rep):
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    assert st["repaired_voxels"] > 100 and st["repair_rounds"] >= 1, st
    print(f"repaired voxels {st['repaired_voxels']}, rounds {st['repair_rounds']}")


@pytest.mark.parametrize("alpha", [1.0, 0.3])
def test_aggressive_culling_is_repaired(alpha):
    # repair with resume under a cull that drops voxels rays need: the image is
    # that of no culling, bitwise
    ls = tiny_walks(n_lines=3000, n_verts=60, seed=9)
    cam = _persp_cam(w=211, h=117)
    r = gpu_grid(ls)
    off = gpu_image(r, cam, alpha=alpha, cull=0)
    vrt.set_option(r.h, vrt.OPT_CULL_DEPTH, 300)
    on = gpu_image(r, cam, alpha=alpha, cull=1)
    st = vrt.get_stats(r.h)
    r.close()
    for a, b in zip(off, on):
        assert np.array_equal(a, b)
    assert st["repaired_voxels"] > 100 and st["retraced_pixels"] > 100, st
    print(f"alpha {alpha}: repaired voxels {st['repaired_voxels']}, rounds {st['repair_rounds']}, "
          f"re-traced pixels {st['retraced_pixels']}")


def test_voxel_shading_argument_errors():
    ls = tiny_walks(n_lines=50, n_verts=20, n=32, seed=2)
    cam = _persp_cam(n=32, w=32, h=24)
    r = gpu_grid(ls)
    vrt.voxelize(r.h)
    c = vrt.camera_c(cam)
    rgba = torch.zeros((24, 32, 4), device="cuda")
    vrt.cull(r.h, c, vrt.params_c(alpha=1.0))
    with pytest.raises(vrt.VrtError) as e:  # the pyramid is needed
        vrt.trace(r.h, c, vrt.params_c(alpha=1.0, voxel_shading=1), rgba)
    assert e.value.status == vrt.ERR_STATE
    vrt.build_mips(r.h)
    for bad in (dict(voxel_shading=2), dict(voxel_shading=1, light=(0.0, 0.0, 0.0)),
                dict(voxel_shading=1, light=(float("nan"), 0.0, 1.0))):
        with pytest.raises(vrt.VrtError) as e:
            vrt.trace(r.h, c, vrt.params_c(alpha=1.0, **bad), rgba)
        assert e.value.status == vrt.ERR_INVALID_ARG
    with pytest.raises(vrt.VrtError) as e:
        vrt.read_shading(r.h, 32)
    assert e.value.status == vrt.ERR_STATE
    vrt.trace(r.h, c, vrt.params_c(alpha=1.0, voxel_shading=1), rgba)
    vrt.sync(r.h)
    r.close()


def _orbit(cam, deg):
    """The camera turned by deg about the vertical axis through its target."""
    a = np.deg2rad(deg)
    e = np.array(cam.eye) - np.array(cam.target)
    e = np.array([e[0] * np.cos(a) - e[1] * np.sin(a), e[0] * np.sin(a) + e[1] * np.cos(a), e[2]])
    return Camera(width=cam.width, height=cam.height, ortho=cam.ortho,
                  eye=tuple(map(float, np.array(cam.target) + e)), target=cam.target, up=cam.up,
                  fovy_deg=cam.fovy_deg, ortho_h=cam.ortho_h)


@pytest.mark.parametrize("voxel_shading", [0, 1])
def test_static_scene_trace_only_frames(voxel_shading):
    # a static set is voxelized and listed once; each later frame only traces
    # (Sec. 4): from any camera the image equals a full frame's, and the
    # voxel-space field is reused rather than recomputed
    ls = tiny_walks(n_lines=1500, n_verts=60, seed=21)
    cam0 = _persp_cam(w=160, h=96)
    kw = dict(alpha=0.4, ao_cones=6, cull_on=0, voxel_shading=voxel_shading, light=LIGHT)
    r = gpu_grid(ls)
    r.frame(cam0, **kw)
    vrt.sync(r.h)
    got, launches = [], []
    for deg in (0, 25, 70, 160):
        l0 = vrt.get_stats(r.h)["kernel_launches"]
        rgba, fid, ft = r.trace_only(_orbit(cam0, deg), alpha=0.4, ao_cones=6,
                                     voxel_shading=voxel_shading, light=LIGHT)
        vrt.sync(r.h)
        launches.append(vrt.get_stats(r.h)["kernel_launches"] - l0)
        got.append((rgba.cpu().numpy().copy(), fid.cpu().numpy().copy(), ft.cpu().numpy().copy()))
    r.close()
    for deg, g in zip((0, 25, 70, 160), got):
        f = gpu_grid(ls)
        ref = f.frame(_orbit(cam0, deg), **kw)
        vrt.sync(f.h)
        for a, b in zip(g, ref):
            assert np.array_equal(a, b.cpu().numpy())
        f.close()
    assert not np.array_equal(got[0][0], got[2][0])
    # one trace launch per frame: no list build, and the field is reused
    assert launches == [1, 1, 1, 1], launches
