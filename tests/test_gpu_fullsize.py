"""Parity at the benchmark's full size: the tractography-like bundles frame
(100k streamlines x 100 vertices = 9.9M segments, 256^3 grid, 1920x1080
perspective, opacity 0.3, culling on), run through the C ABI in the launch
configuration the benchmark times. The oracle cannot build the whole frame in
a test's time, so it checks sampled outputs one by one, each by brute force over
every segment:

  * sampled voxels: count (exact), occupancy code sum (within the oracle's
    near-tie range), and, for voxels that received a list, the list itself
    (bit-exact as a set);
  * sampled pixels: RGBA, first-hit id and depth, with the tolerances and
    near-tie rules of tests/parity.py;

and a property that holds at any size: culling never changes the image (bitwise).
Tolerances are stated in tests/parity.py."""
import os

import numpy as np
import pytest

import oracle
import paper_2510_09081_gb300 as vrt
from gen import linesets as G
from parity import compare_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def frame():
    bs = G.bundles(n_lines=100_000)
    ls = bs.lineset
    cam = G.bundles_camera()
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(torch.from_numpy(ls.xyz).cuda(), ls.offsets)
    rgba, fid, ft = r.frame(cam, alpha=0.3, cull_on=1)
    vrt.sync(r.h)
    out = dict(ls=ls, cam=cam, r=r,
               rgba=rgba.cpu().numpy().reshape(-1, 4).copy(),
               fid=fid.cpu().numpy().reshape(-1).copy(),
               ft=ft.cpu().numpy().reshape(-1).copy(),
               words=vrt.read_grid(r.h, ls.n),
               stats=vrt.get_stats(r.h))
    out["start"], out["len"], out["ids"] = vrt.read_lists(r.h, ls.n)
    out["oracle"] = oracle.Oracle.from_lineset(ls, nthreads=os.cpu_count() or 1)
    yield out
    r.close()
    out["oracle"].close()


def test_fullsize_sampled_voxels(frame):
    ls, o = frame["ls"], frame["oracle"]
    n = ls.n
    rng = np.random.default_rng(20251009)
    # voxels at the midpoints of random segments (mostly occupied), plus
    # uniformly random voxels
    seg = rng.choice(ls.n_vertices - 1, 160, replace=False)
    ok = np.diff(np.searchsorted(ls.offsets, [seg, seg + 1], side="right"), axis=0)[0] == 0
    mid = 0.5 * (ls.xyz[seg[ok]] + ls.xyz[seg[ok] + 1])
    vox = np.clip(np.floor(mid).astype(np.int64), 0, n - 1)[:48]
    vox = np.concatenate([vox, rng.integers(0, n, (16, 3))])
    listed = checked = 0
    for x, y, z in vox:
        ids, (_, lo, hi) = o.voxel_fragments(x, y, z)
        v = (z * n + y) * n + x
        w = int(frame["words"][v])
        assert (w & 0xFFFF) == ids.shape[0], (x, y, z)
        assert lo <= (w >> 16) <= hi, (x, y, z, w >> 16, lo, hi)
        checked += 1
        ln = int(frame["len"][v])
        if ln:
            assert ln == ids.shape[0], (x, y, z)
            s = int(frame["start"][v])
            assert np.array_equal(np.sort(frame["ids"][s:s + ln]), ids), (x, y, z)
            listed += 1
    assert checked == vox.shape[0] and listed >= 30


def test_fullsize_sampled_pixels(frame):
    cam, o = frame["cam"], frame["oracle"]
    npx = cam.width * cam.height
    # random pixels and a 16 x 8 block at the image centre (dense bundles)
    cy, cx = cam.height // 2, cam.width // 2
    block = ((cy - 4 + np.arange(8))[:, None] * cam.width + (cx - 8 + np.arange(16))[None, :]).ravel()
    pix = np.unique(np.concatenate([np.random.default_rng(7).choice(npx, 320, replace=False), block]))
    ref = o.render_pixels(cam, pix, alpha=0.3, brute=True)
    res = compare_image(frame["rgba"][pix], frame["fid"][pix], frame["ft"][pix], ref)
    assert res["col_bad"] == 0, res
    assert res["id_bad"] == 0, res
    assert res["exempt_colour"] <= 0.01 * res["n"] and res["exempt_id"] <= 0.01 * res["n"], res
    assert res["max_t_rel"] < 2e-4, res
    assert res["hits"] >= 100, res


def test_fullsize_paper_hit_key(frame):
    """The paper's 16+16-bit per-voxel hit key on the full frame: hits whose
    depths fall into the same 1/65536 of a voxel's ray interval follow the
    list's (arbitrary) order instead of their exact depths. Counted against the
    default (depth, id) key over the whole image, and checked against the
    oracle's ground truth on the sampled pixels."""
    cam, r, o = frame["cam"], frame["r"], frame["oracle"]
    vrt.set_option(r.h, vrt.OPT_HIT_KEY, vrt.HIT_KEY_16_16)
    try:
        rgba, fid, ft = r.frame(cam, alpha=0.3, cull_on=1, voxelize_first=False)
        vrt.sync(r.h)
    finally:
        vrt.set_option(r.h, vrt.OPT_HIT_KEY, vrt.HIT_KEY_DEPTH_ID)
    rgba = rgba.cpu().numpy().reshape(-1, 4)
    fid = fid.cpu().numpy().reshape(-1)
    ft = ft.cpu().numpy().reshape(-1)
    npx = cam.width * cam.height
    d = np.abs(rgba - frame["rgba"]).max(1)
    changed = int((d > 0).sum())
    print(f"16+16 key: {changed} of {npx} pixels differ from the (depth, id) key, max "
          f"|dRGBA| {d.max():.2e}; first ids differ at {int((fid != frame['fid']).sum())}")
    assert changed <= 1e-3 * npx
    cy, cx = cam.height // 2, cam.width // 2
    block = ((cy - 4 + np.arange(8))[:, None] * cam.width + (cx - 8 + np.arange(16))[None, :]).ravel()
    pix = np.unique(np.concatenate([np.random.default_rng(7).choice(npx, 320, replace=False), block]))
    ref = o.render_pixels(cam, pix, alpha=0.3, brute=True)
    res = compare_image(rgba[pix], fid[pix], ft[pix], ref)
    assert res["col_bad"] == 0 and res["id_bad"] == 0, res
    assert res["max_t_rel"] < 2e-4, res


def test_fullsize_culling_never_changes_the_image(frame):
    cam, r = frame["cam"], frame["r"]
    rgba, fid, ft = r.frame(cam, alpha=0.3, cull_on=0, voxelize_first=False)
    vrt.sync(r.h)
    assert np.array_equal(rgba.cpu().numpy().reshape(-1, 4), frame["rgba"])
    assert np.array_equal(fid.cpu().numpy().reshape(-1), frame["fid"])
    assert np.array_equal(ft.cpu().numpy().reshape(-1), frame["ft"])
    st = frame["stats"]
    assert st["visible_voxels"] < st["occupied_voxels"]
    assert st["repaired_voxels"] >= 0


def _dilate(m):
    n = m.shape[0]
    p = np.pad(m, 1)
    out = np.zeros_like(m)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out |= p[dz:dz + n, dy:dy + n, dx:dx + n]
    return out


def test_fullsize_voxel_shading_properties(frame):
    # voxel-space shading without AO: every hit's factor is 1/2 + S/2 in
    # [1/2, 1], so against the unshaded frame the first hits, depths and
    # alpha are unchanged and each colour channel lies in [C/2, C]; the field
    # covers exactly the listed voxels' neighbourhoods; culling (with repair)
    # leaves the shaded image unchanged, bitwise
    ls, cam, r = frame["ls"], frame["cam"], frame["r"]
    light = (0.4, 0.5, 0.77)
    out = []
    for cull in (1, 0):
        rgba, fid, ft = r.frame(cam, alpha=0.3, cull_on=cull, voxel_shading=1, light=light)
        vrt.sync(r.h)
        out.append((rgba.cpu().numpy().reshape(-1, 4).copy(), fid.cpu().numpy().reshape(-1).copy(),
                    ft.cpu().numpy().reshape(-1).copy()))
        if cull == 1:
            _, valid = vrt.read_shading(r.h, ls.n)
            _, ln, _ = vrt.read_lists(r.h, ls.n)
            assert np.array_equal(valid, _dilate((ln > 0).reshape(ls.n, ls.n, ls.n)))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    rgba, fid, ft = out[0]
    assert np.array_equal(fid, frame["fid"]) and np.array_equal(ft, frame["ft"])
    assert np.array_equal(rgba[:, 3], frame["rgba"][:, 3])
    c0 = frame["rgba"][:, :3]
    assert (rgba[:, :3] <= c0 + 1e-6).all() and (rgba[:, :3] >= 0.5 * c0 - 1e-6).all()
    hit = fid >= 0
    assert (rgba[hit, :3].sum(1) < 0.95 * c0[hit].sum(1)).mean() > 0.2  # shadows are seen


# --------------------------------------------------------------------------
# Unsteady-flow pathlines: 1M particles x 32 vertices (31M segments) in the ABC
# flow, 512^3 grid, radius 0.25, 1920x1080 from inside the domain, opaque,
# six-cone AO, culling on. The oracle checks sampled voxels and, without AO,
# sampled pixels by brute force; AO is checked against the oracle on the same
# flow at 1/64 of the lines in a 128^3 grid (the same line density per voxel),
# and at full size by properties: it leaves the first hits unchanged and only
# darkens the colour.
@pytest.fixture(scope="module")
def abc_frame():
    ls = G.abc_pathlines(frame=0)
    cam = G.abc_camera(frame=0)
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(torch.from_numpy(ls.xyz).cuda(), ls.offsets)
    out = dict(ls=ls, cam=cam, r=r)
    rgba, fid, ft = r.frame(cam, alpha=1.0, ao_cones=6, cull_on=1)
    vrt.sync(r.h)
    out["ao"] = (rgba.cpu().numpy().reshape(-1, 4).copy(), fid.cpu().numpy().reshape(-1).copy(),
                 ft.cpu().numpy().reshape(-1).copy())
    out["words"] = vrt.read_grid(r.h, ls.n)
    out["start"], out["len"], out["ids"] = vrt.read_lists(r.h, ls.n)
    rgba, fid, ft = r.frame(cam, alpha=1.0, ao_cones=0, cull_on=1, voxelize_first=False)
    vrt.sync(r.h)
    out["plain"] = (rgba.cpu().numpy().reshape(-1, 4).copy(), fid.cpu().numpy().reshape(-1).copy(),
                    ft.cpu().numpy().reshape(-1).copy())
    out["oracle"] = oracle.Oracle.from_lineset(ls, nthreads=os.cpu_count() or 1)
    yield out
    r.close()
    out["oracle"].close()


def test_abc_fullsize_sampled_voxels(abc_frame):
    ls, o = abc_frame["ls"], abc_frame["oracle"]
    n = ls.n
    rng = np.random.default_rng(20251011)
    seg = rng.choice(ls.n_vertices - 1, 96, replace=False)
    ok = np.diff(np.searchsorted(ls.offsets, [seg, seg + 1], side="right"), axis=0)[0] == 0
    mid = 0.5 * (ls.xyz[seg[ok]] + ls.xyz[seg[ok] + 1])
    vox = np.clip(np.floor(mid).astype(np.int64), 0, n - 1)[:32]
    # most voxels are hidden from the camera inside the flow; voxels of
    # segments just in front of the eye are seen, so they get lists
    cam = abc_frame["cam"]
    eye, f = np.array(cam.eye), np.array(cam.target) - np.array(cam.eye)
    f /= np.linalg.norm(f)
    m_all = 0.5 * (ls.xyz[:-1] + ls.xyz[1:])
    rel = m_all - eye
    near = np.nonzero((np.linalg.norm(rel, axis=1) < 6.0) & (rel @ f > 1.0))[0]
    near = near[np.diff(np.searchsorted(ls.offsets, [near, near + 1], side="right"), axis=0)[0] == 0]
    front = np.unique(np.floor(m_all[near]).astype(np.int64), axis=0)
    front = front[rng.permutation(front.shape[0])[:24]]
    vox = np.concatenate([vox, front, rng.integers(0, n, (8, 3))])
    listed = 0
    for x, y, z in vox:
        ids, (_, lo, hi) = o.voxel_fragments(x, y, z)
        v = (z * n + y) * n + x
        w = int(abc_frame["words"][v])
        assert (w & 0xFFFF) == ids.shape[0], (x, y, z)
        assert lo <= (w >> 16) <= hi, (x, y, z, w >> 16, lo, hi)
        ln = int(abc_frame["len"][v])
        if ln:
            assert ln == ids.shape[0], (x, y, z)
            s = int(abc_frame["start"][v])
            assert np.array_equal(np.sort(abc_frame["ids"][s:s + ln]), ids), (x, y, z)
            listed += 1
    assert listed >= 10


def test_abc_fullsize_sampled_pixels_without_ao(abc_frame):
    cam, o = abc_frame["cam"], abc_frame["oracle"]
    pix = np.random.default_rng(8).choice(cam.width * cam.height, 128, replace=False)
    ref = o.render_pixels(cam, pix, alpha=1.0, brute=True)
    rgba, fid, ft = abc_frame["plain"]
    res = compare_image(rgba[pix], fid[pix], ft[pix], ref)
    assert res["col_bad"] == 0 and res["id_bad"] == 0, res
    assert res["exempt_colour"] <= 0.01 * res["n"] and res["exempt_id"] <= 0.01 * res["n"], res
    assert res["max_t_rel"] < 2e-4, res
    assert res["hits"] >= 100, res


def test_abc_fullsize_ao_pixels_against_oracle(abc_frame):
    """Cone AO at full size: the 512^3 pyramid of all 31M segments, whose cones
    sample levels 1 to 5, on 256 sampled pixels against the oracle's full list
    build and fp64 pyramid (about a minute of oracle time on the host)."""
    cam, o = abc_frame["cam"], abc_frame["oracle"]
    pix = np.random.default_rng(10).choice(cam.width * cam.height, 256, replace=False)
    ref = o.render_pixels(cam, pix, alpha=1.0, ao_cones=6)
    rgba, fid, ft = abc_frame["ao"]
    res = compare_image(rgba[pix], fid[pix], ft[pix], ref)
    assert res["col_bad"] == 0 and res["id_bad"] == 0, res
    assert res["exempt_colour"] <= 0.01 * res["n"] and res["exempt_id"] <= 0.01 * res["n"], res
    assert res["max_t_rel"] < 2e-4, res
    assert res["hits"] >= 200, res
    # AO is partial at most of these hits (the test is not trivially AO = 1)
    plain = abc_frame["plain"][0][pix]
    hit = fid[pix] >= 0
    assert (rgba[pix][hit, :3].sum(1) < 0.95 * plain[hit, :3].sum(1)).mean() > 0.2


def test_abc_fullsize_ao_properties(abc_frame):
    rgba_ao, fid_ao, ft_ao = abc_frame["ao"]
    rgba, fid, ft = abc_frame["plain"]
    assert np.array_equal(fid_ao, fid) and np.array_equal(ft_ao, ft)
    hit = fid >= 0
    assert hit.sum() > 0.5 * fid.shape[0]
    assert np.array_equal(rgba_ao[:, 3], rgba[:, 3])
    assert (rgba_ao[:, :3] <= rgba[:, :3] + 1e-6).all() and (rgba_ao[:, :3] >= 0).all()
    # the occluded interior must darken a good share of the hits
    assert (rgba_ao[hit, :3].sum(1) < 0.95 * rgba[hit, :3].sum(1)).mean() > 0.2


def test_abc_fullsize_voxel_shading_properties(abc_frame):
    # opaque, six-cone AO at voxel centres times 1/2 + S/2: first hits and
    # alpha as without shading, colour only darkened, and differently from
    # the per-hit AO image
    cam, r = abc_frame["cam"], abc_frame["r"]
    rgba, fid, ft = r.frame(cam, alpha=1.0, ao_cones=6, cull_on=1, voxel_shading=1,
                            light=(0.4, 0.5, 0.77))
    vrt.sync(r.h)
    rgba, fid, ft = (rgba.cpu().numpy().reshape(-1, 4), fid.cpu().numpy().reshape(-1),
                     ft.cpu().numpy().reshape(-1))
    p_rgba, p_fid, p_ft = abc_frame["plain"]
    assert np.array_equal(fid, p_fid) and np.array_equal(ft, p_ft)
    assert np.array_equal(rgba[:, 3], p_rgba[:, 3])
    assert (rgba[:, :3] <= p_rgba[:, :3] + 1e-6).all() and (rgba[:, :3] >= 0).all()
    hit = fid >= 0
    assert (rgba[hit, :3].sum(1) < 0.95 * p_rgba[hit, :3].sum(1)).mean() > 0.2
    assert np.abs(rgba - abc_frame["ao"][0]).max() > 0.05


def test_abc_reduced_scale_ao_images():
    ls = G.abc_pathlines(n_particles=15_625, n=128, frame=0)
    cam = G.abc_camera(n=128, frame=0, width=320, height=180)
    o = oracle.Oracle.from_lineset(ls, nthreads=os.cpu_count() or 1)
    pix = np.random.default_rng(9).choice(cam.width * cam.height, 600, replace=False)
    ref = o.render_pixels(cam, pix, alpha=1.0, ao_cones=6)
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    rgba, fid, ft = r.frame(cam, alpha=1.0, ao_cones=6, cull_on=1)
    vrt.sync(r.h)
    rgba = rgba.cpu().numpy().reshape(-1, 4)
    fid = fid.cpu().numpy().reshape(-1)
    ft = ft.cpu().numpy().reshape(-1)
    r.close()
    o.close()
    res = compare_image(rgba[pix], fid[pix], ft[pix], ref)
    assert res["col_bad"] == 0 and res["id_bad"] == 0, res
    assert res["exempt_colour"] <= 0.01 * res["n"] and res["exempt_id"] <= 0.01 * res["n"], res
    assert res["hits"] >= 400, res
