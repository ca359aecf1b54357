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
