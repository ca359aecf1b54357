"""Trace paths the default scenes rarely reach, and the bounded device waits,
through the C ABI.

- The whole-warp list path (lists longer than the shared-entry limit, or a
  transparent ray with more hits in one voxel than its slots): forced by the
  test options on the perspective parity scenes, and reached without options by
  a dense bundle that puts hundreds of hits of every ray into one voxel (each
  lane then drops keys and the warp rescans the list).
- The list-offset scan's look-back waits: a test option makes one tile skip
  its publish, so the waits after it run out; vrt_sync reports
  VRT_ERR_TIMEOUT and the grid renders correctly afterwards.
Tolerances are those of tests/parity.py."""
import numpy as np
import pytest

import oracle
import paper_2510_09081_gb300 as vrt
from gen.linesets import Camera, LineSet, tiny_walks
from parity import compare_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _persp_cam(n=64, w=157, h=93):
    return Camera(width=w, height=h, ortho=0, eye=(n * 1.6, n * 1.3, n * 0.9),
                  target=(n / 2, n / 2, n / 2), up=(0, 0, 1), fovy_deg=45.0)


def _image(r, cam, alpha, cull=0):
    rgba, fid, ft = r.frame(cam, alpha=alpha, cull_on=cull)
    vrt.sync(r.h)
    return rgba.cpu().numpy(), fid.cpu().numpy(), ft.cpu().numpy()


def _assert_parity(res, max_exempt=0.01):
    assert res["col_bad"] == 0, res
    assert res["id_bad"] == 0, res
    assert res["exempt_colour"] <= max_exempt * res["n"], res
    assert res["exempt_id"] <= max_exempt * res["n"], res
    assert res["max_t_rel"] < 2e-4, res


@pytest.mark.parametrize("alpha", [1.0, 0.3, 0.1])
def test_whole_warp_path_matches_oracle(alpha):
    ls = tiny_walks(n_lines=600, n_verts=40, seed=123)
    cam = _persp_cam()
    ref = oracle.Oracle.from_lineset(ls).render(cam, alpha=alpha)
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    default = _image(r, cam, alpha)
    vrt.set_option(r.h, vrt.OPT_TRACE_SHORT_LIST, 0)  # every list on the whole-warp path
    forced = _image(r, cam, alpha)
    vrt.set_option(r.h, vrt.OPT_TRACE_SHORT_LIST, 1024)
    r.close()
    res = compare_image(*forced, ref)
    assert res["hits"] > 2000
    _assert_parity(res)
    # both paths composite every hit in (depth, id) order: the same image
    for a, b in zip(default, forced):
        assert np.array_equal(a, b)


def test_few_ray_key_slots_match_oracle():
    """With 2 hit slots per ray, every transparent ray with more than two hits
    in a voxel leaves the shared-entry path for the whole-warp path."""
    ls = tiny_walks(n_lines=600, n_verts=40, seed=123)
    cam = _persp_cam()
    ref = oracle.Oracle.from_lineset(ls).render(cam, alpha=0.3)
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    default = _image(r, cam, 0.3)
    vrt.set_option(r.h, vrt.OPT_TRACE_RAY_KEYS, 2)
    few = _image(r, cam, 0.3)
    with pytest.raises(vrt.VrtError):
        vrt.set_option(r.h, vrt.OPT_TRACE_RAY_KEYS, 33)
    r.close()
    _assert_parity(compare_image(*few, ref))
    for a, b in zip(default, few):
        assert np.array_equal(a, b)


def _dense_bundle(n_lines=600, seed=77):
    """n_lines straight tubes along x through one column of voxels: y within
    0.05 of 16, z spread over 16 +- 0.45, r = 0.4, so a ray looking down z
    through the bundle's middle hits every tube, most of them in one voxel."""
    rng = np.random.default_rng(seed)
    y = 16.0 + rng.uniform(-0.05, 0.05, n_lines)
    z = 16.0 + rng.uniform(-0.45, 0.45, n_lines)
    xyz = np.stack([np.stack([np.full(n_lines, 2.0), y, z], 1),
                    np.stack([np.full(n_lines, 30.0), y, z], 1)], 1).reshape(-1, 3)
    return LineSet(xyz=xyz.astype(np.float32), offsets=np.arange(0, 2 * n_lines + 1, 2), n=32,
                   radius=0.4)


@pytest.mark.parametrize("alpha", [1.0, 0.1, 0.02])
def test_dense_voxel_rescans_match_oracle(alpha):
    """Hundreds of hits per ray in one voxel: lanes keep four keys each, so the
    whole-warp path extracts keys in rounds and rescans the list (alpha 0.02
    composites about 450 hits of one ray). Every tube has the same tangent
    colour, so the colour does not depend on the order of near-equal depths:
    RGBA is compared on every pixel, exemptions aside."""
    ls = _dense_bundle()
    cam = Camera(width=64, height=8, ortho=1, eye=(16.0, 16.0, 40.0), target=(16.0, 16.0, 0.0),
                 up=(0, 1, 0), fovy_deg=45.0, ortho_h=0.1)
    o = oracle.Oracle(ls.xyz, ls.offsets, ls.n, ls.radius, occ_scale=1)
    ref = o.render(cam, alpha=alpha)
    L = o.lists()
    assert L["count"].max() >= 500
    r = vrt.Renderer(ls.n, ls.radius, occ_scale=1)
    r.upload(ls.xyz, ls.offsets)
    rgba, fid, ft = _image(r, cam, alpha)
    r.close()
    d = np.abs(rgba.reshape(-1, 4) - ref["rgba"]).max(1)
    assert d.max() <= 2e-3, d.max()
    res = compare_image(rgba, fid, ft, ref)
    assert res["id_bad"] == 0, res
    assert res["exempt_id"] <= 0.05 * res["n"], res
    assert res["hits"] == res["n"]
    if alpha < 1.0:  # stopped at T < 1e-4 after about ln(1e-4) / ln(1 - alpha) hits
        assert (rgba[..., 3] > 1.0 - 2e-4).all()


def test_scan_wait_gives_up_and_the_grid_recovers():
    """Tile 5 of the 64 tiles of a 64^3 scan never publishes: the waits of the
    tiles after it give up after 1024 polls and set the timeout status, which
    vrt_sync returns. With the option off the next frame equals a normal one."""
    ls = tiny_walks(n_lines=600, n_verts=40, seed=123)
    cam = _persp_cam()
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    before = _image(r, cam, 0.3, cull=1)
    vrt.set_option(r.h, vrt.OPT_TEST_SCAN_STALL, 5)
    vrt.voxelize(r.h)
    vrt.cull(r.h, vrt.camera_c(cam), vrt.params_c(alpha=0.3, cull=1))
    with pytest.raises(vrt.VrtError) as e:
        vrt.sync(r.h)
    assert e.value.status == vrt.ERR_TIMEOUT
    vrt.set_option(r.h, vrt.OPT_TEST_SCAN_STALL, -1)
    after = _image(r, cam, 0.3, cull=1)
    r.close()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("alpha", [1.0, 0.3, 0.1])
def test_paper_hit_key_matches_oracle(alpha):
    """The paper's 32-bit hit key (VRT_OPT_HIT_KEY = 16+16: the depth within the
    voxel quantized to 16 bits above the fragment's list index) against the
    oracle's ground-truth order, within the parity tolerances; the pixels where
    its order differs from the default (depth, id) key are few."""
    ls = tiny_walks(n_lines=600, n_verts=40, seed=123)
    cam = _persp_cam()
    ref = oracle.Oracle.from_lineset(ls).render(cam, alpha=alpha)
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    default = _image(r, cam, alpha)
    vrt.set_option(r.h, vrt.OPT_HIT_KEY, vrt.HIT_KEY_16_16)
    k16 = _image(r, cam, alpha)
    with pytest.raises(vrt.VrtError):
        vrt.set_option(r.h, vrt.OPT_HIT_KEY, 2)
    vrt.set_option(r.h, vrt.OPT_HIT_KEY, vrt.HIT_KEY_DEPTH_ID)
    again = _image(r, cam, alpha)
    r.close()
    res = compare_image(*k16, ref)
    assert res["hits"] > 2000
    _assert_parity(res)
    changed = int(np.any(default[0] != k16[0], axis=-1).sum())
    assert changed <= 0.001 * res["n"], changed
    # ids and depths of the first hits: the same hits, exact depths
    same_first = default[1] == k16[1]
    assert same_first.mean() > 0.999
    assert np.array_equal(default[2][same_first], k16[2][same_first])
    for a, b in zip(default, again):
        assert np.array_equal(a, b)
