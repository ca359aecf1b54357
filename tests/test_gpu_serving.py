"""The serving loop (continuous batching of frame requests over resident line
sets): every served frame equals, bitwise, the same frame rendered alone
through the plain calls on a grid that saw the same updates in the same order,
with several frames on the device at once and with sets evicted and uploaded
again under a small HBM budget. Also the one-call frame as a CUDA graph
(equal to the separate calls) and the grid-side autotuner."""
import numpy as np
import pytest

import oracle
import paper_2510_09081_gb300 as vrt
from gen.linesets import Camera, tiny_walks
from parity import compare_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _sets():
    return [tiny_walks(n_lines=400, n_verts=40, n=64, seed=31),
            tiny_walks(n_lines=1500, n_verts=60, n=64, radius=0.3, seed=32),
            tiny_walks(n_lines=300, n_verts=30, n=32, radius=0.5, seed=33, start_lo=4.0, start_hi=28.0),
            tiny_walks(n_lines=2500, n_verts=50, n=64, seed=34)]


def _camera(rng, n, w, h):
    th = rng.uniform(0, 2 * np.pi)
    eye = (n / 2 + 1.6 * n * np.cos(th), n / 2 + 1.6 * n * np.sin(th), n / 2 + 0.4 * n)
    return Camera(width=w, height=h, ortho=0, eye=tuple(map(float, eye)),
                  target=(n / 2, n / 2, n / 2), up=(0, 0, 1), fovy_deg=45.0)


def _requests(sets, n_req, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n_req):
        k = int(rng.integers(len(sets)))
        ls = sets[k]
        w, h = int(rng.integers(40, 97)), int(rng.integers(30, 71))
        upd = None
        first = 0
        if rng.uniform() < 0.6:  # move a block of vertices a little
            cnt = int(rng.integers(1, ls.n_vertices // 10))
            first = int(rng.integers(0, ls.n_vertices - cnt))
            upd = np.clip(ls.xyz[first:first + cnt] + rng.normal(0, 0.2, (cnt, 3)), 1.0,
                          ls.n - 1.0).astype(np.float32)
        reqs.append(dict(set=k, cam=_camera(rng, ls.n, w, h), alpha=float(rng.uniform(0.2, 1.0)),
                         ao=int(rng.uniform() < 0.3) * 6, cull=int(rng.uniform() < 0.5),
                         first=first, update=upd, vs=int(rng.uniform() < 0.3),
                         light=tuple(float(v) for v in rng.normal(size=3))))
    return reqs


def _plain(sets, reqs):
    rs = []
    for ls in sets:
        r = vrt.Renderer(ls.n, ls.radius)
        r.upload(ls.xyz, ls.offsets)
        rs.append(r)
    out = []
    for q in reqs:
        r = rs[q["set"]]
        if q["update"] is not None:
            r.update(q["first"], q["update"])
        rgba, fid, ft = r.frame(q["cam"], alpha=q["alpha"], ao_cones=q["ao"], cull_on=q["cull"],
                                voxel_shading=q["vs"], light=q["light"])
        vrt.sync(r.h)
        out.append((rgba.cpu().numpy().copy(), fid.cpu().numpy().copy(), ft.cpu().numpy().copy()))
    for r in rs:
        r.close()
    return out


def _served(sets, reqs, **kw):
    srv = vrt.Server(**kw)
    ids = [srv.add_set(ls.xyz, ls.offsets, ls.n, ls.radius) for ls in sets]
    bufs, rid = [], {}
    for i, q in enumerate(reqs):
        c = q["cam"]
        b = (torch.zeros((c.height, c.width, 4), device="cuda"),
             torch.zeros((c.height, c.width), dtype=torch.int32, device="cuda"),
             torch.zeros((c.height, c.width), device="cuda"))
        bufs.append(b)
        rid[srv.submit(ids[q["set"]], c, b[0], alpha=q["alpha"], ao_cones=q["ao"], cull_on=q["cull"],
                       first_id=b[1], first_t=b[2], first_vertex=q["first"], update=q["update"],
                       voxel_shading=q["vs"], light=q["light"])] = i
    res = srv.poll(wait=True)
    stats = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    assert len(res) == len(reqs)
    for x in res:
        assert x["status"] == 0, x
        assert x["latency_ms"] >= x["queue_ms"] >= 0.0
    out = [(b[0].cpu().numpy(), b[1].cpu().numpy(), b[2].cpu().numpy()) for b in bufs]
    return out, res, stats


def _assert_equal(a, b):
    for i, (x, y) in enumerate(zip(a, b)):
        for u, v in zip(x, y):
            assert np.array_equal(u, v), i


def test_served_frames_equal_frames_alone():
    sets = _sets()
    reqs = _requests(sets, 40, seed=5)
    alone = _plain(sets, reqs)
    served, res, stats = _served(sets, reqs, max_inflight=4)
    _assert_equal(served, alone)
    assert stats["completed"] == len(reqs) and stats["evictions"] == 0
    assert stats["resident_sets"] == len(sets)
    assert stats["batches"] == 0


def test_batched_small_set_frames_equal_frames_alone():
    """With small_segments = 100000, three of the four sets are small: their
    pending frames go out in batches (one CUDA graph launch per batch)."""
    sets = _sets()
    reqs = _requests(sets, 40, seed=8)
    alone = _plain(sets, reqs)
    served, res, stats = _served(sets, reqs, max_inflight=3, small_segments=100_000)
    _assert_equal(served, alone)
    assert stats["batches"] > 0 and stats["batched_frames"] >= 2 * stats["batches"]


def test_small_set_batches_of_two_equal_frames_alone():
    """Batches capped at two frames, one slot: every batch waits for the one
    before it, and frames of the same set stay in submission order."""
    sets = _sets()[:3]
    reqs = _requests(sets, 18, seed=9)
    alone = _plain(sets, reqs)
    served, res, stats = _served(sets, reqs, max_inflight=1, small_segments=100_000, max_batch=2)
    _assert_equal(served, alone)
    assert stats["batches"] > 0


def test_served_frames_with_evictions_equal_frames_alone():
    sets = _sets()
    reqs = _requests(sets, 40, seed=6)
    alone = _plain(sets, reqs)
    # measure the sets' footprints, then allow about two of them at a time
    sizes = []
    for ls in sets:
        r = vrt.Renderer(ls.n, ls.radius)
        r.upload(ls.xyz, ls.offsets)
        r.frame(_camera(np.random.default_rng(0), ls.n, 96, 70), alpha=0.5, ao_cones=6, cull_on=1,
                voxel_shading=1)
        vrt.sync(r.h)
        sizes.append(vrt.grid_device_bytes(r.h))
        r.close()
    budget = int(sorted(sizes)[-1] + sorted(sizes)[-2] * 1.05)
    served, res, stats = _served(sets, reqs, max_inflight=3, hbm_budget=budget)
    _assert_equal(served, alone)
    assert stats["evictions"] > 0
    assert stats["resident_bytes"] <= budget


def test_server_errors():
    sets = _sets()[:1]
    srv = vrt.Server(max_inflight=2, hbm_budget=1 << 20)  # too small for any set
    sid = srv.add_set(sets[0].xyz, sets[0].offsets, sets[0].n, sets[0].radius)
    cam = _camera(np.random.default_rng(1), 64, 32, 24)
    rgba = torch.zeros((24, 32, 4), device="cuda")
    with pytest.raises(vrt.VrtError) as e:
        srv.submit(sid + 5, cam, rgba)
    assert e.value.status == vrt.ERR_INVALID_ARG
    with pytest.raises(vrt.VrtError) as e:
        srv.submit(sid, cam, rgba, first_vertex=sets[0].n_vertices, update=np.zeros((4, 3), np.float32))
    assert e.value.status == vrt.ERR_INVALID_ARG
    srv.submit(sid, cam, rgba)
    res = srv.poll(wait=True)
    assert len(res) == 1 and res[0]["status"] == vrt.ERR_OOM
    srv.close()


def test_served_frames_match_the_oracle():
    """Every frame of a served mix (updates, culling, AO, voxel-space shading,
    several frames in flight) against the CPU oracle rendering the same set in
    the state that request saw, within the parity tolerances."""
    sets = _sets()[:3]
    reqs = _requests(sets, 18, seed=11)
    served, res, _ = _served(sets, reqs, max_inflight=3)
    state = [ls.xyz.copy() for ls in sets]
    n_hits = 0
    for i, q in enumerate(reqs):
        ls = sets[q["set"]]
        if q["update"] is not None:
            state[q["set"]][q["first"]:q["first"] + q["update"].shape[0]] = q["update"]
        o = oracle.Oracle(state[q["set"]], ls.offsets, ls.n, ls.radius)
        ref = o.render(q["cam"], alpha=q["alpha"], ao_cones=q["ao"], voxel_shading=q["vs"],
                       light=q["light"])
        o.close()
        r = compare_image(*served[i], ref)
        assert r["col_bad"] == 0 and r["id_bad"] == 0, (i, q["alpha"], q["ao"], q["vs"], r)
        assert r["exempt_colour"] <= 0.01 * r["n"] and r["exempt_id"] <= 0.01 * r["n"], (i, r)
        n_hits += r["hits"]
    assert n_hits > 5000


def test_bad_request_fails_at_submit_and_leaves_the_set_intact():
    """A request whose camera or parameters vrt_cull / vrt_trace would reject
    fails in vrt_server_submit, before any of its work (its vertex update
    included) reaches the device; the set's next frames equal the frames
    rendered alone."""
    ls = _sets()[0]
    rng = np.random.default_rng(4)
    good = _requests([ls], 3, seed=12)
    srv = vrt.Server(max_inflight=2)
    sid = srv.add_set(ls.xyz, ls.offsets, ls.n, ls.radius)
    cam = _camera(rng, ls.n, 48, 32)
    rgba = torch.zeros((32, 48, 4), device="cuda")
    upd = (ls.xyz[:50] + 0.25).astype(np.float32)
    bad_kw = [dict(ao_cones=5), dict(alpha=0.0), dict(alpha=1.5), dict(cull_on=3), dict(k=7),
              dict(voxel_shading=2), dict(voxel_shading=1, light=(0.0, 0.0, 0.0))]
    for kw in bad_kw:
        with pytest.raises(vrt.VrtError) as e:
            srv.submit(sid, cam, rgba, first_vertex=0, update=upd, **kw)
        assert e.value.status == vrt.ERR_INVALID_ARG, kw
    bad_cam = Camera(width=48, height=32, ortho=0, eye=(1.0, 2.0, 3.0), target=(1.0, 2.0, 3.0),
                     up=(0, 0, 1), fovy_deg=45.0)
    with pytest.raises(vrt.VrtError) as e:
        srv.submit(sid, bad_cam, rgba, first_vertex=0, update=upd)
    assert e.value.status == vrt.ERR_INVALID_ARG
    assert "camera" in str(e.value)
    bufs = []
    for q in good:
        c = q["cam"]
        b = torch.zeros((c.height, c.width, 4), device="cuda")
        bufs.append(b)
        srv.submit(sid, c, b, alpha=q["alpha"], ao_cones=q["ao"], cull_on=q["cull"],
                   first_vertex=q["first"], update=q["update"], voxel_shading=q["vs"], light=q["light"])
    res = srv.poll(wait=True)
    srv.close()
    assert [x["status"] for x in res] == [0] * len(good)
    alone = _plain([ls], good)
    for b, a in zip(bufs, alone):
        assert np.array_equal(b.cpu().numpy(), a[0])


def test_graph_frames_equal_separate_calls():
    sets = _sets()
    ls = sets[1]
    reqs = [q for q in _requests([ls], 12, seed=7)]
    for q in reqs:  # the same image size throughout, so frames after the first are captured
        q["cam"] = _camera(np.random.default_rng(len(q)), ls.n, 80, 60)
    alone = _plain([ls], reqs)
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    vrt.set_option(r.h, vrt.OPT_GRAPH, 1)
    got = []
    for q in reqs:
        c = vrt.camera_c(q["cam"])
        rgba = torch.zeros((c.height, c.width, 4), device="cuda")
        fid = torch.zeros((c.height, c.width), dtype=torch.int32, device="cuda")
        ft = torch.zeros((c.height, c.width), device="cuda")
        upd = q["update"]
        if upd is not None and len(got) % 3 == 0:
            upd = torch.from_numpy(upd).cuda()
        elif upd is not None and len(got) % 3 == 1:
            upd = torch.from_numpy(upd).pin_memory()  # pageable numpy otherwise (runs uncaptured)
        vrt.frame(r.h, c, vrt.params_c(q["alpha"], q["ao"], q["cull"], 0, q["vs"], q["light"]),
                  rgba, fid, ft, first_vertex=q["first"], update=upd)
        vrt.sync(r.h)
        got.append((rgba.cpu().numpy(), fid.cpu().numpy(), ft.cpu().numpy()))
    r.close()
    _assert_equal(got, alone)


def test_tune_grid_side():
    ls = _sets()[0]
    cam = _camera(np.random.default_rng(3), ls.n, 96, 64)
    best, ms = vrt.tune_grid_side(ls.xyz, ls.offsets, ls.n, ls.radius, cam, [32, 64, 128], alpha=0.5)
    assert best in (32, 64, 128)
    assert all(np.isfinite(v) and v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())


def test_tune_shapes_and_tile_widths_give_the_same_image():
    """The tuner measures every (grid side, trace tile) pair; the tile shape of
    the transparent trace changes speed only: images are bitwise equal."""
    ls = _sets()[1]
    cam = _camera(np.random.default_rng(5), ls.n, 96, 64)
    (side, tile), ms = vrt.tune_shapes(ls.xyz, ls.offsets, ls.n, ls.radius, cam, [32, 64],
                                       tiles=(2, 4, 8, 16), alpha=0.4, cull_on=1)
    assert len(ms) == 8 and all(np.isfinite(v) and v > 0 for v in ms.values())
    assert ms[(side, tile)] == min(ms.values())
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    imgs = []
    for tw in (4, 2, 8, 16):
        vrt.set_option(r.h, vrt.OPT_TRACE_TILE, tw)
        rgba, fid, ft = r.frame(cam, alpha=0.4, cull_on=1)
        vrt.sync(r.h)
        imgs.append((rgba.cpu().numpy().copy(), fid.cpu().numpy().copy(), ft.cpu().numpy().copy()))
    with pytest.raises(vrt.VrtError):
        vrt.set_option(r.h, vrt.OPT_TRACE_TILE, 3)
    r.close()
    for img in imgs[1:]:
        for a, b in zip(imgs[0], img):
            assert np.array_equal(a, b)
