"""vrt_scan_counts_noalloc, the list-offset scan for callers that cannot
allocate device memory where they need it (memory owned by a pool or arena,
loops that must not grow memory mid-frame, real-time paths), must give the
same offsets as the grid's own list build (vrt_cull), call after call, while
its scratch lives in a fixed array inside the library.

This file is collected last so that, if it fails, a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import paper_2510_09081_gb300 as vrt
from gen.linesets import Camera, tiny_walks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def to_brick_order(canon, n):
    """Canonical voxel order (x fastest) -> the grid's 4^3-brick order."""
    a = canon.reshape(n // 4, 4, n // 4, 4, n // 4, 4)   # bz, z, by, y, bx, x
    return np.ascontiguousarray(a.transpose(0, 2, 4, 1, 3, 5)).reshape(-1)


def from_brick_order(b, n):
    a = b.reshape(n // 4, n // 4, n // 4, 4, 4, 4)        # bz, by, bx, z, y, x
    return np.ascontiguousarray(a.transpose(0, 3, 1, 4, 2, 5)).reshape(-1)


def grid_offsets(cull):
    """Words and list offsets from the existing entry points (no trace, so no
    repair allocations)."""
    ls = tiny_walks(n_lines=1500, n_verts=50, seed=31)
    cam = Camera(width=120, height=90, ortho=0, eye=(100.0, 85.0, 50.0), target=(32, 32, 32),
                 up=(0, 0, 1), fovy_deg=45.0)
    r = vrt.Renderer(ls.n, ls.radius)
    r.upload(ls.xyz, ls.offsets)
    vrt.voxelize(r.h)
    vrt.cull(r.h, vrt.camera_c(cam), vrt.params_c(alpha=0.3, cull=cull))
    vrt.sync(r.h)
    words = vrt.read_grid(r.h, ls.n)
    start, length, ids = vrt.read_lists(r.h, ls.n)
    r.close()
    return ls.n, words, start, length, ids.shape[0]


def run_noalloc(words_b, marks_b, n):
    dev_words = torch.from_numpy(words_b.view(np.int32)).cuda()
    dev_marks = None if marks_b is None else torch.from_numpy(marks_b.view(np.int32)).cuda()
    offsets = torch.full((n ** 3,), -1, dtype=torch.int32, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    vrt.scan_counts_noalloc(dev_words, offsets, marks=dev_marks, total=total, status=status)
    torch.cuda.synchronize()
    off = from_brick_order(offsets.cpu().numpy().view(np.uint32), n)
    return off, int(total.cpu().numpy().view(np.uint32)[0]), int(status.cpu()[0])


@pytest.mark.parametrize("cull", [0, 1])
def test_noalloc_scan_matches_the_list_build_twice(cull):
    n, words, start, length, n_ids = grid_offsets(cull)
    wb = to_brick_order(words, n)
    marks_b = None
    if cull:
        listed = to_brick_order((length > 0).astype(np.uint8), n)
        marks_b = np.packbits(listed.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").astype(np.uint32).reshape(-1)
    listed = length > 0
    assert listed.sum() > 1000
    for call in range(2):
        off, total, status = run_noalloc(wb, marks_b, n)
        assert status == 0, f"call {call}: a bounded wait gave up"
        assert np.array_equal(off[listed], start[listed]), f"call {call}: offsets differ"
        assert total == n_ids, f"call {call}: total {total} vs {n_ids}"


def test_noalloc_scan_rejects_sizes_beyond_its_scratch():
    words = torch.zeros(4096, dtype=torch.int32, device="cuda")
    offsets = torch.zeros(4096, dtype=torch.int32, device="cuda")
    with pytest.raises(vrt.VrtError) as e:
        vrt.scan_counts_noalloc(words, offsets, n_voxels=512 ** 3 + 4096)
    assert e.value.status == vrt.ERR_INVALID_ARG
    assert "scratch" in str(e.value)
    with pytest.raises(vrt.VrtError) as e:
        vrt.scan_counts_noalloc(words, offsets, n_voxels=4095)
    assert e.value.status == vrt.ERR_INVALID_ARG
