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
    """Sizes beyond the fixed scratch are rejected by the C entry point before
    any device work (called through the C ABI directly, since the binding
    would refuse these sizes first); sizes beyond the tensors by the binding."""
    import ctypes
    words = torch.zeros(4096, dtype=torch.int32, device="cuda")
    offsets = torch.zeros(4096, dtype=torch.int32, device="cuda")
    lib = vrt.load()
    for n in (512 ** 3 + 4096, 4095, 0):
        st = lib.vrt_scan_counts_noalloc(ctypes.c_void_p(words.data_ptr()), None,
                                         ctypes.c_void_p(offsets.data_ptr()), n, None, None, None)
        assert st == vrt.ERR_INVALID_ARG, n
        if n > 512 ** 3:
            assert b"scratch" in lib.vrt_last_error(None)
    for kw in (dict(n_voxels=8192), dict(marks=torch.zeros(64, dtype=torch.int32, device="cuda"))):
        with pytest.raises(vrt.VrtError) as e:
            vrt.scan_counts_noalloc(words, offsets, **kw)
        assert e.value.status == vrt.ERR_INVALID_ARG
    with pytest.raises(vrt.VrtError):
        vrt.scan_counts_noalloc(words, torch.zeros(2048, dtype=torch.int32, device="cuda"))


def test_noalloc_scan_reports_a_total_past_32_bits():
    """2^17 voxels of count 65535 sum to 8.6e9 > 2^32 - 1: status bit 1, and
    each offset is its prefix sum modulo 2^32."""
    n = 1 << 17
    words = torch.full((n,), 0xFFFF, dtype=torch.int32, device="cuda")
    offsets = torch.zeros(n, dtype=torch.int32, device="cuda")
    total = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    vrt.scan_counts_noalloc(words, offsets, total=total, status=status)
    torch.cuda.synchronize()
    want = (np.arange(n, dtype=np.uint64) * 65535) % (1 << 32)
    assert np.array_equal(offsets.cpu().numpy().view(np.uint32).astype(np.uint64), want)
    assert int(total.cpu().numpy().view(np.uint32)[0]) == (n * 65535) % (1 << 32)
    assert int(status.cpu()[0]) == vrt.NOALLOC_WRAPPED


def test_noalloc_scan_wait_gives_up_then_scans_correctly_again():
    """A test option makes tile 3 of 64 skip its publish: the waits after it
    run out (after 1024 polls) and set status bit 0; with the option off, two
    calls in a row give the right offsets again."""
    n = 64 * 4096
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 9, n).astype(np.uint32)
    words = torch.from_numpy(counts.view(np.int32)).cuda()
    want = np.concatenate([[0], np.cumsum(counts.astype(np.uint64))[:-1]])
    offsets = torch.zeros(n, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    try:
        vrt.set_option(None, vrt.OPT_TEST_SCAN_STALL, 3)
        vrt.scan_counts_noalloc(words, offsets, status=status)
        torch.cuda.synchronize()
    finally:
        vrt.set_option(None, vrt.OPT_TEST_SCAN_STALL, -1)
    assert int(status.cpu()[0]) & vrt.NOALLOC_GAVE_UP
    for call in range(2):
        status.zero_()
        offsets.fill_(-1)
        vrt.scan_counts_noalloc(words, offsets, status=status)
        torch.cuda.synchronize()
        assert int(status.cpu()[0]) == 0, call
        assert np.array_equal(offsets.cpu().numpy().view(np.uint32), want.astype(np.uint32)), call
