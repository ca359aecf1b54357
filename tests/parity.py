"""Comparison helpers for the parity tests (GPU path vs the CPU oracle).

Tolerances:
  * lists and per-voxel counts: bit-exact (lists compared after a per-voxel sort
    by segment id);
  * per-voxel occupancy code sums: exact, except that a contribution whose
    fp64 value sits within 1e-3 of a rounding boundary may round either way
    (the oracle returns the allowed [lo, hi] range per voxel);
  * first-hit ids: equal to the oracle's, or to its single alternative when
    exactly one near-tie event (grazing ray, hit on a clip plane or the grid
    boundary, depth tie) could change it, or exempt when several could;
  * RGBA: |difference| <= 2e-3 per channel against the primary or alternative
    oracle result, same exemption rule.
"""
from __future__ import annotations

import numpy as np

RGBA_TOL = 2e-3


def gpu_fragments(start, length, ids):
    """Sorted (voxel << 32 | id) keys of a GPU list set (canonical voxel order)."""
    nz = np.nonzero(length)[0]
    ln = length[nz].astype(np.int64)
    st = start[nz].astype(np.int64)
    total = int(ln.sum())
    vox = np.repeat(nz.astype(np.uint64), ln)
    base = np.repeat(st - np.concatenate([[0], np.cumsum(ln)[:-1]]), ln)
    pos = base + np.arange(total, dtype=np.int64)
    keys = (vox << np.uint64(32)) | ids[pos].astype(np.uint64)
    keys.sort()
    return keys


def oracle_fragments(L):
    cnt = L["count"].astype(np.int64)
    vox = np.repeat(np.arange(cnt.shape[0], dtype=np.uint64), cnt)
    return (vox << np.uint64(32)) | L["ids"].astype(np.uint64)


def check_words(words, L):
    count = words & 0xFFFF
    occ = words >> 16
    assert np.array_equal(count, L["count"]), "per-voxel counts differ"
    bad = (occ < L["occ_lo"]) | (occ > L["occ_hi"])
    assert not bad.any(), f"{int(bad.sum())} voxels with occupancy outside the oracle's range"


def check_lists(start, length, ids, L, words=None):
    g = gpu_fragments(start, length, ids)
    o = oracle_fragments(L)
    assert g.shape == o.shape, f"fragment count {g.shape[0]} vs oracle {o.shape[0]}"
    assert np.array_equal(g, o), "list contents differ"


def compare_image(rgba, fid, ft, ref, tol=RGBA_TOL, check_t=True):
    """rgba [Npx, 4], fid [Npx], ft [Npx] from the GPU; ref from Oracle.render.
    Returns a dict of mismatch statistics (asserts nothing)."""
    rgba = rgba.reshape(-1, 4)
    fid = fid.reshape(-1)
    ft = ft.reshape(-1)
    ex_c = (ref["exempt"] & 1) != 0
    ex_i = (ref["exempt"] & 2) != 0
    d0 = np.abs(rgba - ref["rgba"]).max(1)
    d1 = np.abs(rgba - ref["rgba_alt"]).max(1)
    col_bad = (np.minimum(d0, d1) > tol) & ~ex_c
    id_bad = (fid != ref["first_id"]) & (fid != ref["first_id_alt"]) & ~ex_i
    same = (fid == ref["first_id"]) & (fid >= 0)
    t_err = np.abs(ft[same] - ref["first_t"][same]) / (1.0 + np.abs(ref["first_t"][same]))
    return dict(n=int(fid.shape[0]), col_bad=int(col_bad.sum()), id_bad=int(id_bad.sum()),
                exempt_colour=int(ex_c.sum()), exempt_id=int(ex_i.sum()),
                max_dcol=float(np.where(ex_c, 0, np.minimum(d0, d1)).max(initial=0.0)),
                max_t_rel=float(t_err.max(initial=0.0)), hits=int((fid >= 0).sum()),
                col_bad_idx=np.nonzero(col_bad)[0][:10], id_bad_idx=np.nonzero(id_bad)[0][:10])
