"""The oracle against the hand-derived closed forms stored in
tests/golden/closed_forms.txt (each line cites the passage it follows)."""
import json
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    out = []
    with open(os.path.join(HERE, "golden", "closed_forms.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            fn, args, want, cite, why = (x.strip() for x in line.split("|"))
            out.append(pytest.param(fn, json.loads(args), want, id=f"{fn}: {why[:40]}"))
    return out


def _lines_along_y(xs, n):
    """One 2-vertex polyline along y through the centre of every voxel column
    (x, *, z) with x in xs, reaching past both grid faces."""
    xyz = [((x + 0.5, -0.5, z + 0.5), (x + 0.5, n + 0.5, z + 0.5)) for x in xs for z in range(n)]
    xyz = np.array(xyz, np.float32).reshape(-1, 3)
    return xyz, np.arange(0, xyz.shape[0] + 1, 2, dtype=np.int64)


def _ao_field(field, n):
    """Occupancy fields with closed-form pyramids: with r = r_min = 0.5 a line
    through voxel centres gives its voxels occupancy 1 and their neighbours 0."""
    xs = {"alternate": range(0, n, 2), "wall": range(n // 2), "full": range(n)}[field]
    xyz, off = _lines_along_y(xs, n)
    return oracle.Oracle(xyz, off, n, 0.5, r_min=0.5)


@pytest.mark.parametrize("fn,args,want", _cases())
def test_closed_form(fn, args, want):
    a = dict(args)
    if fn == "line_capsule_entry":
        got = oracle.line_capsule_entry(a["o"], a["d"], a["a"], a["b"], a["r"])
    elif fn == "clipped_capsule_sdf":
        got = oracle.clipped_capsule_sdf(a["p"], a["v0"], a["v1"], n0=a.get("n0", (0, 0, 0)),
                                         n1=a.get("n1", (0, 0, 0)), en0=a.get("en0", 0),
                                         en1=a.get("en1", 0), r=a["r"])
    elif fn == "capsule_occupancy":
        got = oracle.capsule_occupancy(a["p"], a["v0"], a["v1"], r=a["r"], r_min=a["r_min"])
    elif fn == "cone_ao":
        got = _ao_field(a["field"], a["N"]).ao(np.array(a["P"], np.float64))
    elif fn == "mip_single_voxel":
        x, y, z = a["voxel"]
        c = np.array([[x + 0.5, y + 0.5, z + 0.5]] * 2, np.float32)
        levels = oracle.Oracle(c, np.array([0, 2], np.int64), a["N"], 0.5, r_min=0.5).mips()
        assert len(levels) == int(math.log2(a["N"])) + 1
        for l, lv in enumerate(levels):  # arrays are indexed [z, y, x]
            want_l = np.zeros_like(lv)
            want_l[z >> l, y >> l, x >> l] = 8.0 ** -l
            assert np.array_equal(lv, want_l), f"level {l}"
        return
    elif fn == "seg_box_within":
        got = oracle.seg_box_within(np.array(a["A"]), np.array(a["B"]), np.array(a["lo"]), a["S"], a["R"])
        assert bool(got) == (want == "true")
        return
    else:
        raise AssertionError(fn)
    if want == "inf":
        assert got == math.inf
    else:
        assert got == pytest.approx(float(want), abs=1e-12)
