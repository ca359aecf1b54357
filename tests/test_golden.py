"""The oracle against the hand-derived closed forms stored in
tests/golden/closed_forms.txt (each line cites the passage it follows)."""
import json
import math
import os

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


@pytest.mark.parametrize("fn,args,want", _cases())
def test_closed_form(fn, args, want):
    import numpy as np
    a = dict(args)
    if fn == "line_capsule_entry":
        got = oracle.line_capsule_entry(a["o"], a["d"], a["a"], a["b"], a["r"])
    elif fn == "clipped_capsule_sdf":
        got = oracle.clipped_capsule_sdf(a["p"], a["v0"], a["v1"], n0=a.get("n0", (0, 0, 0)),
                                         n1=a.get("n1", (0, 0, 0)), en0=a.get("en0", 0),
                                         en1=a.get("en1", 0), r=a["r"])
    elif fn == "capsule_occupancy":
        got = oracle.capsule_occupancy(a["p"], a["v0"], a["v1"], r=a["r"], r_min=a["r_min"])
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
