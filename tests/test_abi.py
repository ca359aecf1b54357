"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/vrt.h declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

import paper_2510_09081_gb300 as vrt
from paper_2510_09081_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vrt_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return vrt.load()


def test_header_declares_the_binding_symbols():
    assert _declared() == sorted(vrt.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_side_argument_checks(lib):
    """Argument errors are reported before any device work."""
    h = ctypes.c_void_p()
    bad = vrt.GridDesc(n=100, radius=0.4, r_min=0.5, occ_scale=32, max_fragments=0)
    assert lib.vrt_create_grid(ctypes.byref(bad), None, ctypes.byref(h)) == vrt.ERR_INVALID_ARG
    assert b"power of two" in lib.vrt_last_error(None)
    bad = vrt.GridDesc(n=64, radius=0.0, r_min=0.5, occ_scale=32, max_fragments=0)
    assert lib.vrt_create_grid(ctypes.byref(bad), None, ctypes.byref(h)) == vrt.ERR_INVALID_ARG
    assert lib.vrt_create_grid(None, None, ctypes.byref(h)) == vrt.ERR_INVALID_ARG
    assert lib.vrt_voxelize(None) == vrt.ERR_INVALID_ARG
    assert lib.vrt_destroy(None) == vrt.OK


def test_option_and_message_checks_without_a_grid(lib):
    """Options without a grid: only the no-allocation scan's test stall is
    process-wide; everything else needs a grid. Messages are per host thread."""
    import threading
    assert lib.vrt_set_option(None, vrt.OPT_GRAPH, 1) == vrt.ERR_INVALID_ARG
    assert lib.vrt_set_option(None, vrt.OPT_TEST_SCAN_STALL, -2) == vrt.ERR_INVALID_ARG
    assert b"stall tile" in lib.vrt_last_error(None)
    assert lib.vrt_set_option(None, vrt.OPT_TEST_SCAN_STALL, 7) == vrt.OK
    assert lib.vrt_set_option(None, vrt.OPT_TEST_SCAN_STALL, -1) == vrt.OK
    seen = {}

    def other():
        seen["before"] = lib.vrt_last_error(None)
        lib.vrt_create_grid(None, None, ctypes.byref(ctypes.c_void_p()))
        seen["after"] = lib.vrt_last_error(None)

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["before"] == b""            # a new thread starts with no message
    assert seen["after"] != b"" and b"stall tile" in lib.vrt_last_error(None)


def test_noalloc_binding_checks_sizes_before_the_call(lib):
    """The C call cannot see tensor sizes: the binding refuses an n_voxels
    beyond words, offsets or marks, and tensors that are not 32-bit CUDA ones."""
    torch = pytest.importorskip("torch")
    w = torch.zeros(4096, dtype=torch.int32)
    for kw in (dict(n_voxels=8192), dict(marks=torch.zeros(64, dtype=torch.int32))):
        with pytest.raises(vrt.VrtError) as e:
            vrt.scan_counts_noalloc(w, torch.zeros(4096, dtype=torch.int32), **kw)
        assert e.value.status == vrt.ERR_INVALID_ARG
    with pytest.raises(vrt.VrtError, match="offsets"):
        vrt.scan_counts_noalloc(w, torch.zeros(2048, dtype=torch.int32))
    with pytest.raises(vrt.VrtError, match="CUDA tensor"):
        vrt.scan_counts_noalloc(w, torch.zeros(4096, dtype=torch.int32))
    with pytest.raises(vrt.VrtError, match="32-bit"):
        vrt.scan_counts_noalloc(w, torch.zeros(4096, dtype=torch.int64))


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(vrt, "_lib", None)
    monkeypatch.setattr(vrt, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(vrt.VrtError):
        vrt.load()


def test_build_targets_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


STRUCTS = {"vrt_grid_desc": "GridDesc", "vrt_camera": "CameraC", "vrt_render_params": "RenderParamsC",
           "vrt_stats": "StatsC", "vrt_server_desc": "ServerDesc", "vrt_server_result": "ServerResult",
           "vrt_server_stats": "ServerStats"}


def test_binding_structs_match_the_header(tmp_path):
    """Size and every field offset of each struct the binding mirrors, as the
    host compiler lays them out from include/vrt.h."""
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    lines = ['#include <cstddef>', '#include <cstdio>', '#include "vrt.h"', 'int main() {']
    for cname, pyname in STRUCTS.items():
        lines.append(f'  std::printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in getattr(vrt, pyname)._fields_:
            lines.append(f'  std::printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.cpp"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cxx, "-std=c++17", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, pyname in STRUCTS.items():
        py = getattr(vrt, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
