"""The C-ABI library builds, loads and exports every entry point its header declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2109_07073_b300 as vg
from paper_2109_07073_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b(vgicp_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ["vgicp_build_voxelmap", "vgicp_linearize", "vgicp_overlap", "vgicp_overlap_matrix",
              "vgicp_create", "vgicp_destroy", "vgicp_release", "vgicp_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_covers_every_export(lib):
    assert sorted(vg.EXPORTS) == sorted(n for n in declared_functions() if n in vg.EXPORTS)
    missing = [n for n in declared_functions() if n not in vg.EXPORTS]
    assert not missing, missing


def test_host_only_calls_without_a_gpu(lib):
    vg.load()
    o = vg.vgicp_options_default()
    assert o.precision == vg.VGICP_PREC_F32 and o.chunk_points == 2048 and o.linearize_variant == 0 and o.overlap_cull == 1
    assert vg.load().vgicp_status_string(4) == b"VGICP_ERR_EMPTY"
    assert vg.load().vgicp_last_error(None) == b"null context"
    # null context is rejected before any CUDA call
    assert vg.load().vgicp_release(None, 0) == 1
