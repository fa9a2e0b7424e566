"""The C-ABI library loads without a GPU and exports every entry point that
include/gs.h declares; the binding covers exactly those names.  No compute
call is made here."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(gs_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    return __graft_entry__._gs_build_module().build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gs_project", "gs_render_with_grads", "gs_upscale", "gs_render", "gs_create", "gs_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ct.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(libpath):
    import paper_2503_14171_gb300 as gs
    assert gs.exported_symbols() == declared_functions()


def test_status_strings_without_gpu(libpath):
    import paper_2503_14171_gb300 as gs
    assert gs.gs_status_string(gs.GS_OK) == "GS_OK"
    assert gs.gs_status_string(gs.GS_ERR_CAPACITY) == "GS_ERR_CAPACITY"
    assert gs.gs_last_error(None) == ""


def test_struct_layouts_match_header(libpath):
    """Sizes of the ABI structs as the C compiler lays them out."""
    import paper_2503_14171_gb300 as gs
    assert ct.sizeof(gs.GsGaussians) == 8 + 4 + 4 + 6 * 8
    assert ct.sizeof(gs.GsCamera) == 21 * 4
    assert ct.sizeof(gs.GsOptions) == 32
