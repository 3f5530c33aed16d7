"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/rhi.h.
No compute calls (no GPU here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rhi.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*(rhi_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_0901_1110_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rhi_create", "rhi_set_state", "rhi_implicit_step", "rhi_get_state",
                 "rhi_get_stats", "rhi_destroy", "rhi_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    import paper_0901_1110_gb300 as rhi
    assert set(rhi._SIGS) == set(declared_functions())


def test_library_targets_sm_103a(libpath):
    """The build compiles every translation unit for sm_103a alone (the -gencode flag the
    build passes to nvcc)."""
    from paper_0901_1110_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH
