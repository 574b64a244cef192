"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol
declared in include/homb.h (no compute call is made here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import __graft_entry__
    return __graft_entry__._builder().build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "homb.h")).read()
    return sorted(set(re.findall(r"^(?:hom_status|const char\*)\s+(hom_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("hom_create", "hom_destroy", "hom_bounds", "hom_workspace_size", "hom_matvec",
                     "hom_coefficient", "hom_rhs", "hom_energy", "hom_fft", "hom_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in header_functions():
        assert hasattr(lib, name), name
    lib.hom_version.restype = ctypes.c_char_p
    assert lib.hom_version().startswith(b"homb")


def test_binding_names_match_header(libpath):
    import paper_1404_3614_gb300.binding as bd
    for name in header_functions():
        assert hasattr(bd, name), name


def test_struct_layouts_match_header(libpath):
    import paper_1404_3614_gb300.binding as bd
    # hom_inclusion: 2 int32 + 3 + 3 + 9 doubles
    assert ctypes.sizeof(bd.hom_inclusion) == 8 + 15 * 8
    assert ctypes.sizeof(bd.hom_problem) == 4 + 12 + 24 + 72 + 8 + 8 + 8 + 12 + 4
    assert ctypes.sizeof(bd.hom_opts) == 4 + 4 + 8 + 4 + 4 + 4 + 4 + 4 + 4


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = ctypes.CDLL(libpath)
    h = ctypes.c_void_p()
    st = lib.hom_create(ctypes.byref(h), 0)
    assert st != 0   # HOM_ERR_CUDA, no crash
