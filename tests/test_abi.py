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
    assert ctypes.sizeof(bd.hom_problem) == 4 + 12 + 24 + 72 + 8 + 8 + 8 + 12 + 4 + 4 + 4   # + smooth, padding
    assert ctypes.sizeof(bd.hom_opts) == 4 + 4 + 8 + 4 + 4 + 4 + 4 + 4 + 4 + 4 + 4 + 8   # + warm_start, net


def test_struct_layouts_match_a_c_compiler(libpath, tmp_path):
    """Every struct of the header, compiled by the host C compiler: its size and the offset of
    each field equal the ctypes mirror in the binding (the binding cannot drift from the ABI)."""
    import shutil
    import subprocess
    import paper_1404_3614_gb300.binding as bd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"hom_inclusion": bd.hom_inclusion, "hom_problem": bd.hom_problem, "hom_opts": bd.hom_opts,
               "hom_report": bd.hom_report, "hom_field_io": bd.hom_field_io, "hom_batch_io": bd.hom_batch_io,
               "hom_net_config": bd.hom_net_config}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "homb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} @sizeof %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for name, cls in structs.items():
        assert got[(name, "@sizeof")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = ctypes.CDLL(libpath)
    h = ctypes.c_void_p()
    st = lib.hom_create(ctypes.byref(h), 0)
    assert st != 0   # HOM_ERR_CUDA, no crash
