"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/h4d.h declares.  No compute call is made (no GPU here)."""
import os
import re

import pytest

from paper_2307_11447_gb300 import lib as h4d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(h4d_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("h4d_create", "h4d_set_mu", "h4d_set_protocol", "h4d_run_md", "h4d_run_trials",
                     "h4d_get_counts", "h4d_get_energies", "h4d_get_work", "h4d_destroy", "h4d_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = h4d.lib()
    for name in sorted(declared_functions()):
        assert hasattr(L, name), name


def test_library_is_built_for_sm103a():
    """the build compiles every translation unit with one gencode, sm_103a (the kernel's
    binary version is checked at run time on the GPU, tests/test_gpu_device.py)"""
    from paper_2307_11447_gb300 import build as b

    path = h4d.library_path()
    assert os.path.exists(path)
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_names_every_code():
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert h4d.strerror(code) and h4d.strerror(code) != "unknown error"
    assert h4d.strerror(-99) == "unknown error"


def test_structure_sizes_match_header_layout():
    import ctypes
    # h4d_record: 10 int32 + 6 double
    assert h4d.RECORD_DTYPE.itemsize == 88
    assert ctypes.sizeof(h4d.h4d_counts) == 8 * 26
