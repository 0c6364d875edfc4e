"""CPU-only checks of the C-ABI library: it loads and exports every entry point that
include/dh.h declares (no CUDA call is made)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(dh_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_00923_b300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dh_plan_create", "dh_render_stack", "dh_pca_window", "dh_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_2004_00923_b300 import _lib
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == declared_functions()


def test_status_strings_without_gpu(lib):
    assert lib.dh_status_string(0) == b"ok"
    assert lib.dh_status_string(2) == b"unsupported size"
    assert lib.dh_version().startswith(b"libdh")


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.dh_plan_create(None, 64, 64, 785e-9, 0.35, 20e-6, 32) == 1
    assert lib.dh_plan_create(ctypes.byref(h), 48, 64, 785e-9, 0.35, 20e-6, 32) == 2
    assert lib.dh_plan_create(ctypes.byref(h), 64, 8192, 785e-9, 0.35, 20e-6, 32) == 2
    assert lib.dh_plan_create(ctypes.byref(h), 64, 64, 785e-9, 0.35, 20e-6, 24) == 2
    assert lib.dh_plan_create(ctypes.byref(h), 64, 64, -1.0, 0.35, 20e-6, 32) == 1
    assert lib.dh_plan_create(ctypes.byref(h), 64, 64, 785e-9, float("nan"), 20e-6, 32) == 1
    lib.dh_destroy(None)  # NULL-safe


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle (test infrastructure) and has no CPU path."""
    pkg = os.path.join(ROOT, "paper_2004_00923_b300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "dh_oracle" not in src, fn
