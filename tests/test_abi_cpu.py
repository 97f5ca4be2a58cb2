"""CPU-side checks of the C ABI boundary (no GPU needed): the CUDA library
builds and loads, exports every entry point that include/cpma.h declares, and
its host-only calls behave; the product package never touches the oracle."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cpma.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cpma_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_05055_gb300 import cpma
    return cpma.lib()


def test_header_declares_the_set_interface():
    names = declared_functions()
    for n in ("cpma_create", "cpma_insert_batch", "cpma_delete_batch", "cpma_has_batch",
              "cpma_range_map", "cpma_size", "cpma_bytes"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_default_config_and_strerror(lib):
    from paper_2305_05055_gb300 import cpma
    c = cpma.default_config()
    assert (c.leaf_bytes, c.tau_leaf, c.tau_root, c.rho_leaf, c.rho_root,
            c.grow_num, c.grow_den, c.build_pm, c.rebuild_pm, c.codec) == (
        512, 900, 700, 100, 300, 6, 5, 500, 0, 0)
    assert lib.cpma_strerror(0) == b"ok"
    assert b"invalid" in lib.cpma_strerror(-1)


def test_null_handle_is_rejected_without_a_gpu(lib):
    v = C.c_uint64()
    assert lib.cpma_size(None, C.byref(v)) == -1
    assert lib.cpma_bytes(None, C.byref(v)) == -1
    assert lib.cpma_insert_batch(None, None, 0, 0, None, None) == -1


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2305_05055_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
                assert "cpma_oracle" not in src, f
