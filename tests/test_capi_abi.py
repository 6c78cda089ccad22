"""The C ABI library loads and exports every entry point include/di.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "di.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(di_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_06350_gb300 import build as b
    b.build()
    from paper_1501_06350_gb300 import _lib
    return _lib


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["di_graph_create", "di_graph_destroy", "di_state_create", "di_solve", "di_resume",
                 "di_update_edges", "di_frontier_select", "di_residual_l1", "di_status_str"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (di_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    # the Python binding covers the same set, with the same names
    assert sorted(lib.SIGNATURES) == _declared()


def test_load_and_host_only_calls(lib):
    L = lib.lib()
    assert L.di_status_str(lib.DI_ERR_NOT_CONVERGED) == b"DI_ERR_NOT_CONVERGED"
    o = lib.default_opts()
    assert o.theta_factor == 1.0 and o.use_graph == 1 and o.max_sweeps == 100000
    # argument checks reject bad input before touching a device
    h = ctypes.c_void_p()
    assert L.di_graph_create(0, 0, None, None, None, 0, 0, 0, None, ctypes.byref(h)) == lib.DI_ERR_INVALID_ARG
    assert L.di_graph_create(4, 0, None, None, None, 0, 0, 0, None, ctypes.byref(h)) == lib.DI_ERR_INVALID_ARG
    assert L.di_solve(None, None, 0.85, None, 1e-9, None, None, None, 0, None) == lib.DI_ERR_INVALID_ARG


def test_product_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_1501_06350_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "liboracle" not in src and "di_oracle" not in src, f
