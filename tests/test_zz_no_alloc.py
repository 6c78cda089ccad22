"""The allocation-free |v|_1 entry point (for callers that must not allocate
device memory, e.g. a serving loop whose memory is fully reserved by its own
pool) gives the same result as the allocating entry point di_residual_l1,
call after call, through the C ABI.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1501_06350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_06350_gb300 import build as b
    b.build()
    from paper_1501_06350_gb300 import _lib
    return _lib


def _graph(L, n):
    g = synth.small_graph(n, 3 * n, 21)
    h = ctypes.c_void_p()
    L.check(L.lib().di_graph_create(n, g.nnz, g.ptr.ctypes.data_as(ctypes.c_void_p),
                                    g.idx.ctypes.data_as(ctypes.c_void_p), None, L.DI_W_NONE,
                                    L.DI_LAYOUT_CSR, L.DI_MEM_HOST, None, ctypes.byref(h)),
            "di_graph_create")
    return h


@pytest.mark.parametrize("n", [1, 3000, 250_001])
def test_noalloc_matches_allocating_entry_point(lib, n):
    L = lib
    h = _graph(L, n)
    try:
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for seed in (1, 2):                      # two calls in a row, different data
            v = torch.from_numpy(np.random.default_rng(seed).standard_normal(n)).cuda()
            ptr = ctypes.c_void_p(v.data_ptr())
            ref, got = ctypes.c_double(), ctypes.c_double()
            L.check(L.lib().di_residual_l1(h, ptr, ctypes.byref(ref), L.DI_MEM_DEVICE, stream),
                    "di_residual_l1")
            L.check(L.lib().di_residual_l1_noalloc(h, ptr, ctypes.byref(got), stream),
                    "di_residual_l1_noalloc")
            exact = math.fsum(np.abs(v.cpu().numpy()))
            # same kernel, same fixed summation order: the same double
            assert got.value == ref.value
            assert abs(got.value - exact) <= n * 2.3e-16 * exact
    finally:
        L.lib().di_graph_destroy(h)


def test_noalloc_refuses_host_vectors(lib):
    # a host vector is refused on the host (DI_ERR_INVALID_ARG); nothing is launched
    L = lib
    n = 3000
    h = _graph(L, n)
    try:
        v = np.random.default_rng(3).standard_normal(n)
        out = ctypes.c_double(-1.0)
        rc = L.lib().di_residual_l1_noalloc(h, v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out), None)
        assert rc == L.DI_ERR_INVALID_ARG and out.value == -1.0
        pinned = torch.from_numpy(v).pin_memory()
        rc = L.lib().di_residual_l1_noalloc(h, ctypes.c_void_p(pinned.data_ptr()), ctypes.byref(out), None)
        assert rc == L.DI_ERR_INVALID_ARG and out.value == -1.0
    finally:
        L.lib().di_graph_destroy(h)


def test_noalloc_rejects_graphs_beyond_its_scratch(lib):
    L = lib
    n = (1 << 16) * 2048 + 1                     # one node past the static scratch
    ptr = np.zeros(n + 1, dtype=np.int64)
    h = ctypes.c_void_p()
    L.check(L.lib().di_graph_create(n, 0, ptr.ctypes.data_as(ctypes.c_void_p), None, None,
                                    L.DI_W_NONE, L.DI_LAYOUT_CSR, L.DI_MEM_HOST, None,
                                    ctypes.byref(h)), "di_graph_create")
    try:
        dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
        out = ctypes.c_double()
        rc = L.lib().di_residual_l1_noalloc(h, ctypes.c_void_p(dummy.data_ptr()), ctypes.byref(out),
                                            None)
        assert rc == L.DI_ERR_INVALID_ARG
    finally:
        L.lib().di_graph_destroy(h)
