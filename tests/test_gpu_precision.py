"""Parity of the FP32-fluid form (iterative refinement) with the CPU oracle.

The FP32 form moves the fluid in FP32 and keeps H, the residual and the stop
test in FP64: after every cycle of FP32 sweeps, the fluid taken in the cycle
(D, summed exactly in FP64) is added to H and the FP64 fluid becomes the
exact residual F + d P D - D, which is (1-d) Z + d P H - H by Eq. HnFn.  So the
same bars as for the plain form apply: x to 1e-9 in L1 against the oracle
(run to 1e-13 or tighter), the certified bound |x - H|_1 <= |F|_1 / (1 - d)
(Theorem 1, Eq. SL), and the returned F equal to the residual of the returned
H recomputed on the CPU in FP64 (<= 1e-13 in L1).
"""
import functools
import math

import numpy as np
import pytest

import oracle
from paper_1501_06350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.85
F32 = dict(precision=1)


@pytest.fixture(scope="module")
def di():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_06350_gb300 import build as b
    b.build()
    from paper_1501_06350_gb300 import di as m
    return m


@functools.lru_cache(maxsize=None)
def graph(key):
    if key == "pa10k":
        return synth.pa_graph(n=10_000, m_target=100_000)
    if key == "web200k":
        return synth.web_graph(n=200_000, m_target=2_000_000, seed_offset=12)
    if key == "web_w":
        return synth.web_graph(n=30_000, m_target=300_000, weighted="lognormal32", seed_offset=14)
    raise KeyError(key)


@functools.lru_cache(maxsize=None)
def canon(key):
    g = graph(key)
    return oracle.canonical_csr(g.n, g.ptr, g.idx, g.w)


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def _x(key, Z=None, tol=1e-13):
    cp, ci, cw = canon(key)
    H, _, info, _ = oracle.di_solve(graph(key).n, cp, ci, cw, D, Z, tol=tol)
    return H


@functools.lru_cache(maxsize=None)
def _x_cached(key, tol):
    return _x(key, tol=tol)


def _check_state(st, key, Z=None, tol=1e-13):
    """Returned F is the exact FP64 residual of the returned H (Eq. HnFn)."""
    g = graph(key)
    cp, ci, cw = canon(key)
    Hs, Fs, _ = st.export()
    r = oracle.residual(g.n, cp, ci, cw, D, Z, Hs)
    assert np.abs(r - Fs).sum() <= tol
    return Hs, Fs, r


@pytest.mark.parametrize("key", ["pa10k", "web200k", "web_w"])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_f32_solve_matches_oracle(di, key, use_graph):
    g = graph(key)
    G = di.Graph(g.n, g.ptr, g.idx, g.w)
    st = di.State(G)
    tol = 1e-10 / (1 - D)
    H, info = st.solve(D, tol=tol, use_graph=use_graph, **F32)
    assert info["converged"] and info["resid_l1"] <= 1e-10
    assert info["refinements"] >= 1 and info["refine_links"] > 0
    x = _x_cached(key, 1e-13)
    err = np.abs(_np(H) - x).sum()
    assert err <= 1e-9
    assert err <= info["bound"] + 1e-13 / (1 - D) + 1e-14
    Hs, Fs, r = _check_state(st, key)
    assert np.array_equal(Hs, _np(H))
    assert math.fsum(np.abs(r)) <= 1e-10 * (1 + 1e-9)


def test_f32_per_node_relative(di):
    g = graph("pa10k")
    G = di.Graph(g.n, g.ptr, g.idx)
    H, info, _ = di.solve(G, D, tol=1e-12, **F32)
    x = _x("pa10k", tol=1e-14)
    assert info["converged"]
    assert (np.abs(_np(H) - x) / x).max() <= 1e-6


@pytest.mark.parametrize("ratio", [1e-2, 1e-4, 1e-7])
def test_f32_refine_ratios(di, ratio):
    g = graph("web200k")
    G = di.Graph(g.n, g.ptr, g.idx)
    st = di.State(G)
    H, info = st.solve(D, tol=1e-9, refine_ratio=ratio, **F32)
    assert info["converged"]
    # a cycle gains about 1/ratio, until FP32 rounding limits it
    assert info["refinements"] >= 2 if ratio >= 1e-4 else info["refinements"] >= 1
    assert np.abs(_np(H) - _x_cached("web200k", 1e-12)).sum() <= 1e-9
    _check_state(st, "web200k")


@pytest.mark.parametrize("zkind", ["signed", "seeds"])
def test_f32_teleport_vectors(di, zkind):
    g = graph("web200k")
    n = g.n
    Z = synth.random_z(n, 2, signed=True) if zkind == "signed" else synth.seed_set_z(n, 500, 3)
    G = di.Graph(n, g.ptr, g.idx)
    st = di.State(G)
    H, info = st.solve(D, Z=Z, tol=1e-9, **F32)
    x = _x("web200k", Z=Z, tol=1e-12)
    assert info["converged"]
    assert np.abs(_np(H) - x).sum() <= 1e-9
    _check_state(st, "web200k", Z=Z)


@pytest.mark.parametrize("case", ["single", "single_loop", "all_dangling", "cycle"])
def test_f32_degenerate_graphs(di, case):
    if case == "single":
        n, src, dst = 1, [], []
    elif case == "single_loop":
        n, src, dst = 1, [0], [0]
    elif case == "all_dangling":
        n, src, dst = 3000, [], []
    else:
        n = 2051
        src, dst = list(range(n)), [(i + 1) % n for i in range(n)]
    ptr = np.zeros(n + 1, np.int64)
    np.add.at(ptr, np.array(src, dtype=np.int64) + 1, 1)
    ptr = np.cumsum(ptr)
    G = di.Graph(n, ptr, np.array(dst, np.int32))
    H, info, _ = di.solve(G, D, tol=1e-12, **F32)
    want = {"single": 1 - D, "single_loop": 1.0, "all_dangling": (1 - D) / n, "cycle": 1.0 / n}[case]
    assert info["converged"]
    assert np.abs(_np(H) - want).sum() <= 1e-11


def test_f32_sweep_cap_keeps_exact_state(di):
    """A capped FP32 solve still folds D into H: F is the residual of H."""
    g = graph("pa10k")
    G = di.Graph(g.n, g.ptr, g.idx)
    st = di.State(G)
    H, info = st.solve(D, tol=1e-12, max_sweeps=5, **F32)
    assert not info["converged"] and info["sweeps"] == 5
    _, Fs, _ = _check_state(st, "pa10k")
    assert info["resid_l1"] == pytest.approx(math.fsum(np.abs(Fs)), rel=1e-12)
    H2, info2 = st.resume(tol=1e-10, **F32)
    assert info2["converged"] and np.abs(_np(H2) - _x_cached("pa10k", 1e-13)).sum() <= 1e-9


def test_f32_update_then_resume(di):
    g = graph("pa10k")
    G = di.Graph(g.n, g.ptr, g.idx)
    st = di.State(G)
    st.solve(D, tol=1e-9, **F32)
    cp, ci, _ = canon("pa10k")
    src, dst, op = synth.edge_batch(cp, ci, g.n, 0.01, 5)
    st.update_edges(src, dst, op)
    qp, qi, _ = oracle.apply_batch(g.n, cp, ci, None, src, dst, op)
    H2, info = st.resume(tol=1e-10 / (1 - D), **F32)
    Hx, _, _, _ = oracle.di_solve(g.n, qp, qi, None, D, tol=1e-13)
    assert info["converged"] and np.abs(_np(H2) - Hx).sum() <= 1e-9
    Hs, Fs, _ = st.export()
    r = oracle.residual(g.n, qp, qi, None, D, None, Hs)
    assert np.abs(r - Fs).sum() <= 1e-13


def test_f32_and_f64_states_interchange(di):
    """An FP64 solve resumed in FP32 and the reverse reach the same x."""
    g = graph("web_w")
    G = di.Graph(g.n, g.ptr, g.idx, g.w)
    a = di.State(G)
    a.solve(D, tol=1e-4)
    Ha, ia = a.resume(tol=1e-10, **F32)
    b = di.State(G)
    b.solve(D, tol=1e-4, **F32)
    Hb, ib = b.resume(tol=1e-10)
    x = _x_cached("web_w", 1e-13)
    assert ia["converged"] and ib["converged"]
    assert np.abs(_np(Ha) - x).sum() <= 1e-9 and np.abs(_np(Hb) - x).sum() <= 1e-9


def test_f32_invalid_ratio(di):
    from paper_1501_06350_gb300 import _lib as L
    g = graph("pa10k")
    G = di.Graph(g.n, g.ptr, g.idx)
    st = di.State(G)
    for r in (0.0, 1.0, -1.0, float("nan")):
        with pytest.raises(L.DIError):
            st.solve(D, refine_ratio=r, **F32)
    with pytest.raises(L.DIError):
        st.solve(D, precision=2)


@functools.lru_cache(maxsize=None)
def web4m():
    return synth.cached(synth.web_graph, n=4_000_000, m_target=40_000_000)


def test_f32_full_size_web_graph(di):
    """The 4M-page / 40M-link web graph in the benchmark's launch configuration:
    the FP32 form's H certified by the exact FP64 residual recomputed on the CPU
    and compared with the oracle's x."""
    g = web4m()
    G = di.Graph(g.n, g.ptr, g.idx)
    st = di.State(G)
    H, info = st.solve(D, tol=1e-9, **F32)
    assert info["converged"]
    Hs, Fs, _ = st.export()
    cp, ci, _ = oracle.canonical_csr(g.n, g.ptr, g.idx)
    gp_, gi_, _ = G.export_csr()
    assert np.array_equal(_np(gp_), cp) and np.array_equal(_np(gi_), ci)
    r = oracle.residual(g.n, cp, ci, None, D, None, Hs)
    assert math.fsum(np.abs(r)) / (1 - D) <= 1e-9 * (1 + 1e-6)
    assert np.abs(r - Fs).sum() <= 1e-12
    x, _, _, _ = oracle.di_solve(g.n, cp, ci, None, D, tol=1e-12)
    assert np.abs(_np(H) - x).sum() <= 1e-9
