"""Parity of the batched personalised solve (B teleport vectors at once) and of
uneven independent graphs solved as one union, with the CPU oracle.

Every column c is a separate PageRank problem x_c = d P x_c + (1-d) Z_c
(Section 2.1): the bar is the single solve's — x_c to 1e-9 in L1 against the
oracle (run to 1e-12), and the returned per-column residual equal to the
oracle's exact FP64 residual of the returned H_c (Eq. HnFn) with
|r_c|_1 / (1-d) <= tol (Theorem 1).  For the union of independent graphs the
solution restricted to each component is that component's own solution.
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
    if key == "web50k":
        return synth.web_graph(n=50_000, m_target=500_000, seed_offset=21)
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


def _check_columns(key, Z, H, res, cols, tol, x_tol=1e-12):
    g = graph(key)
    cp, ci, cw = canon(key)
    for c in cols:
        x, _, _, _ = oracle.di_solve(g.n, cp, ci, cw, D, Z[:, c], tol=x_tol)
        assert np.abs(H[:, c] - x).sum() <= 1e-9, c
        r = oracle.residual(g.n, cp, ci, cw, D, Z[:, c], H[:, c])
        rl1 = math.fsum(np.abs(r))
        assert rl1 / (1 - D) <= tol * (1 + 1e-9), c
        assert abs(rl1 - res[c]) <= 1e-14 + 1e-6 * rl1, c


@pytest.mark.parametrize("use_graph", [1, 0])
def test_batch_64_seed_sets(di, use_graph):
    g = graph("web50k")
    Z = synth.seed_set_batch(g.n, 64, 1)
    G = di.Graph(g.n, g.ptr, g.idx)
    H, res, info = di.solve_batch(G, Z, D, tol=1e-9, use_graph=use_graph)
    assert info["converged"] and info["refinements"] >= 1
    _check_columns("web50k", Z, _np(H), _np(res), range(64), 1e-9)


def test_batch_larger_graph_sampled_columns(di):
    g = graph("web200k")
    Z = synth.seed_set_batch(g.n, 64, 2)
    G = di.Graph(g.n, g.ptr, g.idx)
    H, res, info = di.solve_batch(G, Z, D, tol=1e-9)
    assert info["converged"]
    _check_columns("web200k", Z, _np(H), _np(res), [0, 17, 38, 63], 1e-9)
    assert (_np(res) / (1 - D) <= 1e-9 * (1 + 1e-12)).all()


@pytest.mark.parametrize("B", [1, 5, 33])
def test_batch_fewer_columns_and_host_memory(di, B):
    g = graph("web50k")
    Z = synth.seed_set_batch(g.n, B, 3)
    Z[:, 0] = 1.0 / g.n                      # one uniform column
    G = di.Graph(g.n, g.ptr, g.idx)
    H, res, info = di.solve_batch(G, Z, D, tol=1e-9, device=False)
    assert H.shape == (g.n, B) and res.shape == (B,)
    _check_columns("web50k", Z, H, res, range(min(B, 6)), 1e-9)
    # the uniform column equals the single solve's answer within both bounds
    x1, i1, _ = di.solve(G, D, tol=1e-10)
    assert np.abs(H[:, 0] - _np(x1)).sum() <= 1e-9 + i1["bound"]


def test_batch_weighted_and_zero_column(di):
    g = graph("web_w")
    Z = synth.seed_set_batch(g.n, 16, 4)
    Z[:, 9] = 0.0                             # an empty problem: x = 0 exactly
    G = di.Graph(g.n, g.ptr, g.idx, g.w)
    H, res, info = di.solve_batch(G, Z, D, tol=1e-10)
    H = _np(H)
    assert info["converged"]
    assert np.array_equal(H[:, 9], np.zeros(g.n)) and _np(res)[9] == 0.0
    _check_columns("web_w", Z, H, _np(res), [0, 5, 15], 1e-10, x_tol=1e-13)


def test_batch_degenerate_graphs(di):
    n = 3000                                  # all dangling: x = (1 - d) Z
    G = di.Graph(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
    Z = synth.seed_set_batch(n, 8, 5)
    H, res, info = di.solve_batch(G, Z, D, tol=1e-12)
    assert np.abs(_np(H) - (1 - D) * Z).max() <= 1e-15
    G1 = di.Graph(1, np.array([0, 1], np.int64), np.array([0], np.int32))   # one self-loop
    H1, _, _ = di.solve_batch(G1, np.array([[1.0, 0.5]]), D, tol=1e-13)
    assert np.abs(_np(H1) - np.array([[1.0, 0.5]])).max() <= 1e-12


def test_batch_cap_and_invalid(di):
    from paper_1501_06350_gb300 import _lib as L
    g = graph("web50k")
    G = di.Graph(g.n, g.ptr, g.idx)
    Z = synth.seed_set_batch(g.n, 4, 6)
    _, _, info = di.solve_batch(G, Z, D, tol=1e-12, max_sweeps=3)
    assert not info["converged"]
    for bad in (np.zeros((g.n, 0)), np.zeros((g.n, 65))):
        with pytest.raises(L.DIError):
            di.solve_batch(G, bad, D)
    Zn = Z.copy()
    Zn[7, 2] = np.nan
    with pytest.raises(L.DIError):
        di.solve_batch(G, Zn, D)


def test_union_of_uneven_graphs(di):
    """Independent graphs of uneven sizes as one block-diagonal union, solved in
    one launch of the sweep loop (FP32 form): each component matches its own
    oracle solution and its own residual is within the bound."""
    gs = synth.small_web_graphs(24, 1_000, 20_000, 8.0, 7)
    u, offs, Z = synth.union(gs)
    G = di.Graph(u.n, u.ptr, u.idx)
    st = di.State(G)
    H, info = st.solve(D, Z=Z, tol=1e-9, precision=1)
    assert info["converged"]
    H = _np(H)
    _, F, _ = st.export()
    for k, gk in enumerate(gs):
        a, b = int(offs[k]), int(offs[k + 1])
        cp, ci, _ = oracle.canonical_csr(gk.n, gk.ptr, gk.idx)
        x, _, _, _ = oracle.di_solve(gk.n, cp, ci, None, D, None, tol=1e-12)
        assert np.abs(H[a:b] - x).sum() <= 1e-9, k
        assert math.fsum(np.abs(F[a:b])) / (1 - D) <= 1e-9


@functools.lru_cache(maxsize=None)
def web1m():
    return synth.cached(synth.web_graph, n=1_000_000, m_target=10_000_000, seed_offset=3)


def test_batch_full_size(di):
    """The 1M-page / 10M-link host-structured graph with 64 seed-set teleport
    vectors (1 to 1000 seeds each), as the benchmark runs it."""
    g = web1m()
    Z = synth.seed_set_batch(g.n, 64, 8)
    G = di.Graph(g.n, g.ptr, g.idx)
    H, res, info = di.solve_batch(G, Z, D, tol=1e-9)
    assert info["converged"]
    cp, ci, _ = oracle.canonical_csr(g.n, g.ptr, g.idx)
    gp_, gi_, _ = G.export_csr()
    assert np.array_equal(_np(gp_), cp) and np.array_equal(_np(gi_), ci)
    H = _np(H)
    for c in (0, 31, 63):
        x, _, _, _ = oracle.di_solve(g.n, cp, ci, None, D, Z[:, c], tol=1e-12)
        assert np.abs(H[:, c] - x).sum() <= 1e-9
        r = oracle.residual(g.n, cp, ci, None, D, Z[:, c], H[:, c])
        assert math.fsum(np.abs(r)) / (1 - D) <= 1e-9 * (1 + 1e-9)
