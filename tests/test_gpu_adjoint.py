"""Parity of the adjoint (backward pass) with the CPU oracle.

lambda solves (I - d P)^T lambda = g.  The GPU computes it by diffusion on the
reverse graph and certifies |lambda - H|_inf <= |F|_inf / (1 - d) (rows of P^T
sum to at most 1); the oracle by Jacobi sweeps of the Neumann series to 1e-14.
Tolerances: lambda to the GPU's certified bound plus the oracle's; dL/dZ is
(1 - d) lambda; dL/dw per link against the oracle's formula evaluated on the
oracle's x and lambda, within what the two bounds allow
(|d x_j / W_j| (|d_lambda_k| + |d_(P^T lambda)_j|) <= 2 x_j / W_j tol plus the
x error), and against central finite differences (h = 1e-6) of g . x(w)
computed with dense solves on a 1,000-node graph.
"""
import functools

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
    if key == "pa10k":
        return synth.pa_graph(n=10_000, m_target=100_000)
    if key == "web_w":
        return synth.web_graph(n=30_000, m_target=300_000, weighted="lognormal32", seed_offset=14)
    if key == "web200k_w":
        return synth.web_graph(n=200_000, m_target=2_000_000, weighted="lognormal32", seed_offset=15)
    if key == "web1k_w":
        return synth.web_graph(n=1_000, m_target=8_000, weighted="lognormal32", seed_offset=16)
    raise KeyError(key)


@functools.lru_cache(maxsize=None)
def canon(key):
    g = graph(key)
    return oracle.canonical_csr(g.n, g.ptr, g.idx, g.w)


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def _gvec(n, seed):
    return np.random.default_rng(1000 + seed).standard_normal(n)


@pytest.mark.parametrize("key", ["pa10k", "web_w", "web200k_w"])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_adjoint_matches_oracle(di, key, use_graph):
    g = graph(key)
    cp, ci, cw = canon(key)
    G = di.Graph(g.n, g.ptr, g.idx, g.w)
    gv = _gvec(g.n, 1)
    tol = 1e-11
    x, xi, _ = di.solve(G, D, tol=1e-12)
    lam, gz, gw, info = di.adjoint(G, D, gv, x, tol=tol, use_graph=use_graph)
    assert info["converged"] and info["bound"] <= tol
    lam_o, _ = oracle.adjoint(g.n, cp, ci, cw, D, gv, tol=1e-14)
    lam_g = _np(lam)
    assert np.abs(lam_g - lam_o).max() <= info["bound"] + 1e-14 + 1e-15 * np.abs(lam_o).max()
    # dL/dZ = (1 - d) lambda
    assert np.array_equal(_np(gz), (1.0 - D) * lam_g)
    # dL/dw against the oracle's formula on the oracle's x and lambda
    x_o, _, _, _ = oracle.di_solve(g.n, cp, ci, cw, D, tol=1e-14)
    gw_o = oracle.grad_w(g.n, cp, ci, cw, D, x_o, lam_o)
    src = np.repeat(np.arange(g.n), np.diff(cp))
    W = np.diff(cp).astype(np.float64)
    if cw is not None:
        W = np.zeros(g.n)
        np.add.at(W, src, cw)
    xerr = xi["bound"] + 1e-14 / (1 - D)          # |x_gpu - x|_inf <= |x_gpu - x|_1
    lam_max = np.abs(lam_o).max() + tol
    per_link = (2 * D * tol * x_o[src] + 2 * xerr * lam_max) / W[src]
    assert np.all(np.abs(_np(gw) - gw_o) <= per_link * 1.01 + 1e-15 * np.abs(gw_o).max())


def test_adjoint_duality_on_gpu(di):
    """g . x = (1 - d) lambda . Z with both sides from the GPU."""
    g = graph("web_w")
    G = di.Graph(g.n, g.ptr, g.idx, g.w)
    Z = synth.random_z(g.n, 5)
    gv = _gvec(g.n, 2)
    x, _, _ = di.solve(G, D, Z=Z, tol=1e-13)
    lam, _, _, info = di.adjoint(G, D, gv, tol=1e-13, want_grad_w=False)
    lhs = float(gv @ _np(x))
    rhs = (1 - D) * float(_np(lam) @ Z)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs) + 1e-12


def test_adjoint_finite_differences_1k(di):
    """dL/dw and dL/dZ on a 1,000-page weighted graph against central finite
    differences (h = 1e-6) of g . x(w, Z) with x from dense solves."""
    g = graph("web1k_w")
    cp, ci, cw = canon("web1k_w")
    n = g.n
    G = di.Graph(n, cp, ci, cw)
    rng = np.random.default_rng(3)
    gv = rng.standard_normal(n)
    Z = synth.random_z(n, 6)
    x, _, _ = di.solve(G, D, Z=Z, tol=1e-14)
    lam, gz, gw, info = di.adjoint(G, D, gv, x, tol=1e-14)
    assert info["converged"]
    gw = _np(gw)

    def loss(w, z):
        return float(gv @ oracle.dense_solution(n, cp, ci, w, D, z))

    h = 1e-6
    for e in rng.choice(len(cw), size=24, replace=False):
        wp, wm = cw.copy(), cw.copy()
        wp[e] += h
        wm[e] -= h
        fd = (loss(wp, Z) - loss(wm, Z)) / (2 * h)
        assert abs(fd - gw[e]) <= 1e-7 * np.abs(gw).max() + 1e-10
    for i in rng.choice(n, size=8, replace=False):
        zp, zm = Z.copy(), Z.copy()
        zp[i] += h
        zm[i] -= h
        fd = (loss(cw, zp) - loss(cw, zm)) / (2 * h)
        assert abs(fd - _np(gz)[i]) <= 1e-7 * np.abs(_np(gz)).max() + 1e-10


def test_autograd_function(di):
    g = graph("web1k_w")
    cp, ci, cw = canon("web1k_w")
    n = g.n
    w = torch.tensor(cw, dtype=torch.float32, device="cuda", requires_grad=True)
    Z = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda", requires_grad=True)
    ptr = torch.from_numpy(cp).cuda()
    idx = torch.from_numpy(ci).cuda()
    x = di.pagerank(w, Z, n, ptr, idx, D, 1e-13, 1e-13)
    gv = torch.from_numpy(np.random.default_rng(9).standard_normal(n)).cuda()
    (x * gv).sum().backward()
    w64 = w.detach().double().cpu().numpy()
    x_o = oracle.dense_solution(n, cp, ci, w64, D, Z.detach().cpu().numpy())
    assert np.abs(x.detach().cpu().numpy() - x_o).sum() <= 1e-12
    lam_o, _ = oracle.adjoint(n, cp, ci, w64, D, gv.cpu().numpy(), tol=1e-15)
    gw_o = oracle.grad_w(n, cp, ci, w64, D, x_o, lam_o)
    assert w.grad.dtype == torch.float32 and Z.grad.dtype == torch.float64
    assert np.abs(w.grad.cpu().numpy() - gw_o).max() <= 1e-6 * np.abs(gw_o).max()
    assert np.abs(Z.grad.cpu().numpy() - (1 - D) * lam_o).max() <= 1e-12 * np.abs(lam_o).max()
    # a non-canonical CSR (two links of a row swapped) is refused
    j = int(np.nonzero(np.diff(cp) >= 2)[0][0])
    bad = idx.clone()
    a = int(cp[j])
    bad[a], bad[a + 1] = idx[a + 1], idx[a]
    with pytest.raises(ValueError):
        di.pagerank(w, Z, n, ptr, bad)


def test_adjoint_after_update(di):
    g = graph("pa10k")
    cp, ci, _ = canon("pa10k")
    G = di.Graph(g.n, g.ptr, g.idx)
    st = di.State(G)
    st.solve(D, tol=1e-9)
    gv = _gvec(g.n, 4)
    di.adjoint(G, D, gv, tol=1e-10, want_grad_w=False)        # builds the reverse graph
    src, dst, op = synth.edge_batch(cp, ci, g.n, 0.02, 8)
    st.update_edges(src, dst, op)
    qp, qi, _ = oracle.apply_batch(g.n, cp, ci, None, src, dst, op)
    lam, _, _, info = di.adjoint(G, D, gv, tol=1e-11, want_grad_w=False)
    lam_o, _ = oracle.adjoint(g.n, qp, qi, None, D, gv, tol=1e-14)
    assert np.abs(_np(lam) - lam_o).max() <= info["bound"] + 1e-13


def test_adjoint_degenerate_graphs(di):
    # no links: lambda = g exactly; 2051-cycle with constant g: lambda = g / (1 - d)
    n = 3000
    G = di.Graph(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
    gv = _gvec(n, 5)
    lam, _, _, info = di.adjoint(G, D, gv, tol=1e-12, want_grad_w=False)
    assert np.array_equal(_np(lam), gv)
    n = 2051
    G = di.Graph(n, np.arange(n + 1, dtype=np.int64), ((np.arange(n) + 1) % n).astype(np.int32))
    lam, _, _, info = di.adjoint(G, D, np.full(n, 0.7), tol=1e-12, want_grad_w=False)
    assert info["converged"] and np.abs(_np(lam) - 0.7 / (1 - D)).max() <= 1e-12


def test_adjoint_not_converged_and_invalid(di):
    from paper_1501_06350_gb300 import _lib as L
    g = graph("pa10k")
    G = di.Graph(g.n, g.ptr, g.idx)
    gv = _gvec(g.n, 6)
    lam, _, _, info = di.adjoint(G, D, gv, tol=1e-12, max_sweeps=2, want_grad_w=False)
    assert not info["converged"] and info["sweeps"] == 2
    with pytest.raises(L.DIError):
        di.adjoint(G, D, gv, tol=1e-12, precision=1, want_grad_w=False)
    bad = gv.copy()
    bad[5] = np.inf
    with pytest.raises(L.DIError):
        di.adjoint(G, D, bad, tol=1e-12, want_grad_w=False)
    with pytest.raises(L.DIError):
        di.adjoint(G, 1.0, gv, tol=1e-12, want_grad_w=False)
    # grad_w needs x
    rc = L.lib().di_adjoint(G.handle, D, gv.ctypes.data_as(L.P), None, 1e-9, None, None, None,
                            np.zeros(G.nnz).ctypes.data_as(L.P), None, L.DI_MEM_HOST, None)
    assert rc == L.DI_ERR_INVALID_ARG


@functools.lru_cache(maxsize=None)
def web2m_w():
    return synth.cached(synth.web_graph, n=2_000_000, m_target=20_000_000, weighted="lognormal32",
                        seed_offset=4)


def test_adjoint_full_size(di):
    """The 2M-page / 20M-link weighted web graph (FP32 lognormal weights):
    lambda against the oracle's Jacobi solution in the infinity norm."""
    g = web2m_w()
    G = di.Graph(g.n, g.ptr, g.idx, g.w)
    cp, ci, cw = oracle.canonical_csr(g.n, g.ptr, g.idx, g.w)
    gp_, gi_, gw_ = G.export_csr()
    assert np.array_equal(_np(gp_), cp) and np.array_equal(_np(gi_), ci) and np.array_equal(_np(gw_), cw)
    gv = np.random.default_rng(11).standard_normal(g.n)
    x, _, _ = di.solve(G, D, tol=1e-10)
    lam, gz, gw, info = di.adjoint(G, D, gv, x, tol=1e-10)
    assert info["converged"] and info["bound"] <= 1e-10
    lam_o, _ = oracle.adjoint(g.n, cp, ci, cw, D, gv, tol=1e-13)
    assert np.abs(_np(lam) - lam_o).max() <= info["bound"] + 1e-13
    assert np.isfinite(_np(gw)).all()
