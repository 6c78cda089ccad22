"""The dynamic update at scale: 50,000,000 pages and about 600,000,000 links
(int32 CSR), FP32 fluid with FP64 history, tol 1e-9 (Section 3.5, Theorem
update).

At this size the oracle cannot solve the graph, so the checks are the
properties that hold at any size and node-by-node values the oracle's
arithmetic gives directly:
* the returned history is certified: the FP64 residual (1-d) Z + d P H - H of
  the returned H, computed independently of the library (FP64 index_add over
  the exported links), has |r|_1 / (1-d) <= tol (Theorem 1);
* the returned F is that residual (Eq. HnFn), checked in full and, node by
  node, by a plain CPU sum over the in-links of 2,000 sampled pages;
* the update path (inject d (P' - P) H, re-converge) and a from-scratch solve
  on P' agree to 2 tol in L1 (both are within tol of the unique x').
"""
import math

import numpy as np
import pytest

from paper_1501_06350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.85
TOL = 1e-9
N = 50_000_000
DRAWS = 1_050_000_000      # about 600 M distinct links after the builders' merge


@pytest.fixture(scope="module")
def di():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_06350_gb300 import build as b
    b.build()
    from paper_1501_06350_gb300 import di as m
    return m


def _residual(ptr, idx, H):
    """r = (1-d)/n + d P H - H in FP64 on the device (plain index_add)."""
    n = ptr.numel() - 1
    deg = (ptr[1:] - ptr[:-1]).to(torch.float64)
    share = torch.where(deg > 0, H / deg.clamp(min=1.0), torch.zeros_like(H))
    src = torch.repeat_interleave(torch.arange(n, device=H.device), ptr[1:] - ptr[:-1], output_size=idx.numel())
    PH = torch.zeros_like(H).index_add_(0, idx.to(torch.int64), share[src])
    del src
    return (1.0 - D) / n + D * PH - H


def _sampled_residual(ptr, idx, H, nodes):
    """The same residual node by node on the CPU, from the in-links of `nodes`."""
    ptr, idx, H = ptr.cpu().numpy(), idx.cpu().numpy(), H.cpu().numpy()
    n = len(ptr) - 1
    deg = np.diff(ptr)
    flag = np.zeros(n, dtype=bool)
    flag[nodes] = True
    e = np.nonzero(flag[idx])[0]
    src = np.searchsorted(ptr, e, side="right") - 1
    out = {}
    for i in nodes:
        out[int(i)] = (1.0 - D) / n - float(H[i])
    for s, t in zip(src, idx[e]):
        out[int(t)] += D * float(H[s]) / float(deg[s])
    return out


def test_update_at_scale(di):
    ptr, idx = synth.web_graph_device(N, DRAWS)
    G = di.Graph(N, ptr, idx)
    del ptr, idx
    torch.cuda.empty_cache()
    nnz = G.nnz
    assert 5.0e8 < nnz < 7.5e8
    st = di.State(G)
    H0, info0 = st.solve(D, tol=TOL, precision=1)
    assert info0["converged"]
    cp, ci, _ = G.export_csr(device=True, weights=False)
    src, dst, op = synth.edge_batch_device(cp, ci, N, 0.01, 5)
    del cp, ci
    st.update_edges(src, dst, op)
    H1, info1 = st.resume(tol=TOL, precision=1)
    assert info1["converged"]
    # certificate of the update path, independent of the library's kernels
    cp, ci, _ = G.export_csr(device=True, weights=False)
    Hs, Fs, _ = st.export(device=True)
    r = _residual(cp, ci, Hs)
    rl1 = float(r.abs().sum())
    assert rl1 / (1 - D) <= TOL * (1 + 1e-6)
    assert float((r - Fs).abs().sum()) <= 1e-12
    # node by node on the CPU at sampled pages
    nodes = np.sort(np.random.default_rng(3).choice(N, size=2000, replace=False))
    ref = _sampled_residual(cp, ci, Hs, nodes)
    Fh = Fs.cpu().numpy()
    assert max(abs(ref[int(i)] - Fh[i]) for i in nodes) <= 1e-16
    del r
    # a from-scratch solve on P' reaches the same x' (both within tol)
    st2 = di.State(G)
    H2, info2 = st2.solve(D, tol=TOL, precision=1)
    assert info2["converged"]
    assert float((H1 - H2).abs().sum()) <= 2 * TOL
    assert info1["edge_pushes"] < info2["edge_pushes"]
