"""The seeded input generators (no method arithmetic in them): shapes, seeds and
the structural facts the GPU tests rely on."""
import numpy as np
import pytest

from paper_1501_06350_gb300 import synth


def test_seed_set_batch_columns_are_distributions():
    Z = synth.seed_set_batch(5000, 64, 1)
    assert Z.shape == (5000, 64)
    assert np.allclose(Z.sum(axis=0), 1.0, rtol=0, atol=1e-12)
    k = (Z > 0).sum(axis=0)
    assert k.min() >= 1 and k.max() <= 1000
    # each column uniform over its seeds
    for c in range(64):
        col = Z[:, c]
        assert np.all(col[col > 0] == col[col > 0][0])
    assert np.array_equal(Z, synth.seed_set_batch(5000, 64, 1))


def test_union_is_block_diagonal():
    gs = [synth.small_graph(n, 4 * n, 30 + n) for n in (17, 1, 40, 5)]
    u, offs, Z = synth.union(gs)
    assert u.n == sum(g.n for g in gs) and list(offs) == [0, 17, 18, 58, 63]
    src = np.repeat(np.arange(u.n), np.diff(u.ptr))
    for k, g in enumerate(gs):
        a, b = offs[k], offs[k + 1]
        rows = (src >= a) & (src < b)
        assert np.all((u.idx[rows] >= a) & (u.idx[rows] < b))          # links stay inside
        assert np.array_equal(u.idx[rows] - a, g.idx)                   # in the same order
        assert np.allclose(Z[a:b], 1.0 / g.n)
    assert abs(Z.sum() - len(gs)) < 1e-12


def test_small_web_graphs_sizes():
    gs = synth.small_web_graphs(6, 1_000, 3_000, 8.0, 3)
    for g in gs:
        assert 1_000 <= g.n <= 3_000
        assert abs(g.nnz - 8 * g.n) <= 0.02 * 8 * g.n
        assert g.idx.min() >= 0 and g.idx.max() < g.n


def test_device_generator_on_cpu():
    torch = pytest.importorskip("torch")
    n = 100_000
    ptr, idx = synth.web_graph_device(n, 1_200_000, device="cpu")
    p2, i2 = synth.web_graph_device(n, 1_200_000, device="cpu")
    assert torch.equal(ptr, p2) and torch.equal(idx, i2)               # seeded
    deg = (ptr[1:] - ptr[:-1]).numpy()
    assert ptr[0] == 0 and np.all(deg >= 0) and int(ptr[-1]) == len(idx)
    assert abs((deg == 0).mean() - 0.15) < 0.01                          # dangling share
    assert idx.dtype == torch.int32 and int(idx.min()) >= 0 and int(idx.max()) < n
    src = np.repeat(np.arange(n), deg)
    assert (src == idx.numpy()).mean() < 1e-3                           # self-links only in 1-page hosts
    s, d, o = synth.edge_batch_device(ptr, idx, n, 0.01, 2)
    m = int(ptr[-1])
    assert len(s) == max(1, round(0.01 * m)) and int((o == -1).sum()) == len(s) // 2
    dl = (o == -1).numpy()
    present = set(zip(src.tolist(), idx.numpy().tolist()))
    assert all((int(a), int(b)) in present for a, b in zip(s.numpy()[dl][:200], d.numpy()[dl][:200]))
    assert bool((s != d).all())
