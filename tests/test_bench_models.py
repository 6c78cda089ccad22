"""The byte model of a link update and the error report of bench.py (host
logic, CPU): hand-counted cases, and the model's new degrees against the CSR
that the oracle builds from the same batch."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_1501_06350_gb300 import synth  # noqa: E402


def test_update_bytes_hand_counted():
    # rows: 0 -> {1, 2}, 1 -> {2}, 2 -> {}, 3 -> {0, 1, 2}
    cp = np.array([0, 2, 3, 3, 6], dtype=np.int64)
    # delete 0->1, insert 2->3, insert 0->3: rows 0 and 2 change
    src = np.array([0, 2, 0], dtype=np.int32)
    op = np.array([-1, 1, 1], dtype=np.int8)
    b = bench.update_bytes(cp, 4, src, op)
    # old degrees 2 1 0 3 (6 links), new 2 1 1 3 (7 links), 5 row pointers each
    assert b["csr"] == 4 * 6 + 4 * 5 + 4 * 7 + 4 * 5
    # two changed columns: 8 B of H each, 12 B per old (2 + 0) and new (2 + 1) link
    assert b["inject"] == 8 * 2 + 12 * 2 + 12 * 3
    assert b["batch"] == 9 * 3
    assert b["total"] == b["csr"] + b["inject"] + b["batch"]
    assert b["changed_columns"] == 2 and b["injected_links"] == 5


@pytest.mark.parametrize("seed", range(3))
def test_update_bytes_degrees_match_the_applied_batch(seed):
    g = synth.pa_graph(n=500, m_target=3000)
    cp, ci, _ = oracle.canonical_csr(g.n, g.ptr, g.idx)
    src, dst, op = synth.exact_batch(cp, ci, g.n, 0.05, seed)
    qp, _, _ = oracle.apply_batch(g.n, cp, ci, None, src, dst, op)
    b = bench.update_bytes(cp, g.n, src, op)
    nnz_new = int(qp[-1])
    touched = np.unique(src.astype(np.int64))
    old = np.diff(cp)[touched].sum()
    new = np.diff(qp)[touched].sum()
    assert b["csr"] == 4 * int(cp[-1]) + 4 * (g.n + 1) + 4 * nnz_new + 4 * (g.n + 1)
    assert b["injected_links"] == old + new
    assert b["inject"] == 8 * len(touched) + 12 * (old + new)


def test_error_report():
    e = bench.error_vs_oracle(np.array([1.0, 2.0, 3.0]), np.array([1.0, 2.5, 2.0]))
    assert e["err_l1_vs_oracle"] == pytest.approx(1.5)
    assert e["max_rel_err_vs_oracle"] == pytest.approx(0.5)
