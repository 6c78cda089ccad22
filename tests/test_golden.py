"""Golden fixtures (tests/golden/*.json, written by tests/golden/make_golden.py
from the oracle's dense solve of x = (1-d)(I - dP)^-1 Z, Section 2.1): the
oracle must still reproduce them (CPU), and every form of the library must
reach them within its certified bound (GPU)."""
import glob
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = sorted(glob.glob(os.path.join(HERE, "*.json")))


def _load(path):
    r = json.load(open(path))
    ptr = np.array(r["ptr"], dtype=np.int64)
    idx = np.array(r["idx"], dtype=np.int32)
    w = None if r["w"] is None else np.array([float.fromhex(v) for v in r["w"]])
    z = np.array([float.fromhex(v) for v in r["z"]])
    x = np.array([float.fromhex(v) for v in r["x"]])
    return r["n"], r["d"], ptr, idx, w, z, x


def test_fixtures_present():
    assert len(FILES) >= 4


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_oracle_reproduces_golden(path):
    n, d, ptr, idx, w, z, x = _load(path)
    cp, ci, cw = oracle.canonical_csr(n, ptr, idx, w)
    xd = oracle.dense_solution(n, cp, ci, cw, d, z)
    assert np.abs(xd - x).sum() <= 1e-13
    H, F, info, _ = oracle.di_solve(n, cp, ci, cw, d, z, tol=1e-13)
    assert np.abs(H - x).sum() <= 2e-13


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_library_reaches_golden(path, precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_06350_gb300 import build as b
    b.build()
    from paper_1501_06350_gb300 import di
    n, d, ptr, idx, w, z, x = _load(path)
    G = di.Graph(n, ptr, idx, w)
    st = di.State(G)
    H, info = st.solve(d, Z=torch.from_numpy(z).cuda(), tol=1e-12, precision=precision)
    assert info["converged"]
    assert np.abs(H.cpu().numpy() - x).sum() <= 1e-12 + 1e-13
