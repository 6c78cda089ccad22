"""Pins of the oracle's Section 3.3 helpers: the solution for P completed on its
dangling columns (``oracle.completed_solution``) and the fluid lost at dangling
nodes (``oracle.dangling_loss``).

The references are independent of the helpers: exact rational arithmetic on a
completed matrix built from a link dictionary, the closed form of a graph with
no links (a rank-one completion, solved by the Sherman-Morrison identity),
column-stochasticity of the completion, the paper's normalisation factor
(1-d)/(1-d-d t) applied to the separately pinned dense solution, and the mass
balance of Eq. HnFn, in which the C oracle accumulates its loss l at dangling
diffusions by a different route.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1501_06350_gb300 import synth
from tests import _brute as B

D = 0.85


def _graph(pairs, n):
    src = np.array([a for a, _ in pairs], dtype=np.int64)
    dst = np.array([b for _, b in pairs], dtype=np.int32)
    order = np.argsort(src, kind="stable")
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, src + 1, 1)
    return oracle.canonical_csr(n, np.cumsum(ptr), dst[order])


def _exact_completed(n, acc, d, Z):
    """x = (1-d)(I - d P_c)^-1 Z over Fractions, P_c = P with every column of a
    page without out-links replaced by Z (Section 3.3)."""
    d = Fraction(d)
    cnt = {}
    for (a, _b) in acc:
        cnt[a] = cnt.get(a, 0) + 1
    A = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for (a, b) in acc:
        A[b][a] -= d / cnt[a]
    for j in range(n):
        if j not in cnt:                      # dangling column: teleport by Z
            for i in range(n):
                A[i][j] -= d * Z[i]
    M = [A[i] + [(1 - d) * Z[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [vr - f * vc for vr, vc in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


# ------------------------------------------------------ completed_solution
def test_completed_chain_exact():
    # 0 -> 1, page 1 dangling: P_c = [[0, z0], [1, z1]] (orientation matters)
    Zf = [Fraction(1, 4), Fraction(3, 4)]
    d = Fraction(17, 20)
    # by hand: x0 = d z0 x1 + (1-d) z0,  x1 = d x0 + d z1 x1 + (1-d) z1
    # => x1 (1 - d z1 - d^2 z0) = (1-d)(d z0 + z1),  x0 = d z0 x1 + (1-d) z0
    x1 = (1 - d) * (d * Zf[0] + Zf[1]) / (1 - d * Zf[1] - d * d * Zf[0])
    x0 = d * Zf[0] * x1 + (1 - d) * Zf[0]
    cp, ci, _ = _graph([(0, 1)], 2)
    xc = oracle.completed_solution(2, cp, ci, None, D, np.array([0.25, 0.75]))
    assert xc[0] == pytest.approx(float(x0), abs=4e-16)   # a few ulps of LAPACK rounding
    assert xc[1] == pytest.approx(float(x1), abs=4e-16)
    assert x0 + x1 == 1                       # the completed matrix is stochastic


@pytest.mark.parametrize("s", [1.0, 0.6])
def test_completed_no_links_closed_form(s):
    # every column is Z: P_c = Z 1^T, and (I - d Z 1^T)^-1 Z = Z / (1 - d sum Z)
    n = 6
    Z = synth.random_z(n, 3) * s
    cp = np.zeros(n + 1, dtype=np.int64)
    ci = np.zeros(0, dtype=np.int32)
    xc = oracle.completed_solution(n, cp, ci, None, D, Z)
    assert np.abs(xc - (1 - D) * Z / (1 - D * Z.sum())).max() < 4e-16
    if s == 1.0:
        assert np.abs(xc - Z).max() < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_completed_matches_exact_rational(seed):
    n = 7
    rng = np.random.default_rng(600 + seed)
    pairs = sorted({(int(a), int(b)) for a, b in rng.integers(0, n, size=(14, 2)) if a != b and a < n - 2})
    cp, ci, _ = _graph(pairs, n)
    assert (np.diff(cp) == 0).any()          # pages n-2 and n-1 have no out-links
    acc, _, _, _ = B.merged(n, B.links(cp, ci))
    Zf = [Fraction(k + 1, n * (n + 1) // 2) for k in range(n)]
    want = [float(v) for v in _exact_completed(n, acc, Fraction(17, 20), Zf)]
    xc = oracle.completed_solution(n, cp, ci, None, D, np.array([float(z) for z in Zf]))
    assert np.abs(xc - want).sum() < 1e-15
    assert sum(_exact_completed(n, acc, Fraction(17, 20), Zf)) == 1


@pytest.mark.parametrize("seed", range(3))
def test_completed_is_the_papers_normalisation(seed):
    # Section 3.3: x_c = (1-d) / (1-d-d t) x with t = sum of x over dangling pages
    g = synth.pa_graph(n=300 + 100 * seed, m_target=1500)
    cp, ci, _ = oracle.canonical_csr(g.n, g.ptr, g.idx)
    Z = synth.random_z(g.n, seed)
    x = oracle.dense_solution(g.n, cp, ci, None, D, Z)
    t = x[np.diff(cp) == 0].sum()
    assert t > 0
    xc = oracle.completed_solution(g.n, cp, ci, None, D, Z)
    assert np.abs(xc - (1 - D) / (1 - D - D * t) * x).sum() < 1e-13
    assert xc.sum() == pytest.approx(1.0, abs=1e-13)


# ----------------------------------------------------------- dangling_loss
def test_dangling_loss_chain_and_no_dangling():
    cp, ci, _ = _graph([(0, 1)], 2)
    assert oracle.dangling_loss(cp, np.array([0.3, 0.7])) == 0.7   # page 1 has no out-links
    cp, ci, _ = _graph([(0, 1), (1, 0)], 2)
    assert oracle.dangling_loss(cp, np.array([0.3, 0.7])) == 0.0


def test_dangling_loss_no_links():
    n = 5
    Z = synth.random_z(n, 1)
    cp = np.zeros(n + 1, dtype=np.int64)
    ci = np.zeros(0, dtype=np.int32)
    H, F, info, _ = oracle.di_solve(n, cp, ci, None, D, Z, tol=1e-15)
    assert oracle.dangling_loss(cp, H) == pytest.approx((1 - D) * Z.sum(), abs=1e-16)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("cut", [10, 200, 5000])
def test_dangling_loss_closes_the_mass_balance(seed, cut):
    # Eq. HnFn summed over pages: sum F + (1-d) sum H + d l = (1-d) sum Z, where
    # the C oracle adds to its own l at every diffusion of a dangling page
    g = synth.pa_graph(n=400, m_target=2000)
    cp, ci, _ = oracle.canonical_csr(g.n, g.ptr, g.idx)
    Z = synth.random_z(g.n, seed)
    H, F, info, _ = oracle.di_solve(g.n, cp, ci, None, D, Z, tol=1e-300, max_diffusions=cut)
    l = oracle.dangling_loss(cp, H)
    assert l == pytest.approx(info["l_dangling"], rel=1e-13, abs=1e-18)
    assert l == pytest.approx(((1 - D) * Z.sum() - F.sum() - (1 - D) * H.sum()) / D, rel=1e-10, abs=1e-16)
