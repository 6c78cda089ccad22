"""Pins of the oracle's adjoint routines (the backward pass of the PageRank
solve; not in the paper).

For L = g . x with x = (1 - d)(I - d P)^-1 Z (Section 2.1), the adjoint lambda
solves (I - d P)^T lambda = g; then dL/dZ = (1 - d) lambda and
dL/dw(j,k) = d x_j / W_j (lambda_k - (P^T lambda)_j) for P[i][j] = w(j,i)/W_j
(Eq. def-p).  The references here are a LAPACK solve of the transposed
system, the duality g . x = (1 - d) lambda . Z, closed forms, and central
finite differences of g . x(w, Z) with x from a dense solve.
"""
import numpy as np
import pytest

import oracle

D = 0.85


def _graph(seed, n, m, weighted):
    rng = np.random.default_rng(900 + seed)
    src = rng.integers(0, n, size=m)
    dst = rng.integers(0, n, size=m)
    src[: n // 10] = n - 1                     # a few repeated links and one busy row
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, src + 1, 1)
    ptr = np.cumsum(ptr)
    w = rng.lognormal(size=m) if weighted else None
    return oracle.canonical_csr(n, ptr, dst.astype(np.int32), w)


def _dense_P(n, cp, ci, w):
    """P[i][j] = w(j,i) / sum of row j, written out link by link."""
    P = np.zeros((n, n))
    for j in range(n):
        row = range(int(cp[j]), int(cp[j + 1]))
        tot = sum(1.0 if w is None else float(w[e]) for e in row)
        for e in row:
            P[int(ci[e]), j] += (1.0 if w is None else float(w[e])) / tot
    return P


def _x(n, cp, ci, w, Z):
    return (1 - D) * np.linalg.solve(np.eye(n) - D * _dense_P(n, cp, ci, w), Z)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("weighted", [False, True])
def test_adjoint_matches_dense_transposed_solve(seed, weighted):
    n = 30 + 20 * seed
    cp, ci, cw = _graph(seed, n, 4 * n, weighted)
    g = np.random.default_rng(seed).standard_normal(n)
    lam, it = oracle.adjoint(n, cp, ci, cw, D, g, tol=1e-14)
    ref = np.linalg.solve((np.eye(n) - D * _dense_P(n, cp, ci, cw)).T, g)
    assert np.abs(lam - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    # stopping bound |lambda - lambda_k|_inf <= tol, here with a loose tol
    lam2, it2 = oracle.adjoint(n, cp, ci, cw, D, g, tol=1e-6)
    assert np.abs(lam2 - ref).max() <= 1e-6 and it2 < it


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_duality(seed):
    n = 60
    cp, ci, cw = _graph(10 + seed, n, 5 * n, True)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(n)
    Z = rng.random(n)
    lam, _ = oracle.adjoint(n, cp, ci, cw, D, g, tol=1e-15)
    x, _, _, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-15)
    assert abs(g @ x - (1 - D) * lam @ Z) <= 1e-12 * abs(g @ x) + 1e-15


def test_adjoint_closed_forms():
    # no links: lambda = g
    g = np.array([0.3, -1.0, 2.0])
    lam, _ = oracle.adjoint(3, np.zeros(4, np.int64), np.zeros(0, np.int32), None, D, g)
    assert np.array_equal(lam, g)
    # chain 0 -> 1: P[1][0] = 1, so lambda_1 = g_1 and lambda_0 = g_0 + d g_1
    lam, _ = oracle.adjoint(2, np.array([0, 1, 1], np.int64), np.array([1], np.int32), None, D,
                            np.array([0.5, 2.0]))
    assert lam[1] == 2.0 and abs(lam[0] - (0.5 + D * 2.0)) < 1e-15
    # directed n-cycle with constant g: lambda = g / (1 - d)
    n = 17
    lam, _ = oracle.adjoint(n, np.arange(n + 1, dtype=np.int64), ((np.arange(n) + 1) % n).astype(np.int32),
                            None, D, np.full(n, 0.7), tol=1e-15)
    assert np.abs(lam - 0.7 / (1 - D)).max() < 1e-13


@pytest.mark.parametrize("seed", range(3))
def test_grad_w_matches_central_differences(seed):
    n = 25
    cp, ci, cw = _graph(20 + seed, n, 4 * n, True)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(n)
    Z = rng.random(n)
    x = _x(n, cp, ci, cw, Z)
    lam = np.linalg.solve((np.eye(n) - D * _dense_P(n, cp, ci, cw)).T, g)
    grad = oracle.grad_w(n, cp, ci, cw, D, x, lam)
    h = 1e-6
    fd = np.zeros(len(cw))
    for e in range(len(cw)):
        wp, wm = cw.copy(), cw.copy()
        wp[e] += h
        wm[e] -= h
        fd[e] = (g @ _x(n, cp, ci, wp, Z) - g @ _x(n, cp, ci, wm, Z)) / (2 * h)
    assert np.abs(fd - grad).max() <= 1e-7 * np.abs(grad).max() + 1e-9


def test_grad_w_unweighted_is_the_all_ones_gradient():
    n = 30
    cp, ci, _ = _graph(40, n, 4 * n, False)
    g = np.random.default_rng(4).standard_normal(n)
    Z = np.full(n, 1.0 / n)
    ones = np.ones(len(ci))
    x = _x(n, cp, ci, None, Z)
    lam, _ = oracle.adjoint(n, cp, ci, None, D, g, tol=1e-15)
    a = oracle.grad_w(n, cp, ci, None, D, x, lam)
    b = oracle.grad_w(n, cp, ci, ones, D, x, lam)
    assert np.allclose(a, b, rtol=1e-14, atol=1e-17)
    e = 7
    wp, wm = ones.copy(), ones.copy()
    wp[e] += 1e-6
    wm[e] -= 1e-6
    fd = (g @ _x(n, cp, ci, wp, Z) - g @ _x(n, cp, ci, wm, Z)) / 2e-6
    assert abs(fd - a[e]) <= 1e-7 * np.abs(a).max() + 1e-9


def test_grad_Z_is_scaled_adjoint():
    n = 40
    cp, ci, cw = _graph(50, n, 4 * n, True)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(n)
    Z = rng.random(n)
    lam, _ = oracle.adjoint(n, cp, ci, cw, D, g, tol=1e-15)
    h = 1e-6
    for i in (0, 13, n - 1):
        zp, zm = Z.copy(), Z.copy()
        zp[i] += h
        zm[i] -= h
        fd = (g @ _x(n, cp, ci, cw, zp) - g @ _x(n, cp, ci, cw, zm)) / (2 * h)
        assert abs(fd - (1 - D) * lam[i]) <= 1e-8 * np.abs(lam).max()
