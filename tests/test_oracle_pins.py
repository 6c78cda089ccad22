"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them compares the oracle with
itself: the references are brute-force link dictionaries, closed forms, exact
rational arithmetic, a LAPACK direct solve, the invariant Eq. HnFn, and the
bounds of Theorems 1-3.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1501_06350_gb300 import synth
from tests import _brute as B

D = 0.85


def _rand_multigraph(seed, n, m, weighted=False, loops=True):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=m)
    dst = rng.integers(0, n, size=m)
    if not loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    # unsorted CSR rows, duplicates allowed
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, src + 1, 1)
    ptr = np.cumsum(ptr)
    w = rng.lognormal(size=len(dst)) if weighted else None
    return ptr, dst.astype(np.int32), w


# ---------------------------------------------------------------- Eq. def-p
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("weighted", [False, True])
def test_canonical_csr_matches_bruteforce(seed, layout, weighted):
    n = 1 + seed * 7
    ptr, idx, w = _rand_multigraph(seed, n, 4 * n, weighted)
    acc, bptr, bidx, bw = B.merged(n, B.links(ptr, idx, w, layout))
    optr, oidx, ow = oracle.canonical_csr(n, ptr, idx, w if weighted else None, layout)
    assert np.array_equal(optr, bptr)
    assert np.array_equal(oidx, bidx)
    if weighted:
        assert np.array_equal(ow, bw)  # same left-to-right sums, bit for bit


def test_canonical_csr_rejects_bad_input():
    ptr = np.array([0, 2, 3], dtype=np.int64)
    with pytest.raises(ValueError):
        oracle.canonical_csr(2, ptr, np.array([0, 2, 1], dtype=np.int32))      # index out of range
    with pytest.raises(ValueError):
        oracle.canonical_csr(2, np.array([0, 3, 2], dtype=np.int64), np.array([0, 1, 1], np.int32))
    with pytest.raises(ValueError):
        oracle.canonical_csr(2, ptr, np.array([0, 1, 1], np.int32), np.array([1.0, -1.0, 2.0]))
    with pytest.raises(ValueError):
        oracle.canonical_csr(2, ptr, np.array([0, 1, 1], np.int32), np.array([1.0, np.nan, 2.0]))


@pytest.mark.parametrize("seed", range(4))
def test_transpose_matches_bruteforce(seed):
    n = 3 + 5 * seed
    ptr, idx, w = _rand_multigraph(100 + seed, n, 5 * n, True)
    cp, ci, cw = oracle.canonical_csr(n, ptr, idx, w)
    tp, ti, tw = oracle.transpose(n, cp, ci, cw)
    acc, _, _, _ = B.merged(n, B.links(cp, ci, cw))
    rev = sorted((b, a) for (a, b) in acc)
    assert np.array_equal(ti, np.array([a for _, a in rev], dtype=np.int32))
    assert np.array_equal(np.diff(tp), np.bincount(ci, minlength=n))
    assert np.array_equal(tw, np.array([acc[(a, b)] for b, a in rev]))
    # transposing twice gives the canonical CSR back
    pp, pi, pw = oracle.transpose(n, tp, ti, tw)
    assert np.array_equal(pp, cp) and np.array_equal(pi, ci) and np.array_equal(pw, cw)


# ------------------------------------------------------- closed forms (Section 2.1)
def _solve(n, pairs, Z=None, w=None, tol=1e-15, schedule=oracle.ARGMAX):
    src = np.array([a for a, _ in pairs], dtype=np.int64)
    dst = np.array([b for _, b in pairs], dtype=np.int32)
    order = np.argsort(src, kind="stable")
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, src + 1, 1)
    ptr = np.cumsum(ptr)
    p, i, ww = oracle.canonical_csr(n, ptr, dst[order], None if w is None else np.asarray(w)[order])
    H, F, info, _ = oracle.di_solve(n, p, i, ww, D, Z, tol=tol, schedule=schedule)
    return H, F, info


@pytest.mark.parametrize("schedule", [oracle.ARGMAX, oracle.CYC])
def test_no_links_gives_teleport_share(schedule):
    n = 5
    Z = np.array([0.1, 0.2, 0.3, 0.25, 0.15])
    H, F, info = _solve(n, [], Z, schedule=schedule)
    assert np.abs(H - (1 - D) * Z).sum() < 1e-16
    assert info["l_dangling"] == pytest.approx((1 - D) * Z.sum(), abs=1e-16)


@pytest.mark.parametrize("n", [1, 2, 7, 50])
def test_directed_cycle_is_uniform(n):
    if n == 1:
        pairs = [(0, 0)]                  # a single page linking to itself
    else:
        pairs = [(i, (i + 1) % n) for i in range(n)]
    H, F, info = _solve(n, pairs)
    assert np.abs(H - 1.0 / n).sum() < 1e-13


def test_two_page_chain():
    H, F, _ = _solve(2, [(0, 1)], np.array([0.5, 0.5]))
    x0 = (1 - D) / 2
    assert H[0] == pytest.approx(x0, abs=1e-16)
    assert H[1] == pytest.approx(D * x0 + (1 - D) / 2, abs=1e-15)


def test_out_star_and_in_star():
    k = 6
    Z = np.full(k + 1, 1.0 / (k + 1))
    H, _, _ = _solve(k + 1, [(0, j) for j in range(1, k + 1)], Z)
    xc = (1 - D) * Z[0]
    assert H[0] == pytest.approx(xc, abs=1e-16)
    assert np.allclose(H[1:], D * xc / k + (1 - D) * Z[1:], atol=1e-15, rtol=0)
    H, _, _ = _solve(k + 1, [(j, 0) for j in range(1, k + 1)], Z)
    assert np.allclose(H[1:], (1 - D) * Z[1:], atol=1e-16, rtol=0)
    assert H[0] == pytest.approx(D * H[1:].sum() + (1 - D) * Z[0], abs=1e-15)


def test_self_loop_keeps_its_share():
    # Eq. defF leaves d F(i) P_ii on a looping page: x = d x + (1-d) z => x = z
    H, F, _ = _solve(3, [(0, 0), (1, 2)], np.array([0.5, 0.3, 0.2]))
    assert H[0] == pytest.approx(0.5, abs=1e-14)
    assert H[1] == pytest.approx((1 - D) * 0.3, abs=1e-16)
    assert H[2] == pytest.approx(D * (1 - D) * 0.3 + (1 - D) * 0.2, abs=1e-16)


def test_complete_graph_is_uniform():
    n = 9
    H, _, _ = _solve(n, [(a, b) for a in range(n) for b in range(n) if a != b])
    assert np.abs(H - 1.0 / n).sum() < 1e-13


def test_weighted_pair_closed_form():
    # 0 -> 1 (w=3), 0 -> 2 (w=1), 1 -> 0 (w=2); 2 dangling; Z uniform.
    Z = np.full(3, 1 / 3)
    H, _, _ = _solve(3, [(0, 1), (0, 2), (1, 0)], Z, w=[3.0, 1.0, 2.0])
    # x0 = d x1 + c, x1 = d (3/4) x0 + c, x2 = d (1/4) x0 + c, c = (1-d)/3
    c = (1 - D) / 3
    x0 = (D * c + c) / (1 - D * D * 0.75)
    x1 = D * 0.75 * x0 + c
    x2 = D * 0.25 * x0 + c
    assert np.abs(H - [x0, x1, x2]).sum() < 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_exact_rational_solution(seed):
    n = 7
    ptr, idx, _ = _rand_multigraph(200 + seed, n, 12, loops=False)
    acc, cp, ci, _ = B.merged(n, B.links(ptr, idx))
    Zf = [Fraction(k + 1, n * (n + 1) // 2) for k in range(n)]
    x = [float(v) for v in B.exact_solution(n, acc, Fraction(17, 20), Zf)]
    H, F, info, _ = oracle.di_solve(n, cp, ci, None, 0.85, np.array([float(z) for z in Zf]),
                                    tol=1e-15)
    assert np.abs(H - x).sum() < 1e-14
    xd = oracle.dense_solution(n, cp, ci, None, 0.85, np.array([float(z) for z in Zf]))
    assert np.abs(xd - x).sum() < 1e-14


# ----------------------------------------- Theorem 1, Eq. SL, Eq. HnFn, Section 3.3
def _setup(seed, n, m, weighted=False, zkind="uniform"):
    ptr, idx, w = _rand_multigraph(300 + seed, n, m, weighted)
    cp, ci, cw = oracle.canonical_csr(n, ptr, idx, w)
    acc, _, _, _ = B.merged(n, B.links(ptr, idx, w))
    P = B.dense_P_brute(n, acc, weighted)
    if zkind == "uniform":
        Z = np.full(n, 1.0 / n)
    elif zkind == "random":
        Z = synth.random_z(n, seed)
    else:
        Z = synth.random_z(n, seed, signed=True)
    x = (1 - D) * np.linalg.solve(np.eye(n) - D * P, Z)
    return cp, ci, cw, P, Z, x


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("zkind", ["uniform", "random", "signed"])
def test_di_converges_to_dense_solution(seed, weighted, zkind):
    n = 40 + 30 * seed
    cp, ci, cw, P, Z, x = _setup(seed, n, 4 * n, weighted, zkind)
    H, F, info, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-14)
    assert info["converged"]
    assert np.abs(H - x).sum() <= np.abs(F).sum() / (1 - D) + 1e-14
    assert np.abs(H - x).sum() < 2e-14


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("cut", [1, 17, 150, 900])
def test_invariant_mass_and_bound_on_partial_runs(seed, cut):
    n = 60
    cp, ci, cw, P, Z, x = _setup(seed, n, 240, weighted=seed == 2, zkind="random")
    H, F, info, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-300, max_diffusions=cut)
    assert info["diffusions"] == cut
    # Eq. HnFn: H_k + F_k = F_0 + d P H_k, element by element
    lhs = H + F
    rhs = (1 - D) * Z + D * P @ H
    assert np.max(np.abs(lhs - rhs)) < 1e-15
    # mass: sum F + (1-d) sum H + d * (H on dangling) = (1-d) sum Z
    dang = np.diff(cp) == 0
    mass = F.sum() + (1 - D) * H.sum() + D * H[dang].sum()
    assert mass == pytest.approx((1 - D) * Z.sum(), abs=1e-15)
    # Theorem 1, Eq. SL
    assert np.abs(x - H).sum() <= np.abs(F).sum() / (1 - D) * (1 + 1e-12) + 1e-16
    assert info["l_dangling"] == pytest.approx(H[dang].sum(), abs=1e-16)


@pytest.mark.parametrize("seed", range(3))
def test_completed_normalisation_is_exact(seed):
    # Section 3.3: |x_c - (1-d)/(1-d-d l) H|_1 = |F|_1 / (1-d-d l) for F >= 0
    n = 50
    cp, ci, cw, P, Z, x = _setup(seed, n, 120, zkind="random")
    Pc = P.copy()
    dang = np.diff(cp) == 0
    assert dang.any()
    Pc[:, dang] = Z[:, None]
    xc = (1 - D) * np.linalg.solve(np.eye(n) - D * Pc, Z)
    for cut in (5, 60, 400):
        H, F, info, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-300, max_diffusions=cut)
        assert (F >= 0).all()
        l = info["l_dangling"]
        alpha = (1 - D) / (1 - D - D * l)
        dist = np.abs(xc - alpha * H).sum()
        assert dist == pytest.approx(np.abs(F).sum() / (1 - D - D * l), rel=1e-10, abs=1e-16)


@pytest.mark.parametrize("seed", range(3))
def test_theorem2_round_robin_bound(seed):
    # Theorem 2: DI-cyc, |Z|_1 = 1: |x - H_k| <= d^floor(k/n)
    n = 30
    cp, ci, cw, P, Z, x = _setup(seed, n, 90, zkind="random")
    for rounds in range(0, 12):
        H, F, info, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-300,
                                        max_diffusions=max(rounds * n, 0) or 1,
                                        schedule=oracle.CYC)
        k = info["diffusions"]
        assert np.abs(x - H).sum() <= D ** (k // n) + 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_theorem3_argmax_step_decrease(seed):
    # Theorem 3: each DI-argmax diffusion has |F_k| <= (1 - (1-d)/n) |F_{k-1}|
    n = 40
    cp, ci, cw, P, Z, x = _setup(seed, n, 160, zkind="random")
    _, _, info, tr = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-12, max_diffusions=4000,
                                     trace=True)
    prev = np.concatenate([[(1 - D) * np.abs(Z).sum()], tr[:-1]])
    assert np.all(tr <= (1 - (1 - D) / n) * prev * (1 + 1e-12) + 1e-18)
    # and the bound of Theorem 3 on the error after k steps
    H, F, info, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-300, max_diffusions=500)
    assert np.abs(x - H).sum() <= (1 - (1 - D) / n) ** 500 + 1e-15


# --------------------------------------------------------------- Section 2.2
@pytest.mark.parametrize("seed", range(3))
def test_power_iteration_matches_dense_and_contracts(seed):
    n = 80
    cp, ci, cw, P, Z, x = _setup(seed, n, 300, weighted=seed == 1, zkind="random")
    xp, it = oracle.power_iteration(n, cp, ci, cw, D, Z, tol=1e-16, max_iters=2000)
    assert np.abs(xp - x).sum() < 1e-14
    errs = []
    for k in range(1, 8):
        xk, _ = oracle.power_iteration(n, cp, ci, cw, D, Z, tol=0.0, max_iters=k)
        errs.append(np.abs(xk - x).sum())
    for a, b in zip(errs, errs[1:]):
        assert b <= D * a * (1 + 1e-9)


# --------------------------------------------------------------- Section 3.5
def test_apply_batch_set_semantics():
    n = 6
    acc, cp, ci, cw = B.merged(n, [(0, 1, 1.0), (0, 2, 2.0), (3, 4, 1.5), (5, 0, 1.0)])
    src = np.array([0, 0, 3, 1, 1, 2, 4], dtype=np.int32)
    dst = np.array([2, 3, 4, 5, 5, 2, 4], dtype=np.int32)
    op = np.array([-1, 1, 1, 1, -1, 1, -1], dtype=np.int8)
    wb = np.array([9.0, 4.0, 7.0, 1.0, 1.0, 2.5, 1.0])
    p, i, w = oracle.apply_batch(n, cp, ci, cw, src, dst, op, wb)
    want = {(0, 1): 1.0, (0, 3): 4.0, (3, 4): 7.0, (2, 2): 2.5, (5, 0): 1.0}
    _, bp, bi, bw = B.merged(n, [(a, b, x) for (a, b), x in want.items()])
    assert np.array_equal(p, bp) and np.array_equal(i, bi) and np.array_equal(w, bw)


@pytest.mark.parametrize("seed", range(4))
def test_apply_batch_random_vs_bruteforce(seed):
    n = 25
    ptr, idx, _ = _rand_multigraph(400 + seed, n, 80, loops=False)
    acc, cp, ci, _ = B.merged(n, B.links(ptr, idx))
    src, dst, op = synth.edge_batch(cp, ci, n, 0.3, seed)
    p, i, _ = oracle.apply_batch(n, cp, ci, None, src, dst, op)
    cur = set(acc)
    for a, b, o in zip(src, dst, op):
        (cur.add if o == 1 else cur.discard)((int(a), int(b)))
    _, bp, bi, _ = B.merged(n, [(a, b, 1.0) for a, b in cur])
    assert np.array_equal(p, bp) and np.array_equal(i, bi)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("weighted", [False, True])
def test_update_theorem_reaches_new_solution(seed, weighted):
    n = 70
    ptr, idx, w = _rand_multigraph(500 + seed, n, 280, weighted, loops=False)
    cp, ci, cw = oracle.canonical_csr(n, ptr, idx, w)
    Z = synth.random_z(n, seed)
    H, F, _, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-300, max_diffusions=300)
    src, dst, op = synth.edge_batch(cp, ci, n, 0.2, seed)
    wb = np.full(len(src), 2.0) if weighted else None
    p2, i2, w2 = oracle.apply_batch(n, cp, ci, cw, src, dst, op, wb)
    F2, changed = oracle.update_inject(n, (cp, ci, cw), (p2, i2, w2), D, H, F)
    assert changed > 0
    # F'_0 = F + d (P' - P) H with brute-force dense matrices
    acc0, _, _, _ = B.merged(n, B.links(cp, ci, cw))
    acc1, _, _, _ = B.merged(n, B.links(p2, i2, w2))
    P0 = B.dense_P_brute(n, acc0, weighted)
    P1 = B.dense_P_brute(n, acc1, weighted)
    assert np.max(np.abs(F2 - (F + D * (P1 - P0) @ H))) < 1e-16
    # resumed DI on P' converges to the dense solution of P' (Theorem update)
    H3, F3, info, _ = oracle.di_solve(n, p2, i2, w2, D, F=F2, H=H, tol=1e-14)
    x1 = (1 - D) * np.linalg.solve(np.eye(n) - D * P1, Z)
    assert np.abs(H3 - x1).sum() < 1e-13
    assert np.abs(H3 - x1).sum() <= np.abs(F3).sum() / (1 - D) + 1e-14


# ----------------------------------------------------------- frontier, residual
def test_select_frontier_bruteforce():
    rng = np.random.default_rng(7)
    F = rng.normal(size=500)
    F[::7] = 0.0
    theta = np.abs(F).sum() / len(F)
    want = [i for i in range(len(F)) if abs(F[i]) >= theta and F[i] != 0.0]
    assert oracle.select_frontier(F, theta).tolist() == want
    assert oracle.select_frontier(np.zeros(4), 0.0).tolist() == []


@pytest.mark.parametrize("weighted", [False, True])
def test_residual_is_the_fluid(weighted):
    n = 50
    cp, ci, cw, P, Z, x = _setup(9, n, 200, weighted, "random")
    H, F, _, _ = oracle.di_solve(n, cp, ci, cw, D, Z, tol=1e-300, max_diffusions=77)
    r = oracle.residual(n, cp, ci, cw, D, Z, H)
    assert np.max(np.abs(r - ((1 - D) * Z + D * P @ H - H))) < 1e-16
    assert np.max(np.abs(r - F)) < 1e-15


def test_generators_are_seeded_and_shaped():
    g1 = synth.pa_graph(n=2000, m_target=20000)
    g2 = synth.pa_graph(n=2000, m_target=20000)
    assert np.array_equal(g1.idx, g2.idx) and np.array_equal(g1.ptr, g2.ptr)
    deg = np.diff(g1.ptr)
    assert (deg == 0).sum() == 200
    assert abs(g1.nnz - 20000) <= 200
    assert (g1.idx != np.repeat(np.arange(2000), deg)).all()
    w = synth.web_graph(n=20000, m_target=200000)
    assert abs(w.nnz - 200000) <= 2000
    assert (np.diff(w.ptr) == 0).sum() == 3000
    src = np.repeat(np.arange(w.n), np.diff(w.ptr))
    assert len(np.unique(src * w.n + w.idx)) == w.nnz     # distinct links per page
