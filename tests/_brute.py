"""Brute-force restatements used to pin the oracle (tests only).

Everything here is deliberately naive Python over explicit link lists, so that
it shares nothing with ``oracle/di_oracle.c`` beyond the paper's definitions.
"""
from fractions import Fraction

import numpy as np


def links(ptr, idx, w=None, layout=0):
    """(src, dst, weight) triples in input order."""
    out = []
    for r in range(len(ptr) - 1):
        for e in range(int(ptr[r]), int(ptr[r + 1])):
            a, b = (r, int(idx[e])) if layout == 0 else (int(idx[e]), r)
            out.append((a, b, 1.0 if w is None else float(w[e])))
    return out


def merged(n, triples):
    """dict (src,dst) -> weight summed in input order, and canonical CSR."""
    acc = {}
    for a, b, x in triples:
        acc[(a, b)] = acc[(a, b)] + x if (a, b) in acc else x
    keys = sorted(acc)
    ptr = np.zeros(n + 1, dtype=np.int64)
    for a, _ in keys:
        ptr[a + 1] += 1
    ptr = np.cumsum(ptr)
    idx = np.array([b for _, b in keys], dtype=np.int32)
    w = np.array([acc[k] for k in keys], dtype=np.float64)
    return acc, ptr, idx, w


def dense_P_brute(n, acc, weighted):
    """P[i][j] = w(j,i) / sum_k w(j,k) from the merged link dict (Eq. def-p)."""
    P = np.zeros((n, n))
    out_sum = {}
    out_cnt = {}
    for (a, b), x in sorted(acc.items()):
        out_sum[a] = out_sum.get(a, 0.0) + x
        out_cnt[a] = out_cnt.get(a, 0) + 1
    for (a, b), x in acc.items():
        P[b, a] = (x / out_sum[a]) if weighted else 1.0 / out_cnt[a]
    return P


def exact_solution(n, acc, d, Z):
    """Exact rational x = (1-d)(I - dP)^-1 Z by Gauss-Jordan over Fractions
    (unweighted P, rational d and Z)."""
    d = Fraction(d)
    cnt = {}
    for (a, _b) in acc:
        cnt[a] = cnt.get(a, 0) + 1
    A = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for (a, b) in acc:
        A[b][a] -= d / cnt[a]
    rhs = [(1 - d) * Fraction(z) for z in Z]
    M = [A[i] + [rhs[i]] for i in range(n)]
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
