"""CPU oracle for D-Iteration (arXiv:1501.06350) -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
has no fallback to it.  It shares no code with the CUDA path: the sequential
FP64 routines live in ``di_oracle.c`` (plain C, one thread), and the few
helpers below are plain NumPy/LAPACK restatements of the paper's definitions.

Parity status: every routine is pinned by ``tests/test_oracle_*.py`` against
closed forms, brute force, the dense direct solution (Section 2.1, the closed
form x = (1-d)(I-dP)^-1 Z), the invariant Eq. HnFn and the bounds of
Theorems 1-3; the Section 3.3 helpers (``completed_solution``,
``dangling_loss``) by exact rational solves of the completed matrix, the
rank-one closed form of a graph without links, the paper's normalisation
factor and the mass balance (``tests/test_oracle_completion.py``).  None is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "di_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ARGMAX = 0
CYC = 1


def build(force: bool = False) -> str:
    """Compile di_oracle.c into liboracle.so next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Info(ctypes.Structure):
    _fields_ = [("resid_l1", ctypes.c_double), ("l_dangling", ctypes.c_double),
                ("diffusions", ctypes.c_int64), ("edge_pushes", ctypes.c_int64),
                ("cycles", ctypes.c_int64), ("converged", ctypes.c_int)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        _lib.or_canonical_csr.restype = i64
        _lib.or_canonical_csr.argtypes = [i64, i64, P, P, P, ctypes.c_int, P, P, P]
        _lib.or_transpose.restype = None
        _lib.or_transpose.argtypes = [i64, P, P, P, P, P, P]
        _lib.or_di_init.restype = None
        _lib.or_di_init.argtypes = [i64, ctypes.c_double, P, P, P]
        _lib.or_di_solve.restype = ctypes.c_int
        _lib.or_di_solve.argtypes = [i64, P, P, P, ctypes.c_double, P, P, ctypes.c_double, i64,
                                     ctypes.c_int, P, ctypes.POINTER(_Info)]
        _lib.or_power_iteration.restype = i64
        _lib.or_power_iteration.argtypes = [i64, P, P, P, ctypes.c_double, P, ctypes.c_double,
                                            i64, P]
        _lib.or_apply_batch.restype = i64
        _lib.or_apply_batch.argtypes = [i64, P, P, P, i64, P, P, P, P, P, P, P]
        _lib.or_update_inject.restype = i64
        _lib.or_update_inject.argtypes = [i64, P, P, P, P, P, P, ctypes.c_double, P, P]
        _lib.or_adjoint_jacobi.restype = i64
        _lib.or_adjoint_jacobi.argtypes = [i64, P, P, P, ctypes.c_double, P, ctypes.c_double, i64, P]
        _lib.or_grad_w.restype = None
        _lib.or_grad_w.argtypes = [i64, P, P, P, ctypes.c_double, P, P, P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def canonical_csr(n, ptr, idx, w=None, layout=0):
    """Canonical out-CSR of P's link structure (Section 2.1, Eq. def-p)."""
    lib = _load()
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    w = _f64(w)
    nnz = int(ptr[-1])
    optr = np.zeros(n + 1, dtype=np.int64)
    oidx = np.zeros(max(nnz, 1), dtype=np.int32)
    ow = np.zeros(max(nnz, 1), dtype=np.float64) if w is not None else None
    m = lib.or_canonical_csr(n, nnz, _p(ptr), _p(idx), _p(w), layout, _p(optr), _p(oidx), _p(ow))
    if m < 0:
        raise ValueError("invalid graph input")
    return optr, oidx[:m].copy(), (None if ow is None else ow[:m].copy())


def transpose(n, ptr, idx, w=None):
    """In-link CSR (sources of each target, ascending) of a canonical out-CSR."""
    lib = _load()
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    w = _f64(w)
    nnz = int(ptr[-1])
    tptr = np.zeros(n + 1, dtype=np.int64)
    tidx = np.zeros(max(nnz, 1), dtype=np.int32)
    tw = np.zeros(max(nnz, 1), dtype=np.float64) if w is not None else None
    lib.or_transpose(n, _p(ptr), _p(idx), _p(w), _p(tptr), _p(tidx), _p(tw))
    return tptr, tidx[:nnz].copy(), (None if tw is None else tw[:nnz].copy())


def di_init(n, d, Z=None):
    """F_0 = (1-d) Z, H_0 = 0 (Section 3.1)."""
    lib = _load()
    F = np.zeros(n)
    H = np.zeros(n)
    lib.or_di_init(n, d, _p(_f64(Z)), _p(F), _p(H))
    return F, H


def di_solve(n, ptr, idx, w, d, Z=None, tol=1e-13, max_diffusions=None, schedule=ARGMAX,
             F=None, H=None, trace=False):
    """Sequential D-Iteration (Section 3.1) with the DI-argmax or DI-cyc scheduler
    (Section 3.4), stopping on |F|_1/(1-d) <= tol (Theorem 1).  Pass F and H to
    resume from a given state (Theorem update).  Returns (H, F, info, trace)."""
    lib = _load()
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    w = _f64(w)
    if F is None:
        F, H = di_init(n, d, Z)
    else:
        F = np.array(F, dtype=np.float64, copy=True)
        H = np.array(H, dtype=np.float64, copy=True)
    if max_diffusions is None:
        max_diffusions = 1 << 62
    tr = np.zeros(max_diffusions) if trace else None
    info = _Info()
    rc = lib.or_di_solve(n, _p(ptr), _p(idx), _p(w), d, _p(F), _p(H), tol, max_diffusions,
                         schedule, _p(tr), ctypes.byref(info))
    if rc < 0:
        raise ValueError("invalid solver input")
    out = dict(resid_l1=info.resid_l1, l_dangling=info.l_dangling, diffusions=info.diffusions,
               edge_pushes=info.edge_pushes, cycles=info.cycles, converged=bool(info.converged))
    if trace:
        tr = tr[:info.diffusions].copy()
    return H, F, out, tr


def power_iteration(n, ptr, idx, w, d, Z=None, tol=1e-15, max_iters=10_000):
    """x_{k+1} = d P x_k + (1-d) Z (Section 2.2).  Returns (x, iterations)."""
    lib = _load()
    x = np.zeros(n)
    it = lib.or_power_iteration(n, _p(np.ascontiguousarray(ptr, dtype=np.int64)),
                                _p(np.ascontiguousarray(idx, dtype=np.int32)), _p(_f64(w)), d,
                                _p(_f64(Z)), tol, max_iters, _p(x))
    return x, int(it)


def apply_batch(n, ptr, idx, w, src, dst, op, wb=None):
    """Apply link insertions (+1) / deletions (-1) in batch order; canonical result."""
    lib = _load()
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    op = np.ascontiguousarray(op, dtype=np.int8)
    w = _f64(w)
    wb = _f64(wb)
    m = len(src)
    cap = int(ptr[-1]) + m + 1
    optr = np.zeros(n + 1, dtype=np.int64)
    oidx = np.zeros(cap, dtype=np.int32)
    ow = np.zeros(cap) if w is not None else None
    k = lib.or_apply_batch(n, _p(ptr), _p(idx), _p(w), m, _p(src), _p(dst), _p(wb), _p(op),
                           _p(optr), _p(oidx), _p(ow))
    if k < 0:
        raise ValueError("invalid batch")
    return optr, oidx[:k].copy(), (None if ow is None else ow[:k].copy())


def update_inject(n, old, new, d, H, F):
    """F'_0 = F + d (P' - P) H (Theorem update).  ``old``/``new`` are (ptr, idx, w).
    Returns (F', number of changed columns)."""
    lib = _load()
    F2 = np.array(F, dtype=np.float64, copy=True)
    H = np.ascontiguousarray(H, dtype=np.float64)
    (p0, i0, w0), (p1, i1, w1) = old, new
    ch = lib.or_update_inject(n, _p(np.ascontiguousarray(p0, dtype=np.int64)),
                              _p(np.ascontiguousarray(i0, dtype=np.int32)), _p(_f64(w0)),
                              _p(np.ascontiguousarray(p1, dtype=np.int64)),
                              _p(np.ascontiguousarray(i1, dtype=np.int32)), _p(_f64(w1)), d,
                              _p(H), _p(F2))
    return F2, int(ch)


def adjoint(n, ptr, idx, w, d, g, tol=1e-15, max_iters=100_000):
    """lambda with (I - d P)^T lambda = g (Jacobi sweeps of the Neumann series,
    stopped on the bound |lambda - lambda_k|_inf <= tol).  Returns (lambda, sweeps)."""
    lib = _load()
    lam = np.zeros(n)
    it = lib.or_adjoint_jacobi(n, _p(np.ascontiguousarray(ptr, dtype=np.int64)),
                               _p(np.ascontiguousarray(idx, dtype=np.int32)), _p(_f64(w)), d,
                               _p(_f64(g)), tol, max_iters, _p(lam))
    if it < 0:
        raise ValueError("invalid adjoint input")
    return lam, int(it)


def grad_w(n, ptr, idx, w, d, x, lam):
    """dL/dw per link of the canonical out-CSR for L = g . x, given x and the
    adjoint lambda: d x_j / W_j (lambda_k - (P^T lambda)_j)."""
    lib = _load()
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    out = np.zeros(max(int(ptr[-1]), 1))
    lib.or_grad_w(n, _p(ptr), _p(np.ascontiguousarray(idx, dtype=np.int32)), _p(_f64(w)), d,
                  _p(_f64(x)), _p(_f64(lam)), _p(out))
    return out[:int(ptr[-1])]


# --------------------------------------------------------------------------
# NumPy restatements of plain definitions.
# --------------------------------------------------------------------------

def p_values(ptr, idx, w=None):
    """Per-link P entries w(j,i)/W_j (Section 2.1, Eq. def-p), in CSR order."""
    deg = np.diff(ptr)
    src = np.repeat(np.arange(len(deg)), deg)
    if w is None:
        return 1.0 / deg[src].astype(np.float64), src
    W = np.zeros(len(deg))
    for j in np.nonzero(deg)[0]:  # left-to-right row sums
        s = 0.0
        for v in w[ptr[j]:ptr[j + 1]]:
            s += float(v)
        W[j] = s
    return np.asarray(w, dtype=np.float64) / W[src], src


def dense_P(n, ptr, idx, w=None):
    """Dense n x n diffusion matrix (Section 2.1, Eq. def-p); small n only."""
    P = np.zeros((n, n))
    p, src = p_values(ptr, idx, w)
    for e in range(len(p)):
        P[idx[e], src[e]] += p[e]
    return P


def dense_solution(n, ptr, idx, w, d, Z=None):
    """x = (1-d)(I - dP)^-1 Z (Section 2.1) by a LAPACK direct solve."""
    Z = np.full(n, 1.0 / n) if Z is None else np.asarray(Z, dtype=np.float64)
    A = np.eye(n) - d * dense_P(n, ptr, idx, w)
    return (1.0 - d) * np.linalg.solve(A, Z)


def completed_solution(n, ptr, idx, w, d, Z=None):
    """Solution for P completed on its dangling columns by Z (Section 3.3)."""
    Z = np.full(n, 1.0 / n) if Z is None else np.asarray(Z, dtype=np.float64)
    P = dense_P(n, ptr, idx, w)
    dang = np.diff(ptr) == 0
    P[:, dang] = Z[:, None]
    return (1.0 - d) * np.linalg.solve(np.eye(n) - d * P, Z)


def residual(n, ptr, idx, w, d, Z, H):
    """r = (1-d) Z + d P H - H: by Eq. HnFn this is the exact fluid left for the
    history H, and |x - H|_1 <= |r|_1 / (1-d) (Theorem 1)."""
    ptr = np.asarray(ptr)
    p, src = p_values(ptr, idx, w)
    PH = np.bincount(np.asarray(idx, dtype=np.int64), weights=p * H[src], minlength=n)
    Z = np.full(n, 1.0 / n) if Z is None else np.asarray(Z, dtype=np.float64)
    return (1.0 - d) * Z + d * PH - H


def select_frontier(F, theta):
    """Ascending ids i with |F_i| >= theta and F_i != 0 (the DI-argmax test of
    Section 3.4 applied to a whole fluid snapshot at once)."""
    F = np.asarray(F, dtype=np.float64)
    return np.nonzero((np.abs(F) >= theta) & (F != 0.0))[0].astype(np.int32)


def dangling_loss(ptr, H):
    """l = sum of H over dangling nodes (Section 3.3)."""
    return float(np.asarray(H)[np.diff(ptr) == 0].sum())
