"""Python face of libdi.so: graphs and solver states over torch CUDA tensors
(device memory, streams) or NumPy arrays (host memory).

Argument marshalling only; see include/di.h for the semantics of each call.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

_f64 = torch.float64


def _is_dev(x) -> bool:
    return isinstance(x, torch.Tensor) and x.is_cuda


def _host(x, dtype):
    if isinstance(x, torch.Tensor):
        x = x.cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _p(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _prep(x, dtype_np, dtype_t, mem):
    """Input buffer for `mem`: contiguous cuda tensor or NumPy array."""
    if x is None:
        return None
    if mem == L.DI_MEM_DEVICE:
        if not _is_dev(x):
            x = torch.as_tensor(np.asarray(x)).cuda()
        return x.to(dtype_t).contiguous()
    return _host(x, dtype_np)


class Graph:
    """Canonical diffusion structure of P (Section 2.1, Eq. def-p) on the GPU.

    ``ptr``/``idx``/``w`` may be NumPy arrays (copied from host memory) or CUDA
    tensors (read from device memory).  ``layout`` is "csr" (rows = sources)
    or "csc" (rows = targets).  ``w`` may be float32 or float64.
    """

    def __init__(self, n: int, ptr, idx, w=None, layout: str = "csr"):
        self._h = None
        mem = L.DI_MEM_DEVICE if _is_dev(ptr) else L.DI_MEM_HOST
        ptr = _prep(ptr, np.int64, torch.int64, mem)
        idx = _prep(idx, np.int32, torch.int32, mem)
        wdt = L.DI_W_NONE
        if w is not None:
            is32 = (w.dtype == torch.float32) if isinstance(w, torch.Tensor) else (np.asarray(w).dtype == np.float32)
            wdt = L.DI_W_F32 if is32 else L.DI_W_F64
            w = _prep(w, np.float32 if is32 else np.float64, torch.float32 if is32 else _f64, mem)
        nnz = int(ptr[-1])
        lay = {"csr": L.DI_LAYOUT_CSR, "csc": L.DI_LAYOUT_CSC}[layout]
        h = ctypes.c_void_p()
        L.check(L.lib().di_graph_create(n, nnz, _p(ptr), _p(idx), _p(w), wdt, lay, mem, _stream(),
                                        ctypes.byref(h)), "di_graph_create")
        self._h = h
        self.n = n

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        n, nnz, nd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        wt = ctypes.c_int()
        L.check(L.lib().di_graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nd),
                                      ctypes.byref(wt)), "di_graph_info")
        return dict(n=n.value, nnz=nnz.value, n_dangling=nd.value, weighted=bool(wt.value))

    @property
    def nnz(self) -> int:
        return self.info()["nnz"]

    def _export(self, fn, device: bool, weights: bool):
        nnz = self.nnz
        if device:
            ptr = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
            idx = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
            w = torch.empty(max(nnz, 1), dtype=_f64, device="cuda") if weights else None
            mem = L.DI_MEM_DEVICE
        else:
            ptr = np.empty(self.n + 1, dtype=np.int64)
            idx = np.empty(max(nnz, 1), dtype=np.int32)
            w = np.empty(max(nnz, 1), dtype=np.float64) if weights else None
            mem = L.DI_MEM_HOST
        L.check(fn(self._h, _p(ptr), _p(idx), _p(w), mem, _stream()), fn.__name__)
        return ptr, idx[:nnz], (None if w is None else w[:nnz])

    def export_csr(self, device: bool = False, weights: bool = True):
        return self._export(L.lib().di_graph_export_csr, device, weights)

    def export_csc(self, device: bool = False, weights: bool = True):
        return self._export(L.lib().di_graph_export_csc, device, weights)

    def close(self):
        if self._h is not None and L._LIB is not None:
            L.lib().di_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _out_buffer(n, device: bool):
    return torch.empty(n, dtype=_f64, device="cuda") if device else np.empty(n, dtype=np.float64)


class State:
    """Fluid F and history H of one problem on one graph (Section 3.1)."""

    def __init__(self, graph: Graph):
        self.graph = graph
        h = ctypes.c_void_p()
        L.check(L.lib().di_state_create(graph.handle, ctypes.byref(h)), "di_state_create")
        self._h = h

    def _finish(self, rc, where, info):
        if rc not in (L.DI_OK, L.DI_ERR_NOT_CONVERGED):
            raise L.DIError(rc, where)
        out = info.as_dict()
        out["converged"] = rc == L.DI_OK
        return out

    def solve(self, d: float = 0.85, Z=None, tol: float = 1e-9, out=None, device: bool = True, **opts):
        """x = d P x + (1-d) Z from scratch; returns (H, info)."""
        mem = L.DI_MEM_DEVICE if device else L.DI_MEM_HOST
        Z = _prep(Z, np.float64, _f64, mem)
        H = out if out is not None else _out_buffer(self.graph.n, device)
        info = L.di_info()
        o = L.default_opts(**opts)
        rc = L.lib().di_solve(self.graph.handle, self._h, d, _p(Z), tol, ctypes.byref(o), _p(H),
                              ctypes.byref(info), mem, _stream())
        return H, self._finish(rc, "di_solve", info)

    def resume(self, tol: float = 1e-9, out=None, device: bool = True, **opts):
        mem = L.DI_MEM_DEVICE if device else L.DI_MEM_HOST
        H = out if out is not None else _out_buffer(self.graph.n, device)
        info = L.di_info()
        o = L.default_opts(**opts)
        rc = L.lib().di_resume(self.graph.handle, self._h, tol, ctypes.byref(o), _p(H),
                               ctypes.byref(info), mem, _stream())
        return H, self._finish(rc, "di_resume", info)

    def update_edges(self, src, dst, op, w=None):
        mem = L.DI_MEM_DEVICE if _is_dev(src) else L.DI_MEM_HOST
        src = _prep(src, np.int32, torch.int32, mem)
        dst = _prep(dst, np.int32, torch.int32, mem)
        op = _prep(op, np.int8, torch.int8, mem)
        w = _prep(w, np.float64, _f64, mem)
        L.check(L.lib().di_update_edges(self.graph.handle, self._h, len(src), _p(src), _p(dst), _p(w),
                                        _p(op), mem, _stream()), "di_update_edges")

    def export(self, device: bool = False):
        n = self.graph.n
        H = _out_buffer(n, device)
        F = _out_buffer(n, device)
        l = ctypes.c_double()
        L.check(L.lib().di_state_export(self._h, _p(H), _p(F), ctypes.byref(l),
                                        L.DI_MEM_DEVICE if device else L.DI_MEM_HOST, _stream()),
                "di_state_export")
        return H, F, l.value

    def import_state(self, H, F, d: float):
        mem = L.DI_MEM_DEVICE if _is_dev(H) else L.DI_MEM_HOST
        H = _prep(H, np.float64, _f64, mem)
        F = _prep(F, np.float64, _f64, mem)
        L.check(L.lib().di_state_import(self._h, _p(H), _p(F), d, mem, _stream()), "di_state_import")

    def close(self):
        if getattr(self, "_h", None) is not None and L._LIB is not None:
            L.lib().di_state_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(graph: Graph, d: float = 0.85, Z=None, tol: float = 1e-9, **opts):
    """One-shot solve; returns (H, info, state)."""
    st = State(graph)
    H, info = st.solve(d, Z, tol, **opts)
    return H, info, st


def frontier_select(graph: Graph, F, theta: float):
    """Ascending ids with |F_i| >= theta, F_i != 0 (the solver's selection kernel)."""
    mem = L.DI_MEM_DEVICE if _is_dev(F) else L.DI_MEM_HOST
    F = _prep(F, np.float64, _f64, mem)
    ids = torch.empty(graph.n, dtype=torch.int32, device="cuda") if mem else np.empty(graph.n, np.int32)
    cnt = ctypes.c_int64()
    L.check(L.lib().di_frontier_select(graph.handle, _p(F), theta, _p(ids), ctypes.byref(cnt), mem,
                                       _stream()), "di_frontier_select")
    return ids[:cnt.value]


def residual_l1(graph: Graph, v) -> float:
    mem = L.DI_MEM_DEVICE if _is_dev(v) else L.DI_MEM_HOST
    v = _prep(v, np.float64, _f64, mem)
    out = ctypes.c_double()
    L.check(L.lib().di_residual_l1(graph.handle, _p(v), ctypes.byref(out), mem, _stream()),
            "di_residual_l1")
    return out.value


def adjoint(graph: Graph, d: float, g, x=None, tol: float = 1e-12, device: bool = True, want_grad_w: bool = True,
            **opts):
    """Backward pass of the solve for L = g . x: lambda with (I - d P)^T lambda = g,
    dL/dZ = (1 - d) lambda and dL/dw per link of the canonical out-CSR (needs the
    forward solution x).  Returns (lambda, grad_Z, grad_w or None, info)."""
    mem = L.DI_MEM_DEVICE if device else L.DI_MEM_HOST
    g = _prep(g, np.float64, _f64, mem)
    x = _prep(x, np.float64, _f64, mem)
    n = graph.n
    lam = _out_buffer(n, device)
    gz = _out_buffer(n, device)
    gw = _out_buffer(max(graph.nnz, 1), device) if (want_grad_w and x is not None) else None
    info = L.di_info()
    o = L.default_opts(**opts)
    rc = L.lib().di_adjoint(graph.handle, d, _p(g), _p(x), tol, ctypes.byref(o), _p(lam), _p(gz), _p(gw),
                            ctypes.byref(info), mem, _stream())
    if rc not in (L.DI_OK, L.DI_ERR_NOT_CONVERGED):
        raise L.DIError(rc, "di_adjoint")
    out = info.as_dict()
    out["converged"] = rc == L.DI_OK
    return lam, gz, (None if gw is None else gw[:graph.nnz]), out


class PageRank(torch.autograd.Function):
    """x = (1 - d)(I - d P(w))^-1 Z with gradients for the link weights w and Z.

    forward(w, Z, n, ptr, idx, d, tol, adj_tol): ``ptr``/``idx`` a canonical
    out-CSR (rows sorted by target, no repeated link; e.g. from
    ``Graph.export_csr``) so that ``w`` (CUDA, one weight per link, > 0) is in
    the library's link order; ``Z`` a CUDA vector of n values.  The forward runs
    ``di_solve`` to ``tol``; the backward runs ``di_adjoint`` to ``adj_tol`` on
    the same graph.  x is float64; the gradients come back in the dtypes of w
    and Z.
    """

    @staticmethod
    def forward(ctx, w, Z, n, ptr, idx, d=0.85, tol=1e-12, adj_tol=1e-12):
        G = Graph(n, ptr, idx, w.detach())
        p, i, _ = G.export_csr(device=True, weights=False)
        if not (torch.equal(p.to(torch.int64), ptr.to(p.device, torch.int64))
                and torch.equal(i, idx.to(i.device, torch.int32))):
            raise ValueError("PageRank needs a canonical out-CSR (sorted rows, no repeated link)")
        st = State(G)
        x, info = st.solve(d, Z=Z.detach().to(_f64), tol=tol)
        if not info["converged"]:
            raise RuntimeError(f"di_solve did not converge: {info}")
        ctx.graph, ctx.d, ctx.adj_tol = G, d, adj_tol
        ctx.wdt, ctx.zdt = w.dtype, Z.dtype
        ctx.save_for_backward(x)
        st.close()
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, gz, gw, info = adjoint(ctx.graph, ctx.d, gx.detach().to(_f64).contiguous(), x, tol=ctx.adj_tol,
                                    want_grad_w=ctx.needs_input_grad[0])
        if not info["converged"]:
            raise RuntimeError(f"di_adjoint did not converge: {info}")
        gw_out = gw.to(ctx.wdt) if gw is not None else None
        gz_out = gz.to(ctx.zdt) if ctx.needs_input_grad[1] else None
        return gw_out, gz_out, None, None, None, None, None, None


def pagerank(w, Z, n, ptr, idx, d=0.85, tol=1e-12, adj_tol=1e-12):
    """Differentiable solve: see PageRank."""
    return PageRank.apply(w, Z, n, ptr, idx, d, tol, adj_tol)


def solve_batch(graph: Graph, Z, d: float = 0.85, tol: float = 1e-9, device: bool = True, **opts):
    """B personalised solves at once (Z: n x B, node-major, B <= 64).  Returns
    (H as n x B, per-column |F_c|_1, info)."""
    mem = L.DI_MEM_DEVICE if device else L.DI_MEM_HOST
    if isinstance(Z, torch.Tensor):
        B = int(Z.shape[1])
    else:
        Z = np.asarray(Z)
        B = int(Z.shape[1])
    Zp = _prep(Z.reshape(-1) if not isinstance(Z, torch.Tensor) else Z.reshape(-1), np.float64, _f64, mem)
    n = graph.n
    if device:
        H = torch.empty((n, B), dtype=_f64, device="cuda")
        res = torch.empty(B, dtype=_f64, device="cuda")
    else:
        H = np.empty((n, B), dtype=np.float64)
        res = np.empty(B, dtype=np.float64)
    info = L.di_info()
    o = L.default_opts(**opts)
    rc = L.lib().di_solve_batch(graph.handle, B, d, _p(Zp), tol, ctypes.byref(o), _p(H), _p(res),
                                ctypes.byref(info), mem, _stream())
    if rc not in (L.DI_OK, L.DI_ERR_NOT_CONVERGED):
        raise L.DIError(rc, "di_solve_batch")
    out = info.as_dict()
    out["converged"] = rc == L.DI_OK
    return H, res, out


def autotune(graph: Graph, d: float = 0.85, tol: float = 1e-9, precision: int = 0, budget: int = 20,
             cache: str | None = None):
    """Time candidate launch shapes on this graph and return (options dict for
    State.solve / solve, report dict).  See di_autotune in include/di.h."""
    o = L.di_opts()
    b, dm = ctypes.c_double(), ctypes.c_double()
    tr = ctypes.c_int32()
    L.check(L.lib().di_autotune(graph.handle, d, tol, precision, budget,
                                None if cache is None else cache.encode(), ctypes.byref(o), ctypes.byref(b),
                                ctypes.byref(dm), ctypes.byref(tr), _stream()), "di_autotune")
    opts = {k: getattr(o, k) for k in ("theta_factor", "hub_deg", "piece", "refine_ratio", "precision")}
    return opts, {"best_ms": b.value, "default_ms": dm.value, "trials": tr.value}
