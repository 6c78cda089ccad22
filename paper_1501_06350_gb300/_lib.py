"""ctypes binding of libdi.so: the C ABI of include/di.h under the same names.

Argument marshalling only.  Every step of the solver runs in the library's CUDA
kernels; when the library cannot be loaded this module raises, there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdi.so")

DI_OK = 0
DI_ERR_INVALID_ARG = 1
DI_ERR_BAD_GRAPH = 2
DI_ERR_OOM = 3
DI_ERR_NOT_CONVERGED = 4
DI_ERR_CUDA = 5
DI_ERR_DEVICE_TIMEOUT = 6

DI_LAYOUT_CSR = 0
DI_LAYOUT_CSC = 1
DI_W_NONE = 0
DI_W_F32 = 1
DI_W_F64 = 2
DI_MEM_HOST = 0
DI_MEM_DEVICE = 1
DI_PREC_F64 = 0
DI_PREC_F32 = 1


class di_opts(ctypes.Structure):
    _fields_ = [("theta_factor", ctypes.c_double), ("max_sweeps", ctypes.c_int64),
                ("check_every", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("normalize", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("refine_ratio", ctypes.c_double),
                ("hub_deg", ctypes.c_int32), ("piece", ctypes.c_int32)]


class di_info(ctypes.Structure):
    _fields_ = [("resid_l1", ctypes.c_double), ("l_dangling", ctypes.c_double),
                ("bound", ctypes.c_double), ("bound_completed", ctypes.c_double),
                ("sweeps", ctypes.c_int64), ("diffusions", ctypes.c_int64),
                ("edge_pushes", ctypes.c_int64), ("time_ms", ctypes.c_double),
                ("push_ms", ctypes.c_double), ("push_launches", ctypes.c_int64),
                ("push_edges", ctypes.c_int64), ("push_entries", ctypes.c_int64),
                ("refinements", ctypes.c_int64), ("refine_links", ctypes.c_int64),
                ("resid_inf", ctypes.c_double), ("push_hot_links", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class DIError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = lib().di_status_str(status).decode() if _LIB is not None else str(status)
        extra = ""
        if status == DI_ERR_CUDA and _LIB is not None:
            extra = f" (cudaError {_LIB.di_last_cuda_error()})"
        super().__init__(f"{where}: {name}{extra}")


_LIB = None
P = ctypes.c_void_p
I64 = ctypes.c_int64
INT = ctypes.c_int

# name -> (restype, argtypes), exactly the declarations of include/di.h
SIGNATURES = {
    "di_opts_default": (None, [ctypes.POINTER(di_opts)]),
    "di_status_str": (ctypes.c_char_p, [INT]),
    "di_last_cuda_error": (INT, []),
    "di_kernel_launches": (I64, []),
    "di_probe_atomic_adds": (INT, [INT, ctypes.POINTER(ctypes.c_double), P]),
    "di_graph_create": (INT, [I64, I64, P, P, P, INT, INT, INT, P, ctypes.POINTER(P)]),
    "di_graph_destroy": (INT, [P]),
    "di_graph_info": (INT, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                            ctypes.POINTER(INT)]),
    "di_graph_export_csr": (INT, [P, P, P, P, INT, P]),
    "di_graph_export_csc": (INT, [P, P, P, P, INT, P]),
    "di_state_create": (INT, [P, ctypes.POINTER(P)]),
    "di_state_destroy": (INT, [P]),
    "di_solve": (INT, [P, P, ctypes.c_double, P, ctypes.c_double, ctypes.POINTER(di_opts), P,
                       ctypes.POINTER(di_info), INT, P]),
    "di_resume": (INT, [P, P, ctypes.c_double, ctypes.POINTER(di_opts), P, ctypes.POINTER(di_info),
                        INT, P]),
    "di_update_edges": (INT, [P, P, I64, P, P, P, P, INT, P]),
    "di_state_export": (INT, [P, P, P, P, INT, P]),
    "di_state_import": (INT, [P, P, P, ctypes.c_double, INT, P]),
    "di_autotune": (INT, [P, ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                          ctypes.POINTER(di_opts), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), P]),
    "di_solve_batch": (INT, [P, ctypes.c_int32, ctypes.c_double, P, ctypes.c_double, ctypes.POINTER(di_opts),
                             P, P, ctypes.POINTER(di_info), INT, P]),
    "di_adjoint": (INT, [P, ctypes.c_double, P, P, ctypes.c_double, ctypes.POINTER(di_opts), P, P, P,
                         ctypes.POINTER(di_info), INT, P]),
    "di_frontier_select": (INT, [P, P, ctypes.c_double, P, ctypes.POINTER(I64), INT, P]),
    "di_residual_l1": (INT, [P, P, P, INT, P]),
    "di_residual_l1_noalloc": (INT, [P, P, P, P]),
}


def lib() -> ctypes.CDLL:
    """Load libdi.so (built by ``paper_1501_06350_gb300.build``); raise if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; "
                               f"g.build()'` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status: int, where: str) -> int:
    if status != DI_OK:
        raise DIError(status, where)
    return status


def default_opts(**kw) -> di_opts:
    o = di_opts()
    lib().di_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o
