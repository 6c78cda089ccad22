"""D-Iteration (arXiv:1501.06350) on one GB300: a fluid-diffusion PageRank solver
with its hot path in hand-written sm_103a CUDA behind the C ABI of include/di.h.

Submodules: ``di`` (Graph/State over torch tensors or NumPy arrays), ``_lib``
(ctypes binding, same names as the C ABI), ``build`` (nvcc build of libdi.so),
``synth`` (seeded synthetic inputs).  Importing the package loads nothing; the
first call that needs libdi.so loads it and fails loudly when it is missing.
"""
import importlib

__all__ = ["Graph", "State", "solve", "solve_batch", "autotune", "frontier_select", "residual_l1", "adjoint", "PageRank",
           "pagerank"]


def __getattr__(name):
    if name in __all__:
        return getattr(importlib.import_module(".di", __name__), name)
    raise AttributeError(name)
