"""GB300 (sm_103a) library for the periodic piezoelectric cell problems of
level-set inverse homogenisation (arXiv 2410.03148, §2.2-§2.5).

The product is ``libcell.so`` with the C ABI of ``include/cell.h``; this
package holds its CUDA sources (``csrc/``), the build script and a thin
Python binding.  There is no CPU fallback: every call runs the library's
kernels, and importing the binding fails loudly if the library is missing.
"""
from ._binding import load  # noqa: F401

__all__ = ["load", "Cell", "dh", "figure", "hj_step", "solve_batch", "HomogeniseFn", "homogenise"]


def __getattr__(name):
    if name in ("Cell", "dh", "figure", "hj_step", "solve_batch"):
        from . import cell
        return getattr(cell, name)
    if name in ("HomogeniseFn", "homogenise"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
