"""Brute-force checks for tiny cells, FP64.

Test infrastructure (see oracle/__init__.py).

* ``gauss_eliminate``: dense Gaussian elimination with partial pivoting,
  written out, to solve the pinned system without SuperLU;
* ``element_matrix_brute``: the element matrix integrated with a 5-point
  Gauss rule per direction (exact far beyond the degree-2 integrand).
"""
from __future__ import annotations

import numpy as np

from . import fem


def gauss_eliminate(A, B):
    """Solve A X = B by Gaussian elimination with partial pivoting."""
    A = np.array(A, dtype=float)
    X = np.array(B, dtype=float)
    n = A.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p]] = A[[p, k]]
            X[[k, p]] = X[[p, k]]
        piv = A[k, k]
        f = A[k + 1:, k] / piv
        A[k + 1:, k:] -= np.outer(f, A[k, k:])
        X[k + 1:] -= np.outer(f, X[k])
    for k in range(n - 1, -1, -1):
        X[k] = (X[k] - A[k, k + 1:] @ X[k + 1:]) / A[k, k]
    return X


def solve_dense(P: "fem.CellProblem", pin_node=0):
    """Pinned solve of a small cell problem by dense elimination."""
    Kd = P.Kg.toarray()
    b = P.rhs()
    n = Kd.shape[0]
    fixed = np.arange(4 * pin_node, 4 * pin_node + 4)
    free = np.setdiff1d(np.arange(n), fixed)
    y = np.zeros_like(b)
    y[free] = gauss_eliminate(Kd[np.ix_(free, free)], b[free])
    return fem.project_means(y, P.shape)


def element_matrix_brute(C, e, kappa, h):
    return fem.element_matrix(C, e, kappa, h, npts=5)
