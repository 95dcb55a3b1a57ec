"""Figures of merit of §2.3 and their gradients, FP64 host math.

Test infrastructure (see oracle/__init__.py).

* B_Voigt = C_iijj / 9,
* B_Reuss = 1 / S_iijj with S = C^-1 (Voigt form, engineering shear),
* d_h = d_zxx + d_zyy + d_zzz with d = e S  (in Voigt: d31 + d32 + d33),
* C_zzzz = C_33 (Voigt), the stiffness along the poling direction z (§2.3).

Gradients treat every Voigt entry of C (and e) as an independent variable,
as the upstream gradients of the element sensitivities do.
"""
from __future__ import annotations

import numpy as np

M = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def b_voigt(C):
    return float(M @ C @ M) / 9.0


def b_reuss(C):
    S = np.linalg.inv(C)
    return 1.0 / float(M @ S @ M)


def d_tensor(C, e):
    return e @ np.linalg.inv(C)


def d_h(C, e):
    return float(d_tensor(C, e)[2, :3].sum())


def d_h_grad(C, e):
    """(d d_h / dC [6x6], d d_h / de [3x6]) treating every entry as independent.

    d_h = e_3 . S m with e_3 the third row of e and m = (1,1,1,0,0,0):
    d/de_3p = (S m)_p and d/dC_ij = -(S^T e_3)_i (S m)_j (from dS = -S dC S).
    """
    S = np.linalg.inv(C)
    w = S @ M
    e3 = e[2]
    dC = -np.outer(S.T @ e3, w)
    de = np.zeros((3, 6))
    de[2] = w
    return dC, de


def c_zzzz(C):
    return float(C[2, 2])


def b_voigt_grad(C):
    """d B_Voigt / dC: 1/9 on the normal-normal block."""
    return np.outer(M, M) / 9.0


def b_reuss_grad(C):
    """d B_Reuss / dC = B_Reuss^2 (S^T m)(S m)^T, from dS = -S dC S."""
    S = np.linalg.inv(C)
    b = b_reuss(C)
    return b * b * np.outer(S.T @ M, S @ M)


def c_zzzz_grad(C):
    g = np.zeros((6, 6))
    g[2, 2] = 1.0
    return g
