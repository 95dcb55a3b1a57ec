"""Figures of merit of §2.3 and their gradients, FP64 host math.

Test infrastructure (see oracle/__init__.py).

* B_Voigt = C_iijj / 9,
* B_Reuss = 1 / S_iijj with S = C^-1 (Voigt form, engineering shear),
* d_h = d_zxx + d_zyy + d_zzz with d = e S  (in Voigt: d31 + d32 + d33).
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
    d/de_3p = (S m)_p and d/dC_ij = -(S e_3)_i (S m)_j (from dS = -S dC S).
    """
    S = np.linalg.inv(C)
    w = S @ M
    e3 = e[2]
    dC = -np.outer(S @ e3, w)
    de = np.zeros((3, 6))
    de[2] = w
    return dC, de
