"""Level-set evolution step (Eq. HJ, §2.1), FP64.

Test infrastructure (see oracle/__init__.py).

phi_t + v |grad phi| = 0 advanced by one explicit Euler step with the
first-order Godunov upwind approximation of |grad phi| (the standard
monotone scheme for this Hamilton-Jacobi equation, Osher & Sethian): with
one-sided differences D-_d phi = (phi_i - phi_{i-1})/h_d and
D+_d phi = (phi_{i+1} - phi_i)/h_d on the periodic node grid,

    |grad phi|+ = sqrt(sum_d max(D-_d, 0)^2 + min(D+_d, 0)^2)   (used where v > 0)
    |grad phi|- = sqrt(sum_d min(D-_d, 0)^2 + max(D+_d, 0)^2)   (used where v < 0)
    phi_new     = phi - dt (max(v, 0) |grad phi|+ + min(v, 0) |grad phi|-).

Arrays are (nz, ny, nx) on the unit cell, h_d = 1/n_d.
"""
from __future__ import annotations

import numpy as np


def hj_step(phi, v, dt):
    phi = np.asarray(phi, dtype=float)
    v = np.asarray(v, dtype=float)
    gp = np.zeros_like(phi)
    gm = np.zeros_like(phi)
    for axis in range(3):
        n = phi.shape[axis]
        dm = (phi - np.roll(phi, 1, axis)) * n
        dp = (np.roll(phi, -1, axis) - phi) * n
        gp += np.maximum(dm, 0.0) ** 2 + np.minimum(dp, 0.0) ** 2
        gm += np.minimum(dm, 0.0) ** 2 + np.maximum(dp, 0.0) ** 2
    return phi - dt * (np.maximum(v, 0.0) * np.sqrt(gp) + np.minimum(v, 0.0) * np.sqrt(gm))
