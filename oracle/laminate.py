"""Exact homogenisation of a layered cell, FP64 host math.

Test infrastructure (see oracle/__init__.py).

For rho depending only on the coordinate along one axis a, the cell problem of
§2.2 has a one-dimensional solution: the fields tangential to the layers
(strains eps_bb, gamma_bc with b,c != a, and fields E_b, b != a) are uniform
and equal to their macroscopic values, and the normal fluxes (sigma_aa,
sigma_ab, D_a) are uniform across layers.  Write the constitutive law as
flux = rho L x with x = (eps_Voigt, E), flux = (sigma, D) and
L = [[C, -e^T], [e, kappa]], and split x, flux into normal (n) and tangential
(t) parts.  Uniform normal flux q gives x_n = L_nn^-1 (q / rho - L_nt x_t) per
layer; averaging and imposing <x_n> = xbar_n yields

    q = rho_h (L_nn xbar_n + L_nt x_t),
    <flux_t> = rho_h (L_tn xbar_n + L_tt x_t) + (rho_a - rho_h) (L_tt - L_tn L_nn^-1 L_nt) x_t,

with rho_a = <rho> and rho_h = 1 / <1/rho>.  Hence

    L^H = rho_h L + (rho_a - rho_h) P_t (L_tt - L_tn L_nn^-1 L_nt) P_t^T.

Because rho is constant per element and the layers coincide with element
planes, the exact fluctuation is piecewise linear along the axis and lies in
the Q1 space, so the finite-element H equals this closed form at any mesh size.
"""
from __future__ import annotations

import numpy as np

# Voigt indices (of x = (eps11, eps22, eps33, g23, g13, g12, E1, E2, E3))
# whose conjugate fluxes are continuous across a plane normal to axis a.
_NORMAL = {0: [0, 4, 5, 6], 1: [1, 3, 5, 7], 2: [2, 3, 4, 8]}


def flux_matrix(C, e, kappa):
    L = np.zeros((9, 9))
    L[:6, :6] = C
    L[:6, 6:] = -e.T
    L[6:, :6] = e
    L[6:, 6:] = kappa
    return L


def laminate_tensors(C, e, kappa, layer_rho, axis):
    """Homogenised (C^H, e^H, kappa^H) of equal-thickness layers with scaling
    ``layer_rho`` stacked along ``axis`` (0=x, 1=y, 2=z)."""
    layer_rho = np.asarray(layer_rho, dtype=float)
    rho_a = layer_rho.mean()
    rho_h = 1.0 / (1.0 / layer_rho).mean()
    L = flux_matrix(C, e, kappa)
    n = _NORMAL[axis]
    t = [i for i in range(9) if i not in n]
    Ltt = L[np.ix_(t, t)]
    Ltn = L[np.ix_(t, n)]
    Lnt = L[np.ix_(n, t)]
    Lnn = L[np.ix_(n, n)]
    schur = Ltt - Ltn @ np.linalg.solve(Lnn, Lnt)
    LH = rho_h * L
    LH[np.ix_(t, t)] += (rho_a - rho_h) * schur
    Ch = LH[:6, :6]
    eh = LH[6:, :6]
    kh = LH[6:, 6:]
    return Ch, eh, kh, LH
