"""Element-wise sensitivities of the homogenised tensors, FP64.

Test infrastructure (see oracle/__init__.py).

The paper's shape derivatives sit in its (absent) supplementary material; the
quantity checked here is the derivative with respect to each element's
ersatz scale rho_e, which any level-set shape derivative of this discretised
problem goes through.

The energy form H_IJ = sum_e rho_e W_e^I . K W_e^J (W = total nodal field)
is stationary with respect to the fluctuations (the discrete cell equations
are exactly its first variation), so the implicit dependence of W on rho
drops out and

    dH_IJ / drho_e = W_e^I . K W_e^J,

i.e. the adjoint states are the nine cell solutions themselves.  For a scalar
L = sum_IJ G_IJ H_IJ:  g_e = sum_IJ G_IJ W_e^I . K W_e^J.
"""
from __future__ import annotations

import numpy as np

from . import fem, material


def element_quadforms(P: "fem.CellProblem", y):
    """(E, 9, 9) array of W_e^I . K W_e^J (nondimensional)."""
    dofs = fem.element_dofs(P.shape)
    W = P.Zbar[None] + y[dofs]
    KW = np.einsum("ab,ebJ->eaJ", P.K, W)
    return np.einsum("eaI,eaJ->eIJ", W, KW)


def grad_rho(P, y, G):
    """g_e = sum_IJ G_IJ dH_IJ/drho_e, shape (nz, ny, nx)."""
    Q = element_quadforms(P, y)
    return np.einsum("IJ,eIJ->e", G, Q).reshape(P.shape)


def G_from_si(dC, de, dk, sc):
    """Upstream gradients with respect to the SI tensors -> G with respect to
    the nondimensional H = [[C^, -e^^T], [-e^, -kappa^]].

    C^H = C0 H[:6,:6];  e^H = -sqrt(C0 k0) H[6:, :6] (split evenly between the
    two symmetric blocks of H);  kappa^H = -k0 H[6:, 6:].
    """
    C0, k0 = sc
    se = np.sqrt(C0 * k0)
    G = np.zeros((9, 9))
    G[:6, :6] = C0 * dC
    G[6:, :6] = -0.5 * se * de
    G[:6, 6:] = -0.5 * se * de.T
    G[6:, 6:] = -k0 * dk
    return G


def fd_grad(rho, C, e, kappa, G, elements, step=1e-6):
    """Central finite differences of L(rho) = sum G_IJ H_IJ(rho) at the given
    flat element indices, each from two direct solves."""
    out = []
    flat = rho.ravel()
    for idx in elements:
        vals = []
        for s in (+1.0, -1.0):
            r = flat.copy()
            r[idx] += s * step
            P = fem.CellProblem(r.reshape(rho.shape), C, e, kappa)
            y = P.solve()
            Q = element_quadforms(P, y)
            # sum element-wise contributions (energy form), compensated
            contrib = np.einsum("IJ,eIJ->e", G, Q) * r
            vals.append(contrib)
        diff = vals[0] - vals[1]
        out.append(_fsum(diff) / (2 * step))
    return np.array(out)


def _fsum(a):
    import math
    return math.fsum(a.tolist())
