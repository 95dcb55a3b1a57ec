"""Material tensors: nondimensionalisation and the combined constitutive matrix.

Test infrastructure (see oracle/__init__.py).

§2.2 states that the coefficients differ by ~20 orders of magnitude (C ~ 1e11,
e ~ 1e1, kappa ~ 1e-9) and that the paper nondimensionalises them following
Cao & Neytcheva (2021), without printing the formula.  Reading taken here:

    C0 = max|C_pq|,  k0 = max|kappa_ij|,
    C^ = C / C0,  e^ = e / sqrt(C0 k0),  kappa^ = kappa / k0,

which is exactly the change of variables phi = sqrt(C0/k0) phi^ for the
potential together with scaling the mechanical equation by 1/C0.  The
homogenised tensors transform back with the same factors.
"""
from __future__ import annotations

import numpy as np


def scales(C, kappa):
    """Return (C0, k0) of the nondimensionalisation."""
    return float(np.abs(C).max()), float(np.abs(kappa).max())


def nondimensionalise(C, e, kappa):
    """(C, e, kappa) in SI -> (C^, e^, kappa^, (C0, k0))."""
    C0, k0 = scales(C, kappa)
    return C / C0, e / np.sqrt(C0 * k0), kappa / k0, (C0, k0)


def redimensionalise(Ch, eh, kh, sc):
    """Inverse of :func:`nondimensionalise` applied to homogenised tensors."""
    C0, k0 = sc
    return Ch * C0, eh * np.sqrt(C0 * k0), kh * k0


def constitutive(C, e, kappa):
    """9x9 symmetric matrix D of the bilinear form over (strain, grad phi).

    With sigma = C eps - e^T E, D_i = e eps + kappa E and E = -grad phi
    (§2.2), the integrand of the coupled bilinear form for trial (u, phi) and
    test (v, q) is

        eps(v):C eps(u) + eps(v):e^T grad(phi) + grad(q).e eps(u) - grad(q).kappa grad(phi)

    i.e. [eps(v); grad q]^T D [eps(u); grad phi] with D = [[C, e^T], [e, -kappa]].
    Strains are engineering Voigt vectors (eps11, eps22, eps33, 2eps23, 2eps13, 2eps12).
    """
    D = np.zeros((9, 9))
    D[:6, :6] = C
    D[:6, 6:] = e.T
    D[6:, :6] = e
    D[6:, 6:] = -kappa
    return D


def base_H(C, e, kappa):
    """The 9x9 matrix H = [[C, -e^T], [-e, -kappa]] that the nine unit loads
    produce for a homogeneous cell (what the homogenised H reduces to when the
    fluctuations vanish)."""
    H = np.zeros((9, 9))
    H[:6, :6] = C
    H[:6, 6:] = -e.T
    H[6:, :6] = -e
    H[6:, 6:] = -kappa
    return H
