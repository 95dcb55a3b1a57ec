"""Smoothed-boundary ersatz material, FP64.

Test infrastructure (see oracle/__init__.py).

§2.6 says only that material properties are smoothed within two elements of
the zero level-set contour.  Reading taken here (the common smoothed
Heaviside of level-set topology optimisation):

    H_eta(s) = 0                                   s < -eta
             = (1 + s/eta + sin(pi s/eta)/pi) / 2  |s| <= eta
             = 1                                   s > eta

    rho_e = 1 - (1 - rho_void) H_eta(phi_e),

with eta = 2 h (h the largest element side), rho_void = 1e-3, and phi_e the
mean of the element's 8 nodal level-set values (the trilinear interpolant at
the element centre).  phi < 0 is solid (§2.1, Eq. 1), so rho -> 1 inside the
solid and rho -> rho_void in the void.  The same rho_e scales C, e and kappa.
"""
from __future__ import annotations

import numpy as np


def element_mean(phi):
    """Mean of the 8 periodic nodal values of each element; shape (nz,ny,nx)."""
    acc = np.zeros_like(phi, dtype=float)
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                acc += np.roll(np.roll(np.roll(phi, -c, 0), -b, 1), -a, 2)
    return acc / 8.0


def smoothed_heaviside(s, eta):
    s = np.asarray(s, dtype=float)
    out = np.where(s > eta, 1.0, 0.0)
    mid = np.abs(s) <= eta
    sm = s[mid] / eta
    out[mid] = 0.5 * (1.0 + sm + np.sin(np.pi * sm) / np.pi)
    return out


def rho_from_levelset(phi, rho_void=1e-3, eta=None):
    """Per-element ersatz scaling from nodal level-set values (nz,ny,nx)."""
    nz, ny, nx = phi.shape
    if eta is None:
        eta = 2.0 * max(1.0 / nx, 1.0 / ny, 1.0 / nz)
    return 1.0 - (1.0 - rho_void) * smoothed_heaviside(element_mean(phi), eta)


def smoothed_heaviside_deriv(s, eta):
    """dH_eta/ds = (1 + cos(pi s/eta)) / (2 eta) on |s| <= eta, 0 outside."""
    s = np.asarray(s, dtype=float)
    out = np.zeros_like(s)
    mid = np.abs(s) <= eta
    out[mid] = 0.5 * (1.0 + np.cos(np.pi * s[mid] / eta)) / eta
    return out


def _eta(phi, eta):
    nz, ny, nx = phi.shape
    return 2.0 * max(1.0 / nx, 1.0 / ny, 1.0 / nz) if eta is None else eta


def drho_dphi_e(phi, rho_void=1e-3, eta=None):
    """d rho_e / d phi_e per element (phi_e the element mean)."""
    return -(1.0 - rho_void) * smoothed_heaviside_deriv(element_mean(phi), _eta(phi, eta))


def grad_phi(phi, g_rho, rho_void=1e-3, eta=None):
    """Nodal dL/dphi from element dL/drho through the ersatz map: every
    element mean takes 1/8 of each of its 8 nodes, so node n collects
    g_e drho_e/dphi_e / 8 from the 8 elements that contain it."""
    ge = np.asarray(g_rho, dtype=float) * drho_dphi_e(phi, rho_void, eta)
    acc = np.zeros_like(ge)
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                # element (k, j, i) contains node (k + c, j + b, i + a)
                acc += np.roll(np.roll(np.roll(ge, c, 0), b, 1), a, 2)
    return acc / 8.0
