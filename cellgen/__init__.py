"""Seeded synthetic inputs for the periodic piezoelectric unit-cell problem.

This module is shared by the CUDA library's tests and benchmark and by the CPU
oracle.  It holds *inputs only*: material constant tables, seeded level-set
fields on the periodic node grid, and seeded per-element scaling fields.  None
of the homogenisation method's arithmetic (element matrices, ersatz mapping,
assembly, solves, reductions) lives here.

Grid conventions (shared by every consumer):

* the unit cell [0,1)^3 carries nx*ny*nz periodic nodes at x = (i/nx, j/ny, k/nz);
* arrays are C-ordered with shape (nz, ny, nx), so x is the fastest index;
* element (i,j,k) spans nodes (i+a, j+b, k+c) mod (nx,ny,nz), a,b,c in {0,1};
  element arrays use the same (nz, ny, nx) shape as node arrays.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "pzt5h_class", "pzt5a", "gaussian_levelset", "e1_levelset",
    "laminate_rho", "random_rho", "PZT5A_DH_PC_PER_N",
]

# Hydrostatic strain coefficient of the paper's base PZT-5A, printed in §2.3
# (value quoted in pC/N, three significant figures).
PZT5A_DH_PC_PER_N = 31.7


def pzt5h_class():
    """Transversely isotropic (z-poled) PZT-5H-class constants in SI units.

    Returns (C [6x6, Pa], e [3x6, C/m^2], kappa [3x3, F/m]) in IEEE Voigt
    order (11, 22, 33, 23, 13, 12).  Entries fixed by transverse isotropy
    about z are filled in (C22=C11, C23=C13, C55=C44, e32=e31, e24=e15,
    kappa22=kappa11); C66 is taken as given, not from (C11-C12)/2.
    """
    GPa = 1e9
    C11, C12, C13, C33, C44, C66 = 127.205, 80.212, 84.670, 117.436, 22.988, 23.474
    C = np.zeros((6, 6))
    C[0, 0] = C[1, 1] = C11
    C[0, 1] = C[1, 0] = C12
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = C13
    C[2, 2] = C33
    C[3, 3] = C[4, 4] = C44
    C[5, 5] = C66
    C *= GPa
    e = np.zeros((3, 6))
    e[2, 0] = e[2, 1] = -6.62
    e[2, 2] = 23.24
    e[0, 4] = e[1, 3] = 17.03
    kappa = np.diag([1.503e-8, 1.503e-8, 1.300e-8])
    return C, e, kappa


def pzt5a():
    """The paper's z-poled PZT-5A base material (§2.3), SI units, IEEE Voigt order."""
    C = np.array([
        [12.04, 7.52, 7.51, 0, 0, 0],
        [7.52, 12.04, 7.51, 0, 0, 0],
        [7.51, 7.51, 11.09, 0, 0, 0],
        [0, 0, 0, 2.1, 0, 0],
        [0, 0, 0, 0, 2.1, 0],
        [0, 0, 0, 0, 0, 2.3],
    ]) * 1e10
    e = np.array([
        [0, 0, 0, 0, 12.3, 0],
        [0, 0, 0, 12.3, 0, 0],
        [-5.4, -5.4, 15.8, 0, 0, 0],
    ])
    kappa = np.diag([4.78, 4.78, 7.35]) * 1e-9
    return C, e, kappa


def _node_coords(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                          indexing="ij")
    return x, y, z


def _normalise_by_interface_gradient(phi, shape):
    """Divide phi by the mean finite-difference gradient magnitude over the
    elements whose 8 nodal values change sign, so that phi behaves like a
    distance near its zero contour (a cheap stand-in for reinitialisation)."""
    nz, ny, nx = shape
    p = phi
    # forward differences averaged over the 4 parallel edges of each element
    def sh(a, dz, dy, dx):
        return np.roll(np.roll(np.roll(a, -dz, 0), -dy, 1), -dx, 2)
    corners = [sh(p, c, b, a) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    gx = sum(corners[i + 1] - corners[i] for i in (0, 2, 4, 6)) / 4.0 * nx
    gy = sum(corners[i + 2] - corners[i] for i in (0, 1, 4, 5)) / 4.0 * ny
    gz = sum(corners[i + 4] - corners[i] for i in (0, 1, 2, 3)) / 4.0 * nz
    stack = np.stack(corners)
    cut = (stack.min(0) < 0) & (stack.max(0) > 0)
    if not cut.any():
        return phi
    g = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)[cut].mean()
    return phi / g


def gaussian_levelset(shape, seed: int, n_bumps: int = 8) -> np.ndarray:
    """Seeded level set: threshold minus a sum of periodic Gaussian bumps.

    phi(x) = tau - sum_k a_k exp(-d(x, c_k)^2 / (2 s_k^2)) with d the
    minimum-image periodic distance, centres c_k ~ U[0,1)^3, amplitudes
    a_k ~ U[0.5, 1], widths s_k ~ U[0.08, 0.2]; tau is the median of the bump
    sum over nodes so that about half the cell is solid (phi < 0).  The result
    is normalised so that |grad phi| is about 1 near the interface.
    Returns nodal values, shape (nz, ny, nx), float64.
    """
    if isinstance(shape, int):
        shape = (shape, shape, shape)
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, size=(n_bumps, 3))
    a = rng.uniform(0.5, 1.0, size=n_bumps)
    s = rng.uniform(0.08, 0.2, size=n_bumps)
    x, y, z = _node_coords(shape)
    tot = np.zeros(shape)
    for k in range(n_bumps):
        d2 = 0.0
        for coord, ck in ((x, c[k, 0]), (y, c[k, 1]), (z, c[k, 2])):
            d = coord - ck
            d -= np.round(d)
            d2 = d2 + d * d
        tot += a[k] * np.exp(-d2 / (2.0 * s[k] ** 2))
    tau = np.median(tot)
    return _normalise_by_interface_gradient(tau - tot, shape)


def e1_levelset(shape, normalise: bool = True) -> np.ndarray:
    """The weak-scaling benchmark geometry of §2.5.4 (also the initial design of
    Fig. 1): phi = -cos(2 pi x) cos(2 pi y) cos(2 pi z) - 0.2, at the nodes.
    With ``normalise`` the field is rescaled to unit mean interface gradient."""
    if isinstance(shape, int):
        shape = (shape, shape, shape)
    x, y, z = _node_coords(shape)
    phi = -np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.cos(2 * np.pi * z) - 0.2
    return _normalise_by_interface_gradient(phi, shape) if normalise else phi


def laminate_rho(shape, axis: int, seed: int, lo: float = 1e-3, hi: float = 1.0) -> np.ndarray:
    """Per-element scaling that depends only on the element index along ``axis``
    (0 = x, 1 = y, 2 = z): a seeded layered design, shape (nz, ny, nx)."""
    if isinstance(shape, int):
        shape = (shape, shape, shape)
    rng = np.random.default_rng(seed)
    n_axis = shape[2 - axis]
    layers = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_axis))
    view = [1, 1, 1]
    view[2 - axis] = n_axis
    return np.broadcast_to(layers.reshape(view), shape).copy()


def random_rho(shape, seed: int, lo: float = 1e-3, hi: float = 1.0) -> np.ndarray:
    """Seeded per-element scaling, log-uniform in [lo, hi], shape (nz, ny, nx)."""
    if isinstance(shape, int):
        shape = (shape, shape, shape)
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=shape))
