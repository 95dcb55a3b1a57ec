"""Q1 finite elements for the periodic piezoelectric cell problem, FP64.

Test infrastructure (see oracle/__init__.py).

State equations (§2.2): -div sigma = 0, div D = 0 on the periodic unit cell,
sigma = C eps - e^T E, D = e eps + kappa E, E = -grad phi, with the total
fields split into a macroscopic part (one of nine unit loads, §2.2: the six
unit strains eps^(kl) = (d_ik d_jl + d_il d_jk)/2 and the three unit fields
E^(j) = d_ij) plus a periodic fluctuation.  The supplementary material with the
weak form is not part of the paper text; the weak form used here follows
directly from the state equations: find periodic (u~, phi~) such that for all
periodic (v, q)

    a((u~, phi~), (v, q)) = -a((u_bar, phi_bar), (v, q)),

with a(.,.) the bilinear form of ``material.constitutive`` and (u_bar, phi_bar)
the affine fields u_bar = eps_bar x, phi_bar = -E_bar . x.  Its matrix is the
symmetric indefinite block matrix [[A, B^T], [B, -C]] of Eq. (sym-piezo).  All
blocks are scaled by the element's ersatz factor rho_e (§2.6).

Discretisation: the unit cell is split into nx*ny*nz boxes of size
(1/nx, 1/ny, 1/nz) carrying trilinear (Q1) elements; nodes are periodic, so
there are nx*ny*nz nodes with 4 dofs each, ordered node-major (u1, u2, u3, phi):
global dof = 4*node + comp, node = i + nx*(j + ny*k).  Within an element the
local node n = a + 2b + 4c sits at the corner (a, b, c) and the local dof is
4*n + comp.

The right-hand side is assembled element by element from the affine fields
written in element-local coordinates: constants are in the kernel of every
element matrix, so the local and global affine fields give the same element
load vector, and the local one is periodic-compatible.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import material

# --------------------------------------------------------------------------
# element level
# --------------------------------------------------------------------------

CORNERS = np.array([(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=float)


def shape_gradients(xi):
    """Gradients of the 8 trilinear shape functions on the reference cube
    [0,1]^3 at reference point xi (3,), returned as (8, 3)."""
    g = np.zeros((8, 3))
    for n, (a, b, c) in enumerate(CORNERS):
        f = [xi[0] if a else 1 - xi[0], xi[1] if b else 1 - xi[1], xi[2] if c else 1 - xi[2]]
        d = [1.0 if a else -1.0, 1.0 if b else -1.0, 1.0 if c else -1.0]
        g[n, 0] = d[0] * f[1] * f[2]
        g[n, 1] = f[0] * d[1] * f[2]
        g[n, 2] = f[0] * f[1] * d[2]
    return g


def b_matrix(dN):
    """9x32 matrix mapping local dofs to (engineering Voigt strain, grad phi)
    given physical shape-function gradients dN (8, 3)."""
    B = np.zeros((9, 32))
    for n in range(8):
        gx, gy, gz = dN[n]
        c = 4 * n
        B[0, c + 0] = gx            # eps11
        B[1, c + 1] = gy            # eps22
        B[2, c + 2] = gz            # eps33
        B[3, c + 1] = gz            # gamma23 = du2/dz + du3/dy
        B[3, c + 2] = gy
        B[4, c + 0] = gz            # gamma13 = du1/dz + du3/dx
        B[4, c + 2] = gx
        B[5, c + 0] = gy            # gamma12 = du1/dy + du2/dx
        B[5, c + 1] = gx
        B[6, c + 3] = gx            # grad phi
        B[7, c + 3] = gy
        B[8, c + 3] = gz
    return B


def gauss_points(npts):
    """Tensor Gauss-Legendre rule on [0,1]^3: (points (q,3), weights (q,))."""
    x, w = np.polynomial.legendre.leggauss(npts)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for k in range(npts):
        for j in range(npts):
            for i in range(npts):
                pts.append((x[i], x[j], x[k]))
                wts.append(w[i] * w[j] * w[k])
    return np.array(pts), np.array(wts)


def element_matrix(C, e, kappa, h, npts=2):
    """32x32 element matrix K = int_box B^T D B dx of a box with sides h=(hx,hy,hz).

    2x2x2 Gauss integration is exact: the integrand is a product of two
    Q1 gradients, of degree <= 2 in each coordinate.
    """
    h = np.asarray(h, dtype=float)
    D = material.constitutive(C, e, kappa)
    pts, wts = gauss_points(npts)
    K = np.zeros((32, 32))
    vol = h.prod()
    for p, w in zip(pts, wts):
        dN = shape_gradients(p) / h[None, :]
        B = b_matrix(dN)
        K += (w * vol) * (B.T @ D @ B)
    return K


def unit_strain(p):
    """Symmetric 3x3 macroscopic strain of the Voigt unit load p (0..5) of §2.2:
    eps^(kl)_ij = (d_ik d_jl + d_il d_jk)/2 for (kl) = 11,22,33,23,13,12."""
    kl = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)][p]
    E = np.zeros((3, 3))
    k, l = kl
    E[k, l] += 0.5
    E[l, k] += 0.5
    return E


def affine_loads(h):
    """32x9 nodal values of the nine affine macroscopic fields in element-local
    coordinates: columns 0..5 are u_bar = eps^(p) x for the unit strains,
    columns 6..8 are phi_bar = -x_j for the unit fields E^(j)."""
    h = np.asarray(h, dtype=float)
    Z = np.zeros((32, 9))
    for n in range(8):
        x = CORNERS[n] * h
        for p in range(6):
            Z[4 * n:4 * n + 3, p] = unit_strain(p) @ x
        for j in range(3):
            Z[4 * n + 3, 6 + j] = -x[j]
    return Z


# --------------------------------------------------------------------------
# mesh level
# --------------------------------------------------------------------------

def element_dofs(shape):
    """(E, 32) global dof indices of every element; shape = (nz, ny, nx)."""
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    dofs = np.zeros((i.size, 32), dtype=np.int64)
    for n, (a, b, c) in enumerate(CORNERS.astype(int)):
        node = (i + a) % nx + nx * (((j + b) % ny) + ny * ((k + c) % nz))
        for comp in range(4):
            dofs[:, 4 * n + comp] = 4 * node + comp
    return dofs


def cell_h(shape):
    nz, ny, nx = shape
    return np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])


def assemble(rho, K, shape):
    """Global sparse matrix sum_e rho_e P_e^T K P_e (CSR, 4N x 4N)."""
    dofs = element_dofs(shape)
    r = rho.ravel()
    E = dofs.shape[0]
    rows = np.repeat(dofs, 32, axis=1).ravel()
    cols = np.tile(dofs, (1, 32)).ravel()
    vals = (r[:, None, None] * K[None, :, :]).ravel()
    n = 4 * E
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def rhs(rho, K, Zbar, shape):
    """(4N, 9) right-hand sides b^I = -sum_e rho_e P_e^T K Zbar^I."""
    dofs = element_dofs(shape)
    r = rho.ravel()
    fe = -(K @ Zbar)                                   # (32, 9)
    b = np.zeros((4 * dofs.shape[0], 9))
    np.add.at(b, dofs.ravel(), (r[:, None, None] * fe[None]).reshape(-1, 9))
    return b


def project_means(y, shape):
    """Subtract the mean of each of the 4 nodal components, per load column.
    This removes the null space (3 rigid translations, 1 constant potential)."""
    y = y.copy()
    for comp in range(4):
        y[comp::4] -= y[comp::4].mean(axis=0, keepdims=True)
    return y


def solve_pinned(Kg, b, pin_node=0):
    """Solve the singular, consistent periodic system by fixing the 4 dofs of
    one node to zero and factorising the rest directly (SuperLU)."""
    n = Kg.shape[0]
    fixed = np.arange(4 * pin_node, 4 * pin_node + 4)
    free = np.setdiff1d(np.arange(n), fixed)
    Kff = Kg[free][:, free].tocsc()
    lu = spla.splu(Kff, permc_spec="MMD_AT_PLUS_A")
    y = np.zeros_like(b)
    y[free] = lu.solve(np.ascontiguousarray(b[free]))
    return y


def homogenise(rho, K, Zbar, y, shape):
    """Homogenised 9x9 H from the fluctuation solutions y (4N, 9).

    Returns (H_energy, H_linear):
      H_energy_IJ = sum_e rho_e W_e^I . K W_e^J,  W = Zbar + y_e   (total fields),
      H_linear_IJ = sum_e rho_e Zbar^I . K W_e^J                   (Eqs. hom_C/e/kappa).
    Both equal [[C^H, -e^H^T], [-e^H, -kappa^H]] at the exact discrete solution
    (Vol(D) = 1); the energy form's error is quadratic in the solve error.
    """
    dofs = element_dofs(shape)
    W = Zbar[None, :, :] + y[dofs]                     # (E, 32, 9)
    KW = np.einsum("ab,ebJ->eaJ", K, W)
    r = rho.ravel()
    Hen = np.einsum("e,eaI,eaJ->IJ", r, W, KW)
    Hlin = np.einsum("e,aI,eaJ->IJ", r, Zbar, KW)
    return Hen, Hlin


def split_H(H):
    """H -> (C^H [6x6], e^H [3x6], kappa^H [3x3]); e^H is read from the
    field-load rows (the electric displacement produced by the unit strains)."""
    return H[:6, :6].copy(), -H[6:, :6].copy(), -H[6:, 6:].copy()


def e_from_strain_and_field(H):
    """The two readings of e^H: from <D> under unit strains and from -<sigma>
    under unit fields; reciprocity makes them equal."""
    return -H[6:, :6], -H[:6, 6:].T


class CellProblem:
    """Assembled problem for one design (nondimensional units unless
    ``nondim=False``)."""

    def __init__(self, rho, C, e, kappa, nondim=True):
        rho = np.asarray(rho, dtype=float)
        self.shape = rho.shape
        self.rho = rho
        if nondim:
            self.Cn, self.en, self.kn, self.sc = material.nondimensionalise(C, e, kappa)
        else:
            self.Cn, self.en, self.kn, self.sc = C, e, kappa, (1.0, 1.0)
        self.h = cell_h(self.shape)
        self.K = element_matrix(self.Cn, self.en, self.kn, self.h)
        self.Zbar = affine_loads(self.h)
        self._Kg = None

    @property
    def Kg(self):
        if self._Kg is None:
            self._Kg = assemble(self.rho, self.K, self.shape)
        return self._Kg

    def rhs(self):
        return rhs(self.rho, self.K, self.Zbar, self.shape)

    def solve(self, pin_node=0, project=True):
        y = solve_pinned(self.Kg, self.rhs(), pin_node)
        return project_means(y, self.shape) if project else y

    def homogenise(self, y):
        return homogenise(self.rho, self.K, self.Zbar, y, self.shape)

    def tensors(self, H):
        """Nondimensional H -> SI (C^H, e^H, kappa^H)."""
        Ch, eh, kh = split_H(H)
        return material.redimensionalise(Ch, eh, kh, self.sc)


def solve_cell(rho, C, e, kappa, nondim=True):
    """Full oracle pipeline: returns dict with SI tensors and the raw H's."""
    P = CellProblem(rho, C, e, kappa, nondim=nondim)
    y = P.solve()
    Hen, Hlin = P.homogenise(y)
    Ch, eh, kh = P.tensors(Hen)
    return {"C": Ch, "e": eh, "kappa": kh, "H": Hen, "H_lin": Hlin, "y": y, "problem": P}
