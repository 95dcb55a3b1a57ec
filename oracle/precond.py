"""Blocks of the approximate-Schur-complement preconditioner P_SCP, FP64.

Test infrastructure (see oracle/__init__.py).

§2.5.3 preconditions the nonsymmetric form of Eq. (sym-piezo) with the block
lower-triangular P_SCP = [[A, 0], [-B, Sbar]], where A is the elastic block of
the coupled matrix and Sbar approximates the Schur complement
S = C + B A^-1 B^T element by element:

    Sbar = sum_e rho_e S0,   S0 = C_e + B_e (A_e + shift I)^-1 B_e^T,

with A_e, B_e, C_e the blocks of the unit element matrix (node-major local
dofs 4n + comp: the three displacement dofs of local node n and its potential
dof) and shift = 1e-10 (§2.5.3) making the singular A_e invertible.  The
functions below state these definitions directly; ``block_rows`` evaluates a
block product node by node from the element sum, for sampled checks on grids
too large to assemble.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

U_DOFS = [4 * n + c for n in range(8) for c in range(3)]   # local displacement dofs
P_DOFS = [4 * n + 3 for n in range(8)]                     # local potential dofs
CORNERS = [(n & 1, (n >> 1) & 1, n >> 2) for n in range(8)]  # local node n = a + 2b + 4c


def element_blocks(K0):
    """(A_e 24x24, B_e 8x24, C_e 8x8) of the symmetric element matrix
    [[A, B^T], [B, -C]]: note the minus sign of the potential-potential block."""
    A = K0[np.ix_(U_DOFS, U_DOFS)]
    Bm = K0[np.ix_(P_DOFS, U_DOFS)]
    Cm = -K0[np.ix_(P_DOFS, P_DOFS)]
    return A, Bm, Cm


def local_schur(K0, shift=1e-10):
    """S0 = C_e + B_e (A_e + shift I)^-1 B_e^T (§2.5.3), 8 x 8."""
    A, Bm, Cm = element_blocks(K0)
    return Cm + Bm @ np.linalg.solve(A + shift * np.eye(24), Bm.T)


def block_matrix(K0, block):
    """Element matrix of a preconditioner block: "A" -> A_e (24 x 24, local
    dof 3n + c), "Sbar" -> S0 (8 x 8)."""
    if block == "A":
        return element_blocks(K0)[0]
    return local_schur(K0)


def assemble_block(rho, Ke, nc, shape):
    """sum_e rho_e P_e^T Ke P_e for a block with nc dofs per node (CSR,
    nc N x nc N, global dof nc*node + comp)."""
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    dofs = np.zeros((i.size, 8 * nc), dtype=np.int64)
    for n, (a, b, c) in enumerate(CORNERS):
        node = (i + a) % nx + nx * (((j + b) % ny) + ny * ((k + c) % nz))
        for comp in range(nc):
            dofs[:, nc * n + comp] = nc * node + comp
    R = 8 * nc
    rows = np.repeat(dofs, R, axis=1).ravel()
    cols = np.tile(dofs, (1, R)).ravel()
    vals = (rho.ravel()[:, None, None] * Ke[None, :, :]).ravel()
    n = nc * i.size
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def block_rows(rho, Ke, nc, x, nodes):
    """(len(nodes), nc) values of y = sum_e rho_e P_e^T Ke P_e x at the given
    nodes (i, j, k): for each of the 8 elements around the node, the row of Ke
    belonging to the node's local corner times the element's nodal values.
    x has shape (nc, nz, ny, nx)."""
    nz, ny, nx = rho.shape
    out = np.zeros((len(nodes), nc))
    for q, (i, j, k) in enumerate(nodes):
        for (a, b, c) in CORNERS:          # the node is local corner (a, b, c) of element (i-a, j-b, k-c)
            ei, ej, ek = (i - a) % nx, (j - b) % ny, (k - c) % nz
            la = a + 2 * b + 4 * c
            xe = np.zeros(8 * nc)
            for lb, (a2, b2, c2) in enumerate(CORNERS):
                xe[nc * lb:nc * lb + nc] = x[:, (ek + c2) % nz, (ej + b2) % ny, (ei + a2) % nx]
            out[q] += rho[ek, ej, ei] * (Ke[nc * la:nc * la + nc] @ xe)
    return out
