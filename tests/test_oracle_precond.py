"""Pins of the oracle's preconditioner blocks (§2.5.3) against identities that
do not restate their formulas (no GPU).

* S0 is the Schur complement of the element matrix: eliminating the
  displacements of [[A, B^T], [B, -C]] (applied as a matrix, not blockwise)
  leaves -S0 on the potential rows; the shifted inverse agrees with the
  pseudo-inverse route; constants span its kernel.
* The generic block assembler reproduces the displacement-displacement block
  of the full assembly, and its node-by-node evaluation (block_rows) matches
  the assembled product.
"""
import numpy as np
import pytest

import cellgen
from oracle import fem, material, precond


def _K0(shape=(4, 4, 4), mat=None):
    C, e, k = mat or cellgen.pzt5h_class()
    Cn, en, kn, _ = material.nondimensionalise(C, e, k)
    return fem.element_matrix(Cn, en, kn, fem.cell_h(shape))


@pytest.mark.parametrize("mat", [cellgen.pzt5h_class(), cellgen.pzt5a()])
def test_local_schur_is_elimination_of_displacements(mat):
    K0 = _K0(mat=mat)
    S0 = precond.local_schur(K0, shift=1e-10)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(8)
    # u* minimises the (shifted) displacement energy for the given potential
    A = K0[np.ix_(precond.U_DOFS, precond.U_DOFS)] + 1e-10 * np.eye(24)
    rhs = -K0[np.ix_(precond.U_DOFS, precond.P_DOFS)] @ phi
    u = np.linalg.lstsq(A, rhs, rcond=None)[0]
    v = np.zeros(32)
    v[precond.U_DOFS] = u
    v[precond.P_DOFS] = phi
    y = K0 @ v
    scale = np.abs(S0).max() * np.abs(phi).max()
    np.testing.assert_allclose(y[precond.P_DOFS], -S0 @ phi, atol=1e-8 * scale)
    np.testing.assert_allclose(y[precond.U_DOFS], 1e-10 * u, atol=1e-8 * scale)


def test_local_schur_pinv_route_and_kernel():
    K0 = _K0()
    S0 = precond.local_schur(K0)
    uu, pp = precond.U_DOFS, precond.P_DOFS
    A = K0[np.ix_(uu, uu)]
    Bm = K0[np.ix_(pp, uu)]
    S_pinv = -K0[np.ix_(pp, pp)] + Bm @ np.linalg.pinv(A, rcond=1e-12) @ Bm.T
    assert np.abs(S0 - S_pinv).max() < 1e-7 * np.abs(S0).max()
    np.testing.assert_allclose(S0 @ np.ones(8), 0.0, atol=1e-12 * np.abs(S0).max())
    ev = np.linalg.eigvalsh(0.5 * (S0 + S0.T))
    assert abs(ev[0]) < 1e-10 * ev[-1] and ev[1] > 0


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 2, 2)])
def test_block_assembly_matches_full_assembly(shape):
    rho = cellgen.random_rho(shape, seed=4)
    K0 = _K0(shape)
    Kg = fem.assemble(rho, K0, shape)
    nn = int(np.prod(shape))
    u_global = [4 * n + c for n in range(nn) for c in range(3)]
    Auu = Kg[u_global][:, u_global]
    Ab = precond.assemble_block(rho, precond.block_matrix(K0, "A"), 3, shape)
    assert abs(Auu - Ab).max() < 1e-14 * abs(Auu).max()


@pytest.mark.parametrize("block,nc", [("A", 3), ("Sbar", 1)])
def test_block_rows_match_assembled_product(block, nc):
    shape = (3, 5, 4)
    rho = cellgen.random_rho(shape, seed=5)
    Ke = precond.block_matrix(_K0(shape), block)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((nc,) + shape)
    Ab = precond.assemble_block(rho, Ke, nc, shape)
    y = Ab @ np.moveaxis(x, 0, -1).ravel()          # node-major, comp fastest
    y = np.moveaxis(y.reshape(shape + (nc,)), -1, 0)
    nodes = [(0, 0, 0), (3, 4, 2), (1, 2, 1), (3, 0, 2)]
    got = precond.block_rows(rho, Ke, nc, x, nodes)
    want = np.array([y[:, k, j, i] for (i, j, k) in nodes])
    np.testing.assert_allclose(got, want, atol=1e-13 * np.abs(y).max())


def test_sbar_uniform_row_sums_vanish():
    """Constants are in the kernel of every S0, so of Sbar for any rho."""
    shape = (4, 3, 5)
    rho = cellgen.random_rho(shape, seed=6)
    S = precond.assemble_block(rho, precond.local_schur(_K0(shape)), 1, shape)
    assert np.abs(S @ np.ones(S.shape[0])).max() < 1e-12 * abs(S).max()
