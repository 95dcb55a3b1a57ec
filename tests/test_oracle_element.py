"""Pins of the oracle's element level against closed forms (no GPU).

A wrong sign, index or dropped term in the B matrix, the constitutive matrix,
the quadrature or the affine loads fails at least one of these.
"""
import numpy as np
import pytest

import cellgen
from oracle import dense, ersatz, fem, material


def _materials():
    return [cellgen.pzt5h_class(), cellgen.pzt5a()]


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.25, 0.25, 0.25), (0.5, 1.0, 2.0)])
def test_affine_energy_equals_material(h):
    """For each pair of unit loads the element energy of the affine fields is
    volume x the base H = [[C, -e^T], [-e, -kappa]] (uniform fields, exact)."""
    for C, e, k in _materials():
        Cn, en, kn, _ = material.nondimensionalise(C, e, k)
        K = fem.element_matrix(Cn, en, kn, h)
        Z = fem.affine_loads(h)
        got = Z.T @ K @ Z
        want = np.prod(h) * material.base_H(Cn, en, kn)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_element_matrix_symmetric_and_kernel():
    C, e, k = cellgen.pzt5h_class()
    Cn, en, kn, _ = material.nondimensionalise(C, e, k)
    h = (0.5, 0.75, 1.25)
    K = fem.element_matrix(Cn, en, kn, h)
    assert np.abs(K - K.T).max() < 1e-15
    # translations, constant potential and infinitesimal rotations carry no energy
    x = fem.CORNERS * np.asarray(h)
    modes = []
    for comp in range(4):
        v = np.zeros(32)
        v[comp::4] = 1.0
        modes.append(v)
    for (i, j) in [(0, 1), (0, 2), (1, 2)]:
        v = np.zeros(32)
        v[i::4] = x[:, j]
        v[j::4] = -x[:, i]
        modes.append(v)
    for v in modes:
        assert np.abs(K @ v).max() < 1e-13
    # elastic block is positive semi-definite with exactly 6 zero modes,
    # dielectric block negative semi-definite with 1 zero mode
    uu = [4 * n + c for n in range(8) for c in range(3)]
    pp = [4 * n + 3 for n in range(8)]
    ev = np.linalg.eigvalsh(K[np.ix_(uu, uu)])
    assert (ev > -1e-13).all() and (np.abs(ev) < 1e-12).sum() == 6
    ev = np.linalg.eigvalsh(K[np.ix_(pp, pp)])
    assert (ev < 1e-13).all() and (np.abs(ev) < 1e-12).sum() == 1


def test_two_point_gauss_is_exact():
    C, e, k = cellgen.pzt5a()
    Cn, en, kn, _ = material.nondimensionalise(C, e, k)
    for h in [(1, 1, 1), (0.3, 0.7, 0.2)]:
        K2 = fem.element_matrix(Cn, en, kn, h)
        K5 = dense.element_matrix_brute(Cn, en, kn, h)
        np.testing.assert_allclose(K2, K5, rtol=0, atol=1e-14 * np.abs(K5).max())


def test_laplacian_block_against_textbook_q1():
    """With C = 0, e = 0, kappa = I the phi block is minus the textbook Q1
    Laplacian stiffness of the unit cube: diagonal 1/3, face neighbours 0,
    edge neighbours -1/12, body diagonal -1/12."""
    K = fem.element_matrix(np.zeros((6, 6)), np.zeros((3, 6)), np.eye(3), (1, 1, 1))
    L = -K[3::4, 3::4]
    for a in range(8):
        for b in range(8):
            d = int(np.abs(fem.CORNERS[a] - fem.CORNERS[b]).sum())
            want = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[d]
            assert abs(L[a, b] - want) < 1e-15


def test_unit_strain_loads():
    """Unit strains follow (d_ik d_jl + d_il d_jk)/2 of §2.2: the engineering
    shear of the shear loads is 1."""
    for p in range(6):
        E = fem.unit_strain(p)
        assert np.allclose(E, E.T)
        voigt = [E[0, 0], E[1, 1], E[2, 2], 2 * E[1, 2], 2 * E[0, 2], 2 * E[0, 1]]
        np.testing.assert_array_equal(voigt, np.eye(6)[p])


def test_smoothed_heaviside():
    eta = 0.125
    s = np.linspace(-3 * eta, 3 * eta, 2001)
    H = ersatz.smoothed_heaviside(s, eta)
    assert H[0] == 0.0 and H[-1] == 1.0
    assert abs(ersatz.smoothed_heaviside(np.array([0.0]), eta)[0] - 0.5) < 1e-15
    assert np.all(np.diff(H) >= -1e-15)
    # continuous at +-eta
    for edge in (-eta, eta):
        lo = ersatz.smoothed_heaviside(np.array([edge - 1e-12]), eta)[0]
        hi = ersatz.smoothed_heaviside(np.array([edge + 1e-12]), eta)[0]
        assert abs(lo - hi) < 1e-10
    # odd symmetry about (0, 1/2)
    np.testing.assert_allclose(H + H[::-1], 1.0, atol=1e-14)


def test_element_mean_is_centre_value_of_affine_field():
    n = 6
    i = np.arange(n)
    phi = (0.3 * i[None, None, :] + 0.2 * i[None, :, None] - 0.1 * i[:, None, None]).astype(float)
    m = ersatz.element_mean(phi)
    # interior elements (no periodic wrap): centre value of the affine field
    want = 0.3 * (i[:-1] + 0.5)[None, None, :] + 0.2 * (i[:-1] + 0.5)[None, :, None] \
        - 0.1 * (i[:-1] + 0.5)[:, None, None]
    np.testing.assert_allclose(m[:-1, :-1, :-1], want, atol=1e-14)


def test_rho_limits():
    phi = np.full((4, 4, 4), -1.0)
    assert np.all(ersatz.rho_from_levelset(phi) == 1.0)
    phi = np.full((4, 4, 4), 1.0)
    np.testing.assert_allclose(ersatz.rho_from_levelset(phi, rho_void=1e-3), 1e-3, rtol=1e-14)
