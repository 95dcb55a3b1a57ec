"""Pins of the oracle's Hilbertian extension-regularisation and projection
(oracle/hilbert.py, §2.6 reading): Q1 element matrices against their 1D
tensor-product construction, the periodic Helmholtz operator against the
exact eigenvalues of Fourier modes, and the projection's defining identities
(H-orthogonality to the constraint representers, the prescribed first-order
constraint change, descent of the objective)."""
import numpy as np
import pytest

from oracle import hilbert


def kron3(ax, ay, az):
    # local node n = a + 2b + 4c: x fastest, so the z factor is the outermost
    return np.kron(az, np.kron(ay, ax))


@pytest.mark.parametrize("h", [(0.25, 0.25, 0.25), (0.2, 0.125, 0.5)])
def test_element_matrices_are_q1_tensor_products(h):
    K, M = hilbert.element_matrices(h)
    m = [hd / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]]) for hd in h]
    s = [np.array([[1.0, -1.0], [-1.0, 1.0]]) / hd for hd in h]
    assert np.allclose(M, kron3(m[0], m[1], m[2]), rtol=0, atol=1e-15)
    Kt = kron3(s[0], m[1], m[2]) + kron3(m[0], s[1], m[2]) + kron3(m[0], m[1], s[2])
    assert np.allclose(K, Kt, rtol=0, atol=1e-14)
    assert abs(M.sum() - h[0] * h[1] * h[2]) < 1e-16
    assert np.abs(K @ np.ones(8)).max() < 1e-14


@pytest.mark.parametrize("kvec", [(0, 0, 0), (1, 0, 0), (2, 1, 0), (1, 2, 3), (3, 2, 2)])
def test_helmholtz_operator_fourier_modes(kvec):
    shape = (6, 5, 8)            # (nz, ny, nx), anisotropic spacing
    alpha = 0.3
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    arg = 2 * np.pi * (kvec[0] * x + kvec[1] * y + kvec[2] * z)
    A = hilbert.helmholtz_matrix(shape, alpha)
    lam = hilbert.symbol(shape, alpha, kvec)
    for mode in (np.cos(arg), np.sin(arg)):
        assert np.abs(A @ mode.ravel() - lam * mode.ravel()).max() < 1e-13 * max(lam, 1e-300) * 10
        if np.abs(mode).max() > 0.5:
            g = hilbert.riesz(shape, alpha, lam * mode)
            assert np.abs(g - mode).max() < 1e-11


def test_constant_mode_and_total_mass():
    shape = (4, 6, 5)
    A = hilbert.helmholtz_matrix(shape, 1.7)
    one = np.ones(np.prod(shape))
    assert np.abs(A @ one - one / np.prod(shape)).max() < 1e-15   # K 1 = 0, sum of M rows = node volume
    assert abs(hilbert.symbol(shape, 1.7, (0, 0, 0)) * np.prod(shape) - 1.0) < 1e-14


def test_velocity_without_constraints_is_normalised_representer():
    shape = (4, 5, 6)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(shape)
    v, (nP, mu, R) = hilbert.velocity(shape, 0.2, d, wJ=2.0)
    g = hilbert.riesz(shape, 0.2, d)
    assert abs(nP - np.sqrt(hilbert.h_inner(shape, 0.2, g, g))) < 1e-12 * nP
    assert np.abs(v - 2.0 * g / nP).max() < 1e-12 * np.abs(v).max()


def test_velocity_of_a_fourier_mode():
    shape = (8, 8, 8)
    alpha = 0.25
    z, y, x = np.meshgrid(*(np.arange(8) / 8,) * 3, indexing="ij")
    mode = np.cos(2 * np.pi * (x + 2 * y))
    lam = hilbert.symbol(shape, alpha, (1, 2, 0))
    v, (nP, _, _) = hilbert.velocity(shape, alpha, lam * mode)
    # ||mode||_H^2 = mode^T A mode = lam |mode|^2
    assert abs(nP - np.sqrt(lam * (mode ** 2).sum())) < 1e-12 * nP
    assert np.abs(v - mode / nP).max() < 1e-10


def test_projection_identities_with_constraints():
    shape = (5, 6, 4)
    alpha = 0.15
    rng = np.random.default_rng(7)
    dJ = rng.standard_normal(shape)
    dCs = [rng.standard_normal(shape), np.ones(shape) + 0.3 * rng.standard_normal(shape)]
    Cs = [0.2, -0.05]
    gJ = hilbert.riesz(shape, alpha, dJ)
    gs = [hilbert.riesz(shape, alpha, dc) for dc in dCs]
    ip = lambda u, v: hilbert.h_inner(shape, alpha, u, v)
    # objective part alone: H-orthogonal to every constraint representer, and a descent direction
    v0, (nP, _, _) = hilbert.velocity(shape, alpha, dJ, dCs, Cs, wJ=1.0, wC=0.0)
    for g in gs:
        assert abs(ip(g, v0)) < 1e-10 * np.sqrt(ip(g, g) * ip(v0, v0))
    assert abs(ip(gJ, v0) - nP) < 1e-10 * nP and nP > 0
    # constraint part: first-order change <g_i, v>_H = w_C C_i
    v, _ = hilbert.velocity(shape, alpha, dJ, dCs, Cs, wJ=1.0, wC=0.7)
    for g, c in zip(gs, Cs):
        assert abs(ip(g, v) - 0.7 * c) < 1e-10 * (1 + abs(c))
    # in the span of the constraints the objective part vanishes
    _, (nP2, _, _) = hilbert.velocity(shape, alpha, 2.0 * dCs[0] - dCs[1], dCs, Cs)
    assert nP2 < 1e-8 * np.sqrt(ip(gJ, gJ))
