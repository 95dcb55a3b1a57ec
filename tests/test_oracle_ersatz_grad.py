"""Pins of the oracle's level-set chain rule (§2.6 ersatz map) against finite
differences (no GPU)."""
import numpy as np

import cellgen
from oracle import ersatz, fem, sensitivity


def test_heaviside_derivative_matches_differences_and_integrates_to_one():
    eta = 0.3
    s = np.linspace(-0.5, 0.5, 201)
    h = 1e-7
    fd = (ersatz.smoothed_heaviside(s + h, eta) - ersatz.smoothed_heaviside(s - h, eta)) / (2 * h)
    d = ersatz.smoothed_heaviside_deriv(s, eta)
    inside = np.abs(np.abs(s) - eta) > 2 * h
    np.testing.assert_allclose(d[inside], fd[inside], atol=1e-6)
    xs = np.linspace(-eta, eta, 20001)
    assert abs(np.trapezoid(ersatz.smoothed_heaviside_deriv(xs, eta), xs) - 1.0) < 1e-8


def test_grad_phi_of_a_linear_functional_matches_differences():
    """L = sum_e w_e rho_e(phi): dL/drho = w exactly, so grad_phi(phi, w) must
    equal the central differences of L in every nodal value."""
    shape = (3, 4, 5)
    phi = cellgen.gaussian_levelset(shape, seed=2) * 0.2   # many elements inside the band
    w = np.random.default_rng(0).standard_normal(shape)
    g = ersatz.grad_phi(phi, w)
    L = lambda p: float((w * ersatz.rho_from_levelset(p)).sum())
    h = 1e-7
    for n in range(phi.size):
        pp, pm = phi.copy().ravel(), phi.copy().ravel()
        pp[n] += h
        pm[n] -= h
        fd = (L(pp.reshape(shape)) - L(pm.reshape(shape))) / (2 * h)
        assert abs(fd - g.ravel()[n]) < 1e-6 * np.abs(g).max() + 1e-8


def test_grad_phi_of_homogenised_objective_matches_differences():
    """Full chain with direct solves at 4^3: L = sum G_IJ H_IJ(rho(phi))."""
    shape = (4, 4, 4)
    C, e, k = cellgen.pzt5h_class()
    phi = cellgen.gaussian_levelset(shape, seed=5) * 0.3
    rng = np.random.default_rng(3)
    G = rng.standard_normal((9, 9))
    G = G + G.T

    def L(p):
        P = fem.CellProblem(ersatz.rho_from_levelset(p), C, e, k)
        H, _ = P.homogenise(P.solve())
        return float((G * H).sum())

    rho = ersatz.rho_from_levelset(phi)
    P = fem.CellProblem(rho, C, e, k)
    g_rho = sensitivity.grad_rho(P, P.solve(), G)
    g = ersatz.grad_phi(phi, g_rho)
    nodes = np.argsort(-np.abs(g.ravel()))[:4]
    h = 1e-6
    for n in nodes:
        pp, pm = phi.copy().ravel(), phi.copy().ravel()
        pp[n] += h
        pm[n] -= h
        fd = (L(pp.reshape(shape)) - L(pm.reshape(shape))) / (2 * h)
        assert abs(fd - g.ravel()[n]) < 1e-5 * abs(g.ravel()[n]) + 1e-9 * np.abs(g).max()
