"""Pins of the oracle's sensitivities against finite differences (no GPU)."""
import numpy as np

import cellgen
from oracle import fem, figures, material, sensitivity


def test_element_sensitivity_matches_central_differences():
    C, e, k = cellgen.pzt5h_class()
    rho = cellgen.random_rho((4, 4, 4), seed=21, lo=0.05)
    rng = np.random.default_rng(0)
    G = rng.standard_normal((9, 9))
    G = G + G.T
    P = fem.CellProblem(rho, C, e, k)
    y = P.solve()
    g = sensitivity.grad_rho(P, y, G).ravel()
    idx = [0, 17, 42, 63]
    fd = sensitivity.fd_grad(rho, C, e, k, G, idx, step=1e-6)
    np.testing.assert_allclose(g[idx], fd, rtol=1e-5, atol=1e-9 * np.abs(g).max())


def test_sensitivities_sum_to_linear_H():
    """H is homogeneous of degree one in rho (scaling every rho_e by t scales
    H by t), so Euler's theorem gives sum_e rho_e dH/drho_e = H."""
    C, e, k = cellgen.pzt5a()
    rho = cellgen.random_rho((4, 4, 4), seed=8)
    P = fem.CellProblem(rho, C, e, k)
    y = P.solve()
    Q = sensitivity.element_quadforms(P, y)
    H, _ = P.homogenise(y)
    np.testing.assert_allclose(np.einsum("e,eIJ->IJ", rho.ravel(), Q), H,
                               atol=1e-13 * np.abs(H).max())


def test_dh_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    C, e, _ = cellgen.pzt5h_class()
    A = rng.standard_normal((6, 6))
    C = C + 0.05 * np.abs(C).max() * (A + A.T) / 6.0
    assert np.linalg.eigvalsh(C).min() > 0
    e = e + rng.standard_normal((3, 6))
    dC, de = figures.d_h_grad(C, e)
    f0 = figures.d_h(C, e)
    for (i, j) in [(0, 0), (2, 2), (0, 2), (3, 3), (5, 1)]:
        s = 1e-6 * np.abs(C).max()
        Cp, Cm = C.copy(), C.copy()
        Cp[i, j] += s
        Cm[i, j] -= s
        fd = (figures.d_h(Cp, e) - figures.d_h(Cm, e)) / (2 * s)
        assert abs(fd - dC[i, j]) < 1e-6 * abs(f0) / np.abs(C).max() + 1e-6 * abs(dC[i, j])
    for (i, j) in [(2, 0), (2, 2), (0, 4), (1, 3)]:
        s = 1e-4
        ep, em = e.copy(), e.copy()
        ep[i, j] += s
        em[i, j] -= s
        fd = (figures.d_h(C, ep) - figures.d_h(C, em)) / (2 * s)
        assert abs(fd - de[i, j]) < 1e-8 * abs(f0) + 1e-8


def test_dh_gradient_nonsymmetric_C():
    """Every Voigt entry is an independent variable: the gradient must also
    hold for a nonsymmetric C (dS = -S dC S gives -(S^T e_3)(S m)^T)."""
    C = _perturbed_C(11)
    C[1, 4] += 3e9
    e = cellgen.pzt5h_class()[1]
    dC, _ = figures.d_h_grad(C, e)
    f0 = figures.d_h(C, e)
    s = 1e-6 * np.abs(C).max()
    for i in range(6):
        for j in range(6):
            Cp, Cm = C.copy(), C.copy()
            Cp[i, j] += s
            Cm[i, j] -= s
            fd = (figures.d_h(Cp, e) - figures.d_h(Cm, e)) / (2 * s)
            assert abs(fd - dC[i, j]) < 1e-6 * abs(f0) / np.abs(C).max() + 1e-6 * abs(dC[i, j])


def test_G_from_si_reproduces_chain_rule():
    """sum G_IJ H_IJ equals sum dC.C^H + de.e^H + dk.kappa^H for a symmetric H."""
    rng = np.random.default_rng(1)
    H = rng.standard_normal((9, 9))
    H = H + H.T
    sc = (1.3e11, 2.0e-8)
    dC, de, dk = rng.standard_normal((6, 6)), rng.standard_normal((3, 6)), rng.standard_normal((3, 3))
    G = sensitivity.G_from_si(dC, de, dk, sc)
    Ch, eh, kh = material.redimensionalise(*fem.split_H(H), sc)
    want = (dC * Ch).sum() + (de * eh).sum() + (dk * kh).sum()
    assert abs((G * H).sum() - want) < 1e-12 * abs(want) + 1e-9


def test_bulk_moduli_of_isotropic_material():
    """B_Voigt = B_Reuss = lambda + 2 mu / 3 for an isotropic stiffness."""
    lam, mu = 3.0, 2.0
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2 * mu
    C[np.arange(3, 6), np.arange(3, 6)] = mu
    assert abs(figures.b_voigt(C) - (lam + 2 * mu / 3)) < 1e-14
    assert abs(figures.b_reuss(C) - (lam + 2 * mu / 3)) < 1e-13


def _perturbed_C(seed):
    rng = np.random.default_rng(seed)
    C, _, _ = cellgen.pzt5h_class()
    A = rng.standard_normal((6, 6))
    C = C + 0.05 * np.abs(C).max() * (A + A.T) / 6.0
    assert np.linalg.eigvalsh(C).min() > 0
    return C


def test_reuss_below_voigt():
    """Hill's bounds: B_Reuss <= B_Voigt for any positive-definite stiffness."""
    for seed in range(5):
        C = _perturbed_C(seed)
        assert figures.b_reuss(C) <= figures.b_voigt(C)


def test_bulk_and_czzzz_gradients_match_finite_differences():
    C = _perturbed_C(7)
    C[0, 1] += 1e9   # an asymmetric C: every entry is an independent variable
    for f, grad in ((figures.b_voigt, figures.b_voigt_grad), (figures.b_reuss, figures.b_reuss_grad),
                    (figures.c_zzzz, figures.c_zzzz_grad)):
        g = grad(C)
        f0 = f(C)
        s = 1e-6 * np.abs(C).max()
        for i in range(6):
            for j in range(6):
                Cp, Cm = C.copy(), C.copy()
                Cp[i, j] += s
                Cm[i, j] -= s
                fd = (f(Cp) - f(Cm)) / (2 * s)
                assert abs(fd - g[i, j]) < 1e-6 * abs(f0) / np.abs(C).max() + 1e-7 * abs(g[i, j])
