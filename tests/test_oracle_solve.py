"""Pins of the oracle's assembled solve and homogenisation (no GPU)."""
import os

import numpy as np
import pytest

import cellgen
from oracle import dense, ersatz, fem, figures, laminate, material, sensitivity

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_pzt5a_hydrostatic_coefficient_matches_paper():
    g = _golden("pzt5a_dh.txt")
    C, e, _ = cellgen.pzt5a()
    assert abs(figures.d_h(C, e) * 1e12 - g["d_h_pC_per_N"]) < g["tolerance_pC_per_N"]


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 2)])
def test_solid_cell_returns_base_material(shape):
    C, e, k = cellgen.pzt5a()
    r = fem.solve_cell(np.ones(shape), C, e, k)
    assert _rel(r["C"], C) < 1e-13
    assert _rel(r["e"], e) < 1e-13
    assert _rel(r["kappa"], k) < 1e-13
    assert abs(figures.d_h(r["C"], r["e"]) - figures.d_h(C, e)) < 1e-13 * abs(figures.d_h(C, e))


def test_uniform_scaling():
    C, e, k = cellgen.pzt5h_class()
    r = fem.solve_cell(np.full((4, 4, 4), 0.37), C, e, k)
    assert _rel(r["C"], 0.37 * C) < 1e-13
    assert _rel(r["e"], 0.37 * e) < 1e-13
    assert _rel(r["kappa"], 0.37 * k) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 5, 4)])
def test_laminate_matches_closed_form(axis, shape):
    C, e, k = cellgen.pzt5h_class()
    rho = cellgen.laminate_rho(shape, axis, seed=11 + axis)
    layers = {0: rho[0, 0, :], 1: rho[0, :, 0], 2: rho[:, 0, 0]}[axis]
    r = fem.solve_cell(rho, C, e, k)
    Ch, eh, kh, _ = laminate.laminate_tensors(C, e, k, layers, axis)
    assert _rel(r["C"], Ch) < 1e-11
    assert np.abs(r["e"] - eh).max() < 1e-11 * np.abs(e).max()
    assert _rel(r["kappa"], kh) < 1e-11


def test_laminate_closed_form_limits():
    """Equal layers give the scaled base material; the closed form's two
    readings of e^H agree (reciprocity)."""
    C, e, k = cellgen.pzt5a()
    Ch, eh, kh, LH = laminate.laminate_tensors(C, e, k, [0.4] * 5, 2)
    assert _rel(Ch, 0.4 * C) < 1e-14 and _rel(kh, 0.4 * k) < 1e-14
    assert np.abs(eh - 0.4 * e).max() < 1e-14 * np.abs(e).max()
    Ch, eh, kh, LH = laminate.laminate_tensors(C, e, k, [1.0, 1e-3, 0.2], 0)
    assert np.abs(-LH[:6, 6:].T - eh).max() < 1e-12 * np.abs(e).max()


@pytest.fixture(scope="module")
def random_cell():
    C, e, k = cellgen.pzt5h_class()
    rho = cellgen.random_rho((4, 4, 4), seed=5)
    return rho, C, e, k, fem.solve_cell(rho, C, e, k)


def test_energy_form_symmetric_and_matches_linear_form(random_cell):
    *_, r = random_cell
    H, Hl = r["H"], r["H_lin"]
    assert np.abs(H - H.T).max() < 1e-14 * np.abs(H).max()
    assert np.abs(H - Hl).max() < 1e-12 * np.abs(H).max()
    e1, e2 = fem.e_from_strain_and_field(H)
    assert np.abs(e1 - e2).max() < 1e-13 * np.abs(H).max()


def test_homogenised_tensors_positive_definite(random_cell):
    *_, r = random_cell
    assert np.linalg.eigvalsh(r["C"]).min() > 0
    assert np.linalg.eigvalsh(r["kappa"]).min() > 0


def test_dense_elimination_equals_sparse_direct(random_cell):
    *_, r = random_cell
    P = r["problem"]
    yd = dense.solve_dense(P)
    assert np.abs(yd - r["y"]).max() < 1e-11 * np.abs(r["y"]).max()


def test_pin_choice_and_projection_do_not_change_H(random_cell):
    *_, r = random_cell
    P = r["problem"]
    y7 = P.solve(pin_node=37, project=False)
    H7, _ = P.homogenise(y7)
    assert np.abs(H7 - r["H"]).max() < 1e-12 * np.abs(r["H"]).max()


def test_residual_of_solution_vanishes(random_cell):
    *_, r = random_cell
    P = r["problem"]
    res = P.Kg @ r["y"] - P.rhs()
    assert np.abs(res).max() < 1e-12 * np.abs(P.rhs()).max()
    # the right-hand sides are orthogonal to the null space
    b = P.rhs()
    for comp in range(4):
        assert np.abs(b[comp::4].sum(axis=0)).max() < 1e-14 * np.abs(b).max() * b.shape[0]


def test_si_and_nondimensional_assemblies_agree():
    """The nondimensionalisation of §2.2 is an exact change of variables."""
    C, e, k = cellgen.pzt5a()
    rho = cellgen.random_rho((4, 3, 4), seed=2)
    a = fem.solve_cell(rho, C, e, k, nondim=True)
    b = fem.solve_cell(rho, C, e, k, nondim=False)
    assert _rel(a["C"], b["C"]) < 1e-8
    assert np.abs(a["e"] - b["e"]).max() < 1e-8 * np.abs(e).max()
    assert _rel(a["kappa"], b["kappa"]) < 1e-8


def test_cyclic_shift_invariance():
    """Translating the design within the cell leaves the tensors unchanged (§2.6)."""
    C, e, k = cellgen.pzt5h_class()
    rho = cellgen.random_rho((4, 4, 4), seed=9)
    a = fem.solve_cell(rho, C, e, k)["H"]
    for ax, s in [(0, 1), (1, 3), (2, 2)]:
        b = fem.solve_cell(np.roll(rho, s, axis=ax), C, e, k)["H"]
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_xy_swap_permutes_tensors():
    """Swapping x and y (a symmetry of the z-poled base material) permutes the
    Voigt indices 11<->22, 23<->13 and the field indices 1<->2."""
    C, e, k = cellgen.pzt5h_class()
    rho = cellgen.random_rho((4, 4, 4), seed=4)
    a = fem.solve_cell(rho, C, e, k)
    b = fem.solve_cell(np.ascontiguousarray(np.swapaxes(rho, 1, 2)), C, e, k)
    P6 = [1, 0, 2, 4, 3, 5]
    P3 = [1, 0, 2]
    assert _rel(b["C"], a["C"][np.ix_(P6, P6)]) < 1e-12
    assert np.abs(b["e"] - a["e"][np.ix_(P3, P6)]).max() < 1e-12 * np.abs(e).max()
    assert _rel(b["kappa"], a["kappa"][np.ix_(P3, P3)]) < 1e-12


def test_gaussian_levelset_design_is_half_solid():
    phi = cellgen.gaussian_levelset(16, seed=0)
    rho = ersatz.rho_from_levelset(phi)
    assert 0.35 < rho.mean() < 0.65
    assert rho.min() >= 1e-3 - 1e-15 and rho.max() <= 1.0
