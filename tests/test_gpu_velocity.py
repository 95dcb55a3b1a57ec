"""GPU parity of the shape-velocity and energy-difference entry points.

* cell_hilbert_velocity (Hilbertian extension-regularisation and projection,
  §2.6) against oracle.hilbert.velocity, which uses a sparse direct solve and
  explicit Gram-Schmidt (the library: Chebyshev iteration and Gram-matrix
  coefficients): FP64, agreement to 1e-10 relative.
* cell_energy_difference (polarisation form of the difference of two
  designs' weighted element energies) against the difference of the
  oracle's element energies (8^3) and of the library's own per-element
  sensitivities (16^3).
"""
import numpy as np
import pytest
import torch

import cellgen
from oracle import ersatz, fem, hilbert, sensitivity

pytestmark = pytest.mark.gpu

MAT = cellgen.pzt5h_class()


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_03148_gb300 import load
    return load()


def dev():
    return torch.device("cuda:0")


def make_cell(design, kind, **opt):
    from paper_2410_03148_gb300 import Cell
    return Cell(torch.as_tensor(np.ascontiguousarray(design), device=dev()), MAT, kind=kind, **opt)


@pytest.mark.parametrize("shape", [(6, 8, 10), (16, 16, 16), (5, 3, 2)])
@pytest.mark.parametrize("ncons", [0, 1, 3])
def test_hilbert_velocity_matches_oracle(shape, ncons):
    rng = np.random.default_rng(41 + ncons)
    cell = make_cell(cellgen.random_rho(shape, seed=2), "rho")
    dJ = rng.standard_normal(shape)
    dCs = [np.ones(shape) + 0.2 * rng.standard_normal(shape) for _ in range(ncons)]
    Cs = list(rng.standard_normal(ncons) * 0.1)
    alpha = 4.0 / min(shape)
    t = lambda a: torch.as_tensor(a, device=dev(), dtype=torch.float64)
    v, nP, its, mu = cell.hilbert_velocity(t(dJ), [t(d) for d in dCs], Cs, alpha=alpha, wJ=1.3, wC=0.6)
    vref, (nPr, mur, _) = hilbert.velocity(shape, alpha, dJ, dCs, Cs, wJ=1.3, wC=0.6)
    v = v.cpu().numpy()
    assert np.abs(v - vref).max() < 1e-10 * np.abs(vref).max(), (its, np.abs(v - vref).max())
    assert abs(nP - nPr) < 1e-10 * nPr
    assert np.allclose(mu, mur, rtol=1e-9, atol=1e-12 * np.abs(mur).max(initial=1.0))


def test_hilbert_velocity_rejects_dependent_constraints():
    from paper_2410_03148_gb300._binding import CellError
    shape = (8, 8, 8)
    cell = make_cell(cellgen.random_rho(shape, seed=2), "rho")
    d = torch.randn(shape, dtype=torch.float64, device=dev())
    with pytest.raises(CellError):
        cell.hilbert_velocity(d, [d, 2.0 * d], [0.1, 0.2])


def test_energy_difference_matches_oracle_8cube():
    shape = (8, 8, 8)
    rho1 = cellgen.random_rho(shape, seed=5, lo=0.05)
    rho2 = rho1.copy()
    rho2[3, 4, 5] *= 1.5
    rng = np.random.default_rng(9)
    dC, de, dk = rng.standard_normal((6, 6)), rng.standard_normal((3, 6)), rng.standard_normal((3, 3))
    cells = [make_cell(r, "rho", precision=0, tol=1e-12) for r in (rho1, rho2)]
    for c in cells:
        c.solve()
    got = cells[0].energy_difference(cells[1], dC, de, dk).cpu().numpy()
    ref = []
    for r in (rho1, rho2):
        P = fem.CellProblem(r, *MAT)
        ref.append(sensitivity.grad_rho(P, P.solve(), sensitivity.G_from_si(dC, de, dk, P.sc)))
    want = ref[0] - ref[1]
    assert np.abs(got - want).max() < 1e-8 * np.abs(ref[0]).max()


def test_energy_difference_equals_difference_of_element_energies_16cube():
    phi = cellgen.gaussian_levelset(16, seed=3)
    a = make_cell(phi, "phi", precision=0, tol=1e-12)
    b = make_cell(phi + 0.01 * np.sin(np.arange(phi.size)).reshape(phi.shape), "phi", precision=0, tol=1e-12)
    de = np.zeros((3, 6)); de[2, :3] = 1.0
    for c in (a, b):
        c.solve()
    got = a.energy_difference(b, None, de, None).cpu().numpy()
    want = a.sensitivity(None, de, None).cpu().numpy() - b.sensitivity(None, de, None).cpu().numpy()
    assert np.abs(got - want).max() < 1e-11 * np.abs(a.sensitivity(None, de, None).cpu().numpy()).max()
    assert np.abs(b.energy_difference(a, None, de, None).cpu().numpy() + got).max() < 1e-13 * np.abs(got).max()
