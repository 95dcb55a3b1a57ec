"""Pins of the oracle's Hamilton-Jacobi step (Eq. HJ) against exact
solutions (no GPU).

A signed-distance slab phi = |x - 1/2| - 1/4 has |grad phi| = 1 away from its
two ridges (x = 1/2 and the periodic wrap), so phi_t + v|grad phi| = 0 moves
it exactly to phi - v t there, and one-sided differences of the linear
pieces are exact: the upwind step must reproduce phi - v dt to rounding at
every node two or more cells from a ridge, for either sign of v and along
each axis.
"""
import numpy as np
import pytest

from oracle import levelset


def _slab(n, axis, shape3):
    x = np.arange(n) / n
    prof = np.abs(x - 0.5) - 0.25
    shape = [1, 1, 1]
    shape[axis] = n
    return np.broadcast_to(prof.reshape(shape), shape3).copy(), x


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("v", [0.7, -0.4])
def test_slab_moves_exactly(axis, v):
    shape3 = [6, 7, 8]
    shape3[axis] = 32
    phi, x = _slab(32, axis, tuple(shape3))
    dt = 0.2 / 32
    out = levelset.hj_step(phi, np.full(phi.shape, v), dt)
    far = (np.abs(x - 0.5) >= 2.0 / 32) & (np.minimum(x, 1 - x) >= 2.0 / 32)
    sel = [slice(None)] * 3
    sel[axis] = far
    np.testing.assert_allclose(out[tuple(sel)], (phi - v * dt)[tuple(sel)], atol=1e-14)


def test_zero_velocity_is_identity_and_axes_commute():
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((5, 6, 7))
    assert np.array_equal(levelset.hj_step(phi, np.zeros_like(phi), 0.01), phi)
    # the grid spacing follows the axis, so the transposition check uses a cube
    phi_c, v_c = rng.standard_normal((6, 6, 6)), rng.standard_normal((6, 6, 6))
    a = levelset.hj_step(phi_c, v_c, 0.003)
    b = levelset.hj_step(phi_c.transpose(2, 1, 0), v_c.transpose(2, 1, 0), 0.003).transpose(2, 1, 0)
    np.testing.assert_allclose(a, b, atol=1e-15)
