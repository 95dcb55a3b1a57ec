"""Host arithmetic of bench.py (no GPU): the oracle baseline's power-law fit
and extrapolation, and the roofline class costs in the units the metric
names."""
import math

import bench


def test_oracle_fit_recovers_an_exact_power_law():
    """t = c * dof^p sampled exactly at three sizes: the least-squares fit in
    log space returns p and extrapolates to c * dof_target^p (ms)."""
    c, p = 3.0e-9, 1.8
    pts = [(n, c * (4 * n ** 3) ** p) for n in (8, 12, 16)]
    ms, p_fit = bench.oracle_fit(pts, 128)
    assert abs(p_fit - p) < 1e-12
    assert math.isclose(ms, 1e3 * c * (4 * 128 ** 3) ** p, rel_tol=1e-10)


def test_oracle_fit_with_one_size_scales_linearly():
    """With one size only there is no exponent to fit: linear in the dof count."""
    ms, p_fit = bench.oracle_fit([(8, 2.0), (8, 2.0)], 16)
    assert p_fit == 1.0
    assert math.isclose(ms, 2.0e3 * 8, rel_tol=1e-12)


def test_apply_roofline_bytes_per_dof_rhs():
    """FP32 operator apply: read x and write y (4 + 4 bytes per dof and load)
    plus rho amortised over 4 dof x 9 loads."""
    assert math.isclose(bench.APPLY_BYTES_PER_DOF_RHS, 8 + 4 / 36, rel_tol=1e-15)
    flops, nbytes, bound, dtype, dof = bench.CLASS_COST["full32"]
    assert flops == 2 * (1024 + 32) and dof == 4 and dtype == "f32"
    # elastic smoother: 3 dof per node, 18 floats per node-load plus rho and dinv shares
    flops, nbytes, bound, dtype, dof = bench.CLASS_COST["elastic0"]
    assert dof == 3 and math.isclose(nbytes, 4 * 18 + 4 * 3 / 9 + 4 / 9, rel_tol=1e-15)
