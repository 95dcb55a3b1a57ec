"""GPU parity of the preconditioner-block applies (§2.5.3: the elastic block A
and Sbar = sum_e rho_e S0) against the FP64 oracle, through cell_apply_block.

Three kernels: SIMT FP64 and FP32, and the node-centric tensor-core kernel
that the fine-level smoothers use (TF32 inputs, FP32 accumulation).
Tolerances: FP64 1e-12 and FP32 2e-6 relative to max|K| max|x| x 8 (as the
full-operator tests); TF32, component-wise: a TF32 input carries a relative
error below 2^-10 (truncation of 13 mantissa bits), a TF32-rounded matrix
entry below 2^-11, so every product term is within 2^-9 of its exact value
and |y - y_ref| <= 2^-9 (|A| |x|)_i + FP32 accumulation (2e-6 |A||x|).
Shapes are (nz, ny, nx); the tensor-core kernel tiles nodes 8 (x) by 16 (y)
inside CTAs of up to 32 x 16 nodes and a chunk of z planes, and masks ragged
edges: the shapes cover one tile (nx = 8), several tiles per CTA, several
CTAs along x, ragged x (nx = 7, 24, 40) and y (ny = 4, 17, 31), and several z
chunks.
"""
import numpy as np
import pytest
import torch

import cellgen
from oracle import fem, material, precond

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


def make_cell(rho):
    from paper_2410_03148_gb300 import Cell
    return Cell(torch.as_tensor(np.ascontiguousarray(rho), device=dev()), MAT, kind="rho")


def unit_K0(shape):
    Cn, en, kn, _ = material.nondimensionalise(*MAT)
    return fem.element_matrix(Cn, en, kn, fem.cell_h(shape))


def oracle_block(rho, block, x):
    """y = sum_e rho_e P_e^T Ke P_e x for x of shape (nrhs, nc, nz, ny, nx)."""
    shape = rho.shape
    nc = 3 if block == "A" else 1
    Ke = precond.block_matrix(unit_K0(shape), block)
    M = precond.assemble_block(rho, Ke, nc, shape)
    Mabs = abs(M)
    ys, bs = [], []
    for xr in x:
        v = np.moveaxis(xr, 0, -1).ravel()
        ys.append(np.moveaxis((M @ v).reshape(shape + (nc,)), -1, 0))
        bs.append(np.moveaxis((Mabs @ np.abs(v)).reshape(shape + (nc,)), -1, 0))
    return np.array(ys), np.array(bs), Ke


SHAPES = [(3, 4, 8), (5, 17, 16), (7, 31, 24), (40, 16, 32), (4, 8, 64), (3, 5, 7), (2, 18, 40)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("block", ["A", "Sbar"])
@pytest.mark.parametrize("kind", ["f64", "f32", "tc"])
def test_block_apply_matches_oracle(shape, block, kind):
    rho = cellgen.random_rho(shape, seed=11)
    cell = make_cell(rho)
    nc = 3 if block == "A" else 1
    nrhs = 9 if block == "Sbar" else 4   # Sbar: 3 groups of 4 loads, the last ragged
    rng = np.random.default_rng(12)
    x = rng.standard_normal((nrhs, nc) + shape)
    dt = torch.float64 if kind == "f64" else torch.float32
    xt = torch.as_tensor(x, device=dev(), dtype=dt)
    y = cell.apply_block(block, xt, tensor_cores=(kind == "tc")).double().cpu().numpy()
    yref, bound, Ke = oracle_block(rho, block, xt.double().cpu().numpy())
    err = np.abs(y - yref)
    if kind == "tc":
        assert np.all(err <= 2.0 ** -9 * bound + 2e-6 * bound.max()), (err / bound).max()
    else:
        tol = 1e-12 if kind == "f64" else 2e-6
        assert err.max() < tol * np.abs(Ke).max() * np.abs(x).max() * 8


@pytest.mark.parametrize("block", ["A", "Sbar"])
def test_block_apply_tc_is_reproducible(block):
    shape = (16, 16, 16)
    cell = make_cell(cellgen.random_rho(shape, seed=13))
    nc = 3 if block == "A" else 1
    x = torch.randn((9, nc) + shape, device=dev(), generator=torch.Generator(dev()).manual_seed(0))
    y1 = cell.apply_block(block, x, tensor_cores=True)
    y2 = cell.apply_block(block, x, tensor_cores=True)
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("block", ["A", "Sbar"])
def test_block_apply_tc_sampled_full_size(block, n):
    """64^3 and 128^3 (the benchmark grids, same launch configuration as the
    smoothers): sampled nodes on tile, CTA and z-chunk boundaries (multiples of
    8, 16 and 32 and their neighbours, both periodic ends) against the
    oracle's node-by-node element sum, for loads 0, 4 and 8."""
    shape = (n, n, n)
    rho = cellgen.random_rho(shape, seed=14)
    cell = make_cell(rho)
    nc = 3 if block == "A" else 1
    nrhs = 9
    rng = np.random.default_rng(15)
    x = rng.standard_normal((nrhs, nc) + shape).astype(np.float32)
    y = cell.apply_block(block, torch.as_tensor(x, device=dev()), tensor_cores=True).double().cpu().numpy()
    Ke = precond.block_matrix(unit_K0(shape), block)
    edges = sorted({c for m in (0, 8, 16, 32, n // 2, n - 32, n - 16, n - 8) for c in (m - 1, m, m + 1)
                    if 0 <= c < n} | {n - 1})
    xs, ys, zs = edges, edges[::2], edges[1::3]
    nodes = [(i, j, k) for i in xs for j in ys for k in zs]
    for r in (0, 4, 8):
        want = precond.block_rows(rho, Ke, nc, x[r].astype(np.float64), nodes)
        bound = precond.block_rows(rho, np.abs(Ke), nc, np.abs(x[r]).astype(np.float64), nodes)
        got = np.array([y[r, :, k, j, i] for (i, j, k) in nodes])
        err = np.abs(got - want)
        assert np.all(err <= 2.0 ** -9 * bound + 2e-6 * bound.max()), (err / bound).max()


@pytest.mark.parametrize("shape", [(20, 18, 40), (9, 33, 64), (5, 6, 7)])
def test_every_tensor_core_tile_gives_the_same_bits(shape):
    """The autotuner may pick any CTA tile (x width 8/16/32, z-chunk length):
    each one must give bitwise the result of the default tile, on ragged grids
    (partial x tiles, partial 16-row y tiles, chunks that do not divide nz) and
    for chunk lengths beyond nz.  Invalid tiles are rejected."""
    from paper_2410_03148_gb300._binding import CellError
    cell = make_cell(cellgen.random_rho(shape, seed=16))
    nz, ny, nx = shape
    xmax = 32 if nx >= 32 else (nx + 7) // 8 * 8
    g = torch.Generator(dev()).manual_seed(3)
    for block, nc in (("A", 3), ("Sbar", 1)):
        x = torch.randn((9, nc) + shape, device=dev(), generator=g)
        cell.set_tile(block, 0, 0)
        ref = cell.apply_block(block, x, tensor_cores=True)
        for xt in (8, 16, 32):
            if xt > xmax:
                continue
            for L in sorted({1, 2, 3, 4, 7, 16, nz, nz + 5}):
                cell.set_tile(block, xt, L)
                y = cell.apply_block(block, x, tensor_cores=True)
                assert torch.equal(y, ref), (block, xt, L)
    for bad in ((24, 4), (8, 0), (-8, 4), (64, 4)):
        with pytest.raises(CellError):
            cell.set_tile("A", *bad)
    if xmax < 32:
        with pytest.raises(CellError):
            cell.set_tile("Sbar", 32, 4)
