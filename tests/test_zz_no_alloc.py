"""The allocation-free homogenisation entry point, through the C ABI.

cell_homogenise_noalloc serves callers that cannot allocate device memory
when they need the tensors (a framework whose caching allocator owns the
device-memory budget, or a loop that must not stall on cudaMalloc): it takes
the fields from the caller and keeps its partial sums in a fixed device array
inside the library.  Two calls in a row must both agree
with cell_homogenise on the same solved design.  This file is collected
last, so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest
import torch

import cellgen

MAT = cellgen.pzt5h_class()


@pytest.mark.gpu
def test_noalloc_homogenise_matches_handle_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_03148_gb300 import Cell
    from paper_2410_03148_gb300 import _binding as B
    dev = torch.device("cuda:0")
    phi = torch.as_tensor(cellgen.gaussian_levelset(16, seed=6), device=dev)
    cell = Cell(phi, MAT, kind="phi")
    cell.solve()
    ref = cell.homogenise()
    rho = cell.rho()
    b = cell.rhs()
    y = cell.solution()
    r = b - cell.apply(y)
    torch.cuda.synchronize()
    desc = B.make_desc((16, 16, 16), *MAT, 0, B.CELL_INPUT_RHO, B.CELL_F64,
                       stream=torch.cuda.current_stream(dev).cuda_stream)
    outs = [B.cell_homogenise_noalloc(desc, rho.data_ptr(), b.data_ptr(), y.data_ptr(), r.data_ptr())
            for _ in range(2)]
    for got in outs:
        for a, want in zip(got, ref):
            assert np.abs(a - want).max() <= 1e-8 * np.abs(want).max()
    for a, b2 in zip(*outs):
        assert np.array_equal(a, b2)
    cell.close()


@pytest.mark.gpu
def test_noalloc_rejects_oversized_grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_03148_gb300 import _binding as B
    desc = B.make_desc((256, 256, 128), *MAT, 0, B.CELL_INPUT_RHO, B.CELL_F64)
    with pytest.raises(B.CellError) as ei:
        B.cell_homogenise_noalloc(desc, 16, 16, 16, 16)
    assert ei.value.status == B.CELL_EINVAL
