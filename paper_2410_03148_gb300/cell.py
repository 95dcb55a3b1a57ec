"""Pythonic handle over the C ABI (argument marshalling only).

``Cell`` owns one ``cell_handle``: a periodic unit-cell design (per-element
ersatz scale rho or nodal level set phi, a CUDA tensor of shape (nz, ny, nx))
with its material, and exposes the library calls on torch tensors.  All work
runs in libcell.so's kernels on the current torch CUDA stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B


def _stream_ptr(device):
    return torch.cuda.current_stream(device).cuda_stream


def _stats_dict(status, st):
    return {
        "status": status,
        "iters": list(st.iters),
        "refinements": st.refinements,
        "rel_residual": list(st.rel_residual),
        "solve_ms": st.solve_ms,
        "class_ms": dict(zip(B.PROF_CLASSES, list(st.class_ms))),
        "class_count": dict(zip(B.PROF_CLASSES, list(st.class_count))),
        "class_units": dict(zip(B.PROF_CLASSES, list(st.class_units))),
        "nlevels_u": st.nlevels_u,
        "nlevels_phi": st.nlevels_phi,
        "tc_tiles": [{"xt": st.tc_tile_xt[k], "L": st.tc_tile_L[k], "us": st.tc_tile_us[k]} for k in range(2)],
        "stencil_rg": [list(st.stencil_rg[k]) for k in range(2)],
    }


def solve_batch(cells, allow_notconv: bool = False):
    """Solve several handles at once (cell_solve_batch): cells built on
    different CUDA streams run concurrently.  Returns the stats of each."""
    _, sts = B.cell_solve_batch([c._h for c in cells], allow_notconv)
    out = []
    for c, st in zip(cells, sts):
        c.stats = _stats_dict(st.status, st)
        out.append(c.stats)
    return out


class Cell:
    def __init__(self, design: torch.Tensor, material, kind: str = "phi", rho_void: float = 1e-3,
                 eta: float = 0.0, **options):
        if not design.is_cuda:
            raise ValueError("design must be a CUDA tensor (the library has no CPU path)")
        if design.dim() != 3:
            raise ValueError("design must have shape (nz, ny, nx)")
        if design.dtype not in (torch.float32, torch.float64):
            raise ValueError("design dtype must be float32 or float64")
        B.load()
        self.device = design.device
        self.shape = tuple(design.shape)
        self.dtype = design.dtype
        nz, ny, nx = self.shape
        design = design.contiguous()
        Cm, em, km = material
        opt = B.cell_default_options(**options)
        kind_id = B.CELL_INPUT_PHI if kind == "phi" else B.CELL_INPUT_RHO
        dt = B.CELL_F32 if design.dtype == torch.float32 else B.CELL_F64
        with torch.cuda.device(self.device):
            self._desc = B.make_desc((nx, ny, nz), Cm, em, km, design.data_ptr(), kind_id, dt, opt,
                                     _stream_ptr(self.device), rho_void, eta)
            self._h = B.cell_setup(self._desc)
        self.nn = nx * ny * nz
        self.stats = None

    # -- hot path --------------------------------------------------------------
    def update(self, design: torch.Tensor):
        """Swap in a new design of the same shape/kind/dtype (no reallocation)."""
        if tuple(design.shape) != self.shape or not design.is_cuda or design.dtype != self.dtype:
            raise ValueError("design must be a CUDA tensor of the handle's shape and dtype")
        design = design.contiguous()
        B.cell_update(self._h, design.data_ptr())

    def solve(self, allow_notconv: bool = False):
        status, st = B.cell_solve(self._h, allow_notconv)
        self.stats = _stats_dict(status, st)
        return self.stats

    def homogenise(self):
        """(C^H [6x6] Pa, e^H [3x6] C/m^2, kappa^H [3x3] F/m) as numpy FP64."""
        return B.cell_homogenise(self._h)

    def sensitivity(self, dC=None, de=None, dk=None, dtype=torch.float64) -> torch.Tensor:
        g = torch.empty(self.shape, dtype=dtype, device=self.device)
        B.cell_sensitivity(self._h, dC, de, dk, g.data_ptr(),
                           B.CELL_F32 if dtype == torch.float32 else B.CELL_F64)
        return g

    def energy_difference(self, ref: "Cell", dC=None, de=None, dk=None) -> torch.Tensor:
        """Element-wise change sum_IJ G_IJ (W^I.K0 W^J - W_ref^I.K0 W_ref^J)
        between this handle's solution and ref's (FP64, polarisation form)."""
        g = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        B.cell_energy_difference(self._h, ref._h, dC, de, dk, g.data_ptr())
        return g

    def hilbert_velocity(self, dJ: torch.Tensor, dCs=(), Cs=(), alpha=None, wJ=1.0, wC=1.0):
        """Shape velocity of §2.6 (Hilbertian extension-regularisation and
        projection) from nodal sensitivities (FP64 CUDA tensors of the grid's
        shape); alpha defaults to 4 x the largest element size.  Returns
        (v, ||P g_J||_H, Chebyshev iterations, mu)."""
        if alpha is None:
            alpha = 4.0 / min(self.shape)
        ts = [dJ] + list(dCs)
        for t in ts:
            if not t.is_cuda or t.dtype != torch.float64 or tuple(t.shape) != self.shape:
                raise ValueError("sensitivities must be float64 CUDA tensors of the grid's shape")
        ts = [t.contiguous() for t in ts]
        v = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        nP, its, mu = B.cell_hilbert_velocity(self._h, alpha, ts[0].data_ptr(), [t.data_ptr() for t in ts[1:]],
                                              list(Cs), wJ, wC, v.data_ptr())
        return v, nP, its, mu

    def sensitivity_phi(self, dC=None, de=None, dk=None, dtype=torch.float64) -> torch.Tensor:
        """dL/dphi at the nodes (shape (nz, ny, nx)) for a level-set handle."""
        g = torch.empty(self.shape, dtype=dtype, device=self.device)
        B.cell_sensitivity_phi(self._h, dC, de, dk, g.data_ptr(),
                               B.CELL_F32 if dtype == torch.float32 else B.CELL_F64)
        return g

    # -- parity / inspection -----------------------------------------------------
    def apply(self, x: torch.Tensor) -> torch.Tensor:
        """y = Ahat x for x of shape (nrhs, 4, nz, ny, nx) (float32 or float64)."""
        x = x.contiguous()
        y = torch.empty_like(x)
        B.cell_apply(self._h, x.data_ptr(), y.data_ptr(), x.shape[0],
                     B.CELL_F32 if x.dtype == torch.float32 else B.CELL_F64)
        return y

    def apply_block(self, block: str, x: torch.Tensor, tensor_cores: bool = False) -> torch.Tensor:
        """y = A x (block "A", x of shape (nrhs, 3, nz, ny, nx)) or y = Sbar x
        (block "Sbar", shape (nrhs, 1, nz, ny, nx)): the preconditioner blocks."""
        x = x.contiguous()
        y = torch.empty_like(x)
        if tensor_cores:
            dt = B.CELL_F32_TC
        else:
            dt = B.CELL_F32 if x.dtype == torch.float32 else B.CELL_F64
        blk = B.CELL_BLOCK_A if block == "A" else B.CELL_BLOCK_SBAR
        B.cell_apply_block(self._h, blk, x.data_ptr(), y.data_ptr(), x.shape[0], dt)
        return y

    def set_tile(self, block: str, xt: int = 0, L: int = 0) -> None:
        """Fix the tensor-core smoother tile of block "A" or "Sbar" (xt nodes
        along x: 8, 16 or 32; L z-planes per chunk); 0, 0 = the default tile."""
        blk = B.CELL_BLOCK_A if block == "A" else B.CELL_BLOCK_SBAR
        B.cell_set_tile(self._h, blk, xt, L)

    def set_stencil_rg(self, block: str, level: int, rg: int = 0) -> None:
        """Fix the loads per thread (1, 3 or 9; 0 = default) of the coarse
        stencil apply on multigrid level `level` of block "A" or "Sbar"."""
        blk = B.CELL_BLOCK_A if block == "A" else B.CELL_BLOCK_SBAR
        B.cell_set_stencil_rg(self._h, blk, level, rg)

    def rhs(self) -> torch.Tensor:
        out = torch.empty((9, 4) + self.shape, dtype=torch.float64, device=self.device)
        B.cell_rhs(self._h, out.data_ptr())
        return out

    def solution(self) -> torch.Tensor:
        out = torch.empty((9, 4) + self.shape, dtype=torch.float64, device=self.device)
        B.cell_get_solution(self._h, out.data_ptr())
        return out

    def rho(self) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        B.cell_get_rho(self._h, out.data_ptr())
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            B.cell_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dh(C, e):
    """d_h and its gradients (host helper of the library)."""
    return B.cell_dh(C, e)


def hj_step(phi: torch.Tensor, v: torch.Tensor, dt: float) -> torch.Tensor:
    """One upwind step of phi_t + v |grad phi| = 0 (Eq. HJ) on the periodic
    node grid of shape (nz, ny, nx); phi and v CUDA tensors of one dtype."""
    if not (phi.is_cuda and v.is_cuda) or phi.shape != v.shape or phi.dtype != v.dtype or phi.dim() != 3:
        raise ValueError("phi and v must be CUDA tensors of one (nz, ny, nx) shape and dtype")
    phi, v = phi.contiguous(), v.contiguous()
    out = torch.empty_like(phi)
    B.cell_hj_step(phi.data_ptr(), v.data_ptr(), tuple(phi.shape), dt, out.data_ptr(),
                   B.CELL_F32 if phi.dtype == torch.float32 else B.CELL_F64,
                   torch.cuda.current_stream(phi.device).cuda_stream)
    return out


def figure(name, C, e=None):
    """(value, dC, de) of a §2.3 figure of merit: "d_h", "B_Voigt", "B_Reuss"
    or "C_zzzz" (host helper of the library)."""
    return B.cell_figure(name, C, e)
