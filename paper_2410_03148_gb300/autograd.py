"""torch.autograd wrapper: design -> (C^H, e^H, kappa^H), backward by the
library's sensitivity kernels (the cell solutions are their own adjoint
states, because the energy form of the homogenised tensors is stationary in
the fluctuation fields).  The design is either the per-element ersatz scale
rho_e or the nodal level set phi (then the gradient is chained through the
§2.6 smoothing on the device)."""
from __future__ import annotations

import torch

from .cell import Cell


class HomogeniseFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, design, material, kind, options):
        cell = Cell(design.detach(), material, kind=kind, **(options or {}))
        cell.solve()
        Ch, eh, kh = cell.homogenise()
        ctx.cell = cell
        ctx.kind = kind
        ctx.dtype = design.dtype
        dev = design.device
        f = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
        return f(Ch), f(eh), f(kh)

    @staticmethod
    def backward(ctx, gC, ge, gk):
        to_np = lambda t: None if t is None else t.detach().double().cpu().numpy()
        sens = ctx.cell.sensitivity_phi if ctx.kind == "phi" else ctx.cell.sensitivity
        g = sens(to_np(gC), to_np(ge), to_np(gk), dtype=torch.float64)
        return g.to(ctx.dtype), None, None, None


def homogenise(design: torch.Tensor, material, kind: str = "rho", **options):
    """Differentiable homogenised tensors of a design (CUDA, (nz,ny,nx)):
    per-element rho (kind="rho") or nodal level set phi (kind="phi")."""
    return HomogeniseFn.apply(design, material, kind, options)
