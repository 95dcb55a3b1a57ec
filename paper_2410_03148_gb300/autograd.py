"""torch.autograd wrapper: rho_e -> (C^H, e^H, kappa^H), backward by the
library's sensitivity kernel (the cell solutions are their own adjoint states,
because the energy form of the homogenised tensors is stationary in the
fluctuation fields)."""
from __future__ import annotations

import torch

from .cell import Cell


class HomogeniseFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, material, options):
        cell = Cell(rho.detach(), material, kind="rho", **(options or {}))
        cell.solve()
        Ch, eh, kh = cell.homogenise()
        ctx.cell = cell
        ctx.rho_dtype = rho.dtype
        dev = rho.device
        f = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
        return f(Ch), f(eh), f(kh)

    @staticmethod
    def backward(ctx, gC, ge, gk):
        to_np = lambda t: None if t is None else t.detach().double().cpu().numpy()
        g = ctx.cell.sensitivity(to_np(gC), to_np(ge), to_np(gk), dtype=torch.float64)
        return g.to(ctx.rho_dtype), None, None


def homogenise(rho: torch.Tensor, material, **options):
    """Differentiable homogenised tensors of a per-element design rho (CUDA, (nz,ny,nx))."""
    return HomogeniseFn.apply(rho, material, options)
