"""torch.autograd.Function for the compliance J(rho) = f^T u(rho).

Forward: set the densities, solve K(rho) u = f (Eq. (2)), return J.
Backward: compliance is self-adjoint, so no second solve is needed:
dJ/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e (Eq. (3)), computed by
the library's sensitivity kernel from the stored u and scaled by grad_out.
All arithmetic runs in libtopo.so; this file only moves tensors.
"""
from __future__ import annotations

import torch

from . import topo


class Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho: torch.Tensor, mesh: "topo.Mesh", opts=None):
        if rho.dtype != torch.float32 or not rho.is_cuda:
            raise TypeError("rho must be a float32 CUDA tensor")
        rho_c = rho.detach().contiguous()
        mesh.set_stream(torch.cuda.current_stream())  # order against torch's work
        mesh.set_density(rho_c)
        mesh.solve(opts)
        c = mesh.compliance()
        ctx.mesh = mesh
        ctx.n = rho_c.numel()
        ctx.device = rho.device
        return torch.tensor(c, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        dc = torch.empty(ctx.n, dtype=torch.float64, device=ctx.device)
        ctx.mesh.set_stream(torch.cuda.current_stream())
        ctx.mesh.sensitivity(dc)  # ordered before later work on the current stream
        g = (grad_out.to(torch.float64) * dc).to(torch.float32)
        return g, None, None


def compliance(rho: torch.Tensor, mesh: "topo.Mesh", opts=None) -> torch.Tensor:
    """J(rho) with a gradient: `compliance(rho, mesh).backward()` fills rho.grad."""
    return Compliance.apply(rho, mesh, opts)
