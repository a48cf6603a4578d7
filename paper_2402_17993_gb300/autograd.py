"""torch.autograd.Function over the library's energy + adjoint gradient.

Forward calls the C ABI once (energy and the full gradient from one
reverse sweep, Section 2.3 energy of the Trotterised ansatz of Eq. 5);
backward scales the stored gradient by the incoming dE.
"""
from __future__ import annotations

import torch


class UCCSDEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, uccsd_ctx):
        if not theta.is_cuda or theta.dtype != torch.float64:
            raise TypeError("theta must be a CUDA float64 tensor")
        th = theta.detach().contiguous()
        batched = th.dim() == 2
        th2 = th if batched else th.unsqueeze(0)
        B = th2.shape[0]
        E = torch.empty(B, dtype=torch.float64, device=th.device)
        g = torch.empty_like(th2)
        uccsd_ctx.energy_grad_device(th2, E, g)
        ctx.save_for_backward(g)
        ctx.batched = batched
        return E if batched else E[0]

    @staticmethod
    def backward(ctx, dE):
        (g,) = ctx.saved_tensors
        if ctx.batched:
            return dE.unsqueeze(1) * g, None
        return dE * g[0], None


def uccsd_energy(theta, uccsd_ctx):
    """Differentiable Trotterised UCCSD energy of a CUDA float64 theta."""
    return UCCSDEnergy.apply(theta, uccsd_ctx)
