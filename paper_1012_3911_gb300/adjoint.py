"""torch.autograd interface of the adjoint gradient in libsop.

``overlap_objective(prop, psi0, phi, field, V, dt, every)`` returns
J = |<phi|psi_N>|^2 for the Schroedinger split steps of the propagator
``prop`` and lets ``J.backward()`` fill the gradients of the field samples
(float64, n_steps x ndim, CPU) and of the potential (float64 CUDA tensor with
the lattice shape).  All arithmetic runs in ``sop_adjoint_gradient`` (one
forward sweep with checkpoints, one backward sweep of costates); this module
only marshals tensors.
"""
from __future__ import annotations

import torch


class OverlapObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, field, V, prop, psi0, phi, dt, every):
        if V.dtype != torch.float64 or not V.is_cuda:
            raise ValueError("V must be a float64 CUDA tensor")
        prop.set_potential(V.detach().contiguous())
        prop.state.copy_(psi0)
        gV = torch.empty(V.shape, dtype=torch.float64, device=V.device)
        J, gE = prop.adjoint_gradient(phi, int(field.shape[0]), float(dt), field.detach().cpu().numpy(),
                                      int(every), gV)
        ctx.save_for_backward(torch.from_numpy(gE).to(field.dtype), gV)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        gE, gV = ctx.saved_tensors
        g = float(gJ)
        return g * gE, g * gV, None, None, None, None, None


def overlap_objective(prop, psi0, phi, field, V, dt: float, every: int = 20):
    """J = |<phi|psi_N>|^2 with adjoint gradients for ``field`` and ``V``."""
    return OverlapObjective.apply(field, V, prop, psi0, phi, dt, every)
