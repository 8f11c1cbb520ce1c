"""torch.autograd.Function over the library's energy/force call.

Forward returns the total energy E (Eq. 4) as a float64 scalar tensor; the
backward pass returns dE/dpos = -F with F the library's analytic force
(Eq. 5), so gradients of anything built on E flow through the GPU adjoint.
"""
import torch

from . import apip as _apip


class EnergyForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, model, box, types, ids):
        n = pos.shape[0]
        force = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        e = torch.zeros(1, dtype=torch.float64, device=pos.device)
        model.energy_forces(pos.detach().contiguous(), box, types, ids, force, e_total_out=e)
        model.sync()
        ctx.save_for_backward(force)
        return e[0]

    @staticmethod
    def backward(ctx, grad_out):
        (force,) = ctx.saved_tensors
        return -force * grad_out, None, None, None, None


def energy(pos, model, box, types, ids):
    """E(pos) with autograd support (dE/dpos = -F)."""
    return EnergyForces.apply(pos, model, box, types, ids)
