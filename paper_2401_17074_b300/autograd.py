"""torch.autograd interface to the TSLB adjoint.

``kinetic_energy(F, solver, state, nsteps)`` runs ``nsteps`` TSLB steps from
``state`` with the per-node acceleration field ``F`` ([3, N] float32 on the
solver's device, full lattice) and returns J = 1/2 sum rho |u|^2 of the final
moments (FP64 reduction on the GPU).  Its backward pass calls the library's
discrete adjoint (checkpointed forward recomputation, transposed step
kernels), so ``J.backward()`` fills ``F.grad`` with dJ/dF.  The solver must be
created with ``checkpoint_every > 0`` on a periodic box.
"""
import torch

from . import DEVICE, tslb_adjoint_force_gradient


class KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, solver, state, nsteps):
        if not F.is_cuda or F.dtype != torch.float32:
            raise TypeError("F must be a CUDA float32 tensor of shape [3, N]")
        solver.init_moments(*state)
        solver.set_force_field(F.detach().contiguous().view(-1))
        solver.step(nsteps)
        d, code = solver.diagnostics()
        ctx.solver = solver
        ctx.nsteps = int(nsteps)
        ctx.shape = F.shape
        return torch.tensor(d["kinetic_energy"], dtype=torch.float64, device=F.device)

    @staticmethod
    def backward(ctx, gJ):
        g = torch.empty(ctx.shape, dtype=torch.float32, device=gJ.device)
        tslb_adjoint_force_gradient(ctx.solver.handle, ctx.nsteps, g, DEVICE)
        return (gJ.to(torch.float32) * g), None, None, None


def kinetic_energy(F, solver, state, nsteps):
    """J(F) = 1/2 sum rho |u|^2 after nsteps; differentiable with respect to F."""
    return KineticEnergy.apply(F, solver, state, nsteps)
