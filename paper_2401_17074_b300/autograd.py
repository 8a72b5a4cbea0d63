"""torch.autograd interface to the TSLB adjoint.

``final_moments(F, solver, state, nsteps)`` runs ``nsteps`` TSLB steps from
``state`` with the per-node acceleration field ``F`` ([3, N] float32 on the
solver's device, full lattice) and returns the final moments (rho [N],
u [3, N], Pi^neq [6, N]) as CUDA float64 tensors.  Any torch objective built
from them back-propagates: the backward pass hands the objective's cotangent
of the final moments to the library's discrete adjoint (``tslb_adjoint``:
checkpointed forward recomputation, transposed step kernels), which returns
dJ/dF.

``kinetic_energy(F, solver, state, nsteps)`` is the special case
J = 1/2 sum rho |u|^2 with the energy reduced in FP64 on the GPU and its
seed built on the device (``tslb_adjoint_force_gradient``).

The solver must be created with ``checkpoint_every > 0``, on a periodic box or
a channel with bounce-back y walls.
"""
import torch

from . import DEVICE, tslb_adjoint, tslb_adjoint_force_gradient, tslb_get_moments


def _run(F, solver, state, nsteps):
    if not F.is_cuda or F.dtype != torch.float32:
        raise TypeError("F must be a CUDA float32 tensor of shape [3, N]")
    solver.init_moments(*state)
    solver.set_force_field(F.detach().contiguous().view(-1))
    solver.step(nsteps)


class FinalMoments(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, solver, state, nsteps):
        _run(F, solver, state, nsteps)
        N = solver.N
        rho = torch.empty(N, dtype=torch.float64, device=F.device)
        u = torch.empty(3 * N, dtype=torch.float64, device=F.device)
        pi = torch.empty(6 * N, dtype=torch.float64, device=F.device)
        tslb_get_moments(solver.handle, rho, u, pi, DEVICE)
        ctx.solver = solver
        ctx.nsteps = int(nsteps)
        ctx.shape = F.shape
        return rho, u.view(3, N), pi.view(6, N)

    @staticmethod
    def backward(ctx, g_rho, g_u, g_pi):
        N = ctx.solver.N
        lam = torch.zeros(10 * N, dtype=torch.float64, device=(g_rho if g_rho is not None else
                                                                 g_u if g_u is not None else g_pi).device)
        if g_rho is not None:
            lam[:N] = g_rho.reshape(-1)
        if g_u is not None:
            lam[N:4 * N] = g_u.reshape(-1)
        if g_pi is not None:
            lam[4 * N:] = g_pi.reshape(-1)
        g = torch.empty(ctx.shape, dtype=torch.float32, device=lam.device)
        tslb_adjoint(ctx.solver.handle, lam, ctx.nsteps, 0, g, DEVICE)
        return g, None, None, None


def final_moments(F, solver, state, nsteps):
    """(rho, u, Pi^neq) after nsteps from state under the force field F; differentiable with respect to F."""
    return FinalMoments.apply(F, solver, state, nsteps)


class KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, solver, state, nsteps):
        _run(F, solver, state, nsteps)
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
