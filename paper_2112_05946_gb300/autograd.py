"""torch.autograd.Function around the FR-SG run and its hand-written discrete adjoint.

FRSGRun.apply(u0, solver, dt, nsteps, checkpoint_every) advances u0 (device float64
[E, Np, M, S]) by nsteps SSP-RK3 steps in the CUDA library (fr_sg_forward_record) and
returns the final state; backward calls fr_sg_adjoint, which recomputes the run from its
checkpoints with the recorded filter decisions and applies the transposed stages.  Both
directions run in the library's kernels; torch only holds the buffers.

FRSGProject.apply(u0_nodal, solver) is the Galerkin projection of nodal initial values
(device float64 [E, Np, Q, S]) onto the gPC modes (fr_sg_project); its backward is the
transposed projection (fr_sg_project_transpose).  Composed with FRSGRun it gives gradients
of a QoI with respect to any parameter the initial data depend on (for instance the
magnitude of the uncertainty, sigma in u0 = f(x) + sigma z).

qoi_mean_var(solver, u) gives E[int u dx] and Var[int u dx] of a scalar state as torch
expressions (the gPC coefficients of the spatial integral are I_k = sum_e J sum_j w_j u_ejk;
orthonormal gPC: E = I_0, Var = sum_{k>=1} I_k^2).
"""
import torch


class FRSGRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver, dt, nsteps, checkpoint_every):
        u0c = u0.detach().contiguous()
        solver.set_state(u0c)
        solver.forward_record(dt, nsteps, checkpoint_every)
        out = torch.empty_like(u0c)
        solver.get_state(out)
        ctx.solver = solver
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = torch.empty_like(grad_out)
        ctx.solver.adjoint(grad_out.contiguous(), g)
        return g, None, None, None, None


class FRSGProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver):
        u0c = u0.detach().contiguous()
        out = torch.empty((solver.E, solver.Np, solver.M, solver.S), dtype=torch.float64, device=u0c.device)
        solver.project(u0c, out)
        ctx.solver = solver
        return out

    @staticmethod
    def backward(ctx, grad_out):
        s = ctx.solver
        g = torch.empty((s.E, s.Np, s.Q, s.S), dtype=torch.float64, device=grad_out.device)
        s.project_transpose(grad_out.contiguous(), g)
        return g, None


def quadrature_weights(solver):
    """J w_j: the solution-point weights of the library times the Jacobian dx/2 (1D)."""
    wx, _ = solver.quadrature()
    dx = (solver.cfg.x1 - solver.cfg.x0) / solver.cfg.nx
    return torch.tensor(0.5 * dx * wx, dtype=torch.float64, device="cuda")


def qoi_mean_var(Jw, u):
    I = torch.einsum("j,ejk->k", Jw, u[..., 0])
    return I[0], torch.sum(I[1:] ** 2)
