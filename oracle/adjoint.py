"""Oracle: gradients of mean / variance QoIs of the 1D scalar FR-SG run w.r.t. the initial
gPC coefficients (the discrete adjoint the GPU library implements by hand).

TEST INFRASTRUCTURE ONLY.  The forward step of oracle.scheme / oracle.capture /
oracle.integrate is written out once more with plain PyTorch CPU float64 ops, with
the filter decisions of every stage frozen (taken from a recorded run of the numpy
oracle), and differentiated by reverse-mode autograd.  The local Lax-Friedrichs
dissipation max(|u_L|, |u_R|) is differentiated along the branch the forward run takes.

QoIs (orthonormal gPC, §2.1 Eq. 3): with I_k = sum_e J sum_j w_j uhat_{e,j,k} the k-th gPC
coefficient of the spatial integral of u,  E[int u dx] = I_0  and  Var[int u dx] =
sum_{k>=1} I_k^2.
"""
import numpy as np
import torch

from . import tables


def _tabs_torch(prob):
    t = tables.fr_tables(prob.P)
    g = tables.gpc_tables(prob.N, prob.Q)
    T = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)   # noqa: E731
    return dict(D=T(t["D"]), lm=T(t["lm"]), lp=T(t["lp"]), dhL=T(t["dhL"]), dhR=T(t["dhR"]), w=T(t["w"]),
                Vx=T(t["Vx"]), Vxinv=T(t["Vx_inv"]), V=T(g["V"]), Pz=T(g["Pz"]))


def _flux(prob, u):
    return prob.adv_speed * u if prob.equation == "advection" else 0.5 * u * u


def _speed(prob, u):
    if prob.equation == "advection":
        return abs(prob.adv_speed) * torch.ones_like(u)
    return torch.abs(u)


def rhs_torch(prob, tt, u):
    """Transcription of oracle.scheme.rhs_1d for periodic scalar problems (same step order)."""
    J = 0.5 * prob.dx
    un = torch.einsum("qk,ejk->ejq", tt["V"], u)
    fhat = torch.einsum("kq,ejq->ejk", tt["Pz"], _flux(prob, un)) / J
    uL = torch.einsum("j,ejk->ek", tt["lm"], u)
    uR = torch.einsum("j,ejk->ek", tt["lp"], u)
    fDL = torch.einsum("j,ejk->ek", tt["lm"], fhat)
    fDR = torch.einsum("j,ejk->ek", tt["lp"], fhat)
    left = torch.roll(uR, 1, dims=0)     # face e-1/2: left state from element e-1
    right = uL
    a = torch.einsum("qk,ek->eq", tt["V"], left)
    b = torch.einsum("qk,ek->eq", tt["V"], right)
    alpha = torch.maximum(_speed(prob, a), _speed(prob, b))
    fI_n = 0.5 * (_flux(prob, a) + _flux(prob, b)) - 0.5 * alpha * (b - a)
    fI = torch.einsum("kq,eq->ek", tt["Pz"], fI_n) / J      # flux on the left face of element e
    fIL = fI
    fIR = torch.roll(fI, -1, dims=0)
    dfdr = (torch.einsum("jm,emk->ejk", tt["D"], fhat) + (fIL - fDL)[:, None, :] * tt["dhL"][None, :, None]
            + (fIR - fDR)[:, None, :] * tt["dhR"][None, :, None])
    return -dfdr


def _filter_torch(prob, tt, u, dt, flags):
    if prob.filter == "none":
        return u
    from .capture import filter_strengths
    lam = torch.as_tensor(filter_strengths(prob, dt), dtype=torch.float64)   # [m, k]
    ut = torch.einsum("mj,ejk->emk", tt["Vxinv"], u)
    filt = torch.einsum("jm,emk->ejk", tt["Vx"], ut * lam[None])
    mask = torch.as_tensor(np.asarray(flags, dtype=bool))[:, None, None]
    return torch.where(mask, filt, u)


def step_torch(prob, tt, u, dt, flags3):
    """One SSP-RK3 step (no limiter: scalar problems) with frozen filter decisions."""
    u0 = u
    u1 = _filter_torch(prob, tt, u0 + dt * rhs_torch(prob, tt, u0), dt, flags3[0])
    u2 = _filter_torch(prob, tt, 0.75 * u0 + 0.25 * (u1 + dt * rhs_torch(prob, tt, u1)), dt, flags3[1])
    return _filter_torch(prob, tt, (1.0 / 3.0) * u0 + (2.0 / 3.0) * (u2 + dt * rhs_torch(prob, tt, u2)), dt,
                         flags3[2])


def qoi_torch(prob, tt, u):
    """(E[int u dx], Var[int u dx]) of the scalar state u [E, Np, M]."""
    I = 0.5 * prob.dx * torch.einsum("j,ejk->k", tt["w"], u)
    return I[0], torch.sum(I[1:] ** 2)


def gradients(prob, uhat0, dt, nsteps, flags):
    """d E[int u(T)] / d uhat(0) and d Var[int u(T)] / d uhat(0) by reverse mode through the
    nsteps-step run; flags: [3 * nsteps][E] filter decisions of the forward run."""
    assert prob.dim == 1 and prob.S == 1 and prob.bc[0] == "periodic"
    tt = _tabs_torch(prob)
    u0 = torch.tensor(np.asarray(uhat0)[..., 0], dtype=torch.float64, requires_grad=True)
    u = u0
    for n in range(nsteps):
        u = step_torch(prob, tt, u, dt, flags[3 * n:3 * n + 3])
    mean, var = qoi_torch(prob, tt, u)
    gm, = torch.autograd.grad(mean, u0, retain_graph=True)
    gv, = torch.autograd.grad(var, u0)
    c = np.ascontiguousarray
    return dict(state=c(u.detach().numpy()[..., None]), mean=float(mean.detach()), var=float(var.detach()),
                grad_mean=c(gm.numpy()[..., None]), grad_var=c(gv.numpy()[..., None]))


def qoi_seeds(prob, uhat):
    """lambda_T = d QoI / d uhat(T) for both QoIs, numpy [E, Np, M, 1]."""
    w = tables.fr_tables(prob.P)["w"]
    J = 0.5 * prob.dx
    I = J * np.einsum("j,ejk->k", w, uhat[..., 0])
    gm = np.zeros(uhat.shape)
    gm[:, :, 0, 0] = J * w[None, :]
    gv = np.zeros(uhat.shape)
    gv[:, :, 1:, 0] = 2.0 * J * w[None, :, None] * I[None, None, 1:]
    return gm, gv
