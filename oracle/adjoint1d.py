"""Oracle: reverse-mode derivatives of a general 1D FR-SG run (scalar or Euler; LLF or HLL;
any boundary kind; exponential, L2 or no filter with frozen decisions; the positivity
limiter differentiated through its scalings beta_1 and beta_2).

TEST INFRASTRUCTURE ONLY.  The forward stage of oracle.scheme.rhs_1d, oracle.capture.limit
and oracle.integrate.ssp_rk3_step is written out once more with plain PyTorch CPU float64
operations and differentiated by autograd.  Discrete choices are taken from the forward
values: the LLF dissipation max(lambda_L, lambda_R) and the HLL branch follow the branch the
values select; the limiter's trigger, its minimum point and the points whose pressure root
enters beta_2 follow the forward run (the minimum is differentiated at its argument); the
filter decisions are frozen (passed in).
"""
import numpy as np
import torch

from . import capture, tables


def _T(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64)


def tabs_torch(prob):
    t = tables.fr_tables(prob.P)
    g = tables.gpc_tables(prob.N, prob.Q)
    return dict(D=_T(t["D"]), lm=_T(t["lm"]), lp=_T(t["lp"]), dhL=_T(t["dhL"]), dhR=_T(t["dhR"]), w=_T(t["w"]),
                Vx=_T(t["Vx"]), Vxinv=_T(t["Vx_inv"]), V=_T(g["V"]), Pz=_T(g["Pz"]))


# ---------------------------------------------------------------- pointwise physics (§3.2, §5.3)

def pressure(prob, u):
    return (prob.gamma - 1.0) * (u[..., 2] - 0.5 * u[..., 1] ** 2 / u[..., 0])


def flux(prob, u):
    if prob.equation == "advection":
        return prob.adv_speed * u
    if prob.equation == "burgers":
        return 0.5 * u * u
    p = pressure(prob, u)
    v = u[..., 1] / u[..., 0]
    return torch.stack([u[..., 1], u[..., 1] * v + p, (u[..., 2] + p) * v], dim=-1)


def _speeds(prob, u):
    """(smallest, largest) characteristic speed and spectral radius at every point."""
    if prob.equation == "advection":
        a = prob.adv_speed * torch.ones_like(u[..., 0])
        return a, a, torch.abs(a)
    if prob.equation == "burgers":
        return u[..., 0], u[..., 0], torch.abs(u[..., 0])
    c = torch.sqrt(prob.gamma * pressure(prob, u) / u[..., 0])
    v = u[..., 1] / u[..., 0]
    return v - c, v + c, torch.abs(v) + c


def interface_flux(prob, uL, uR):
    fL, fR = flux(prob, uL), flux(prob, uR)
    loL, hiL, lamL = _speeds(prob, uL)
    loR, hiR, lamR = _speeds(prob, uR)
    if prob.flux == "hll":
        SL = torch.minimum(loL, loR)[..., None]
        SR = torch.maximum(hiL, hiR)[..., None]
        den = torch.where(SR - SL != 0, SR - SL, torch.ones_like(SR))
        mid = (SR * fL - SL * fR + SL * SR * (uR - uL)) / den
        return torch.where(SL >= 0, fL, torch.where(SR <= 0, fR, mid))
    alpha = torch.maximum(lamL, lamR)[..., None]
    return 0.5 * (fL + fR) - 0.5 * alpha * (uR - uL)


def ghost(prob, side, interior):
    kind = prob.bc[side]
    if kind == "dirichlet":
        return _T(prob.dirichlet[side]).expand_as(interior)
    if kind == "outflow":
        return interior
    if kind == "reflect":
        if prob.equation == "euler":
            sign = _T([1.0, -1.0, 1.0])
            return interior * sign
        return -interior
    raise ValueError(kind)


# ---------------------------------------------------------------- residual (§3.1-3.4)

def rhs(prob, tt, u):
    """Transcription of oracle.scheme.rhs_1d (same step order)."""
    E = u.shape[0]
    J = 0.5 * prob.dx
    un = torch.einsum("qk,ejks->ejqs", tt["V"], u)
    fhat = torch.einsum("kq,ejqs->ejks", tt["Pz"], flux(prob, un)) / J
    uL = torch.einsum("j,ejks->eks", tt["lm"], u)
    uR = torch.einsum("j,ejks->eks", tt["lp"], u)
    fDL = torch.einsum("j,ejks->eks", tt["lm"], fhat)
    fDR = torch.einsum("j,ejks->eks", tt["lp"], fhat)
    if prob.bc[0] == "periodic":
        left = torch.cat([uR[E - 1:E], uR[0:E - 1], uR[E - 1:E]], dim=0)
        right = torch.cat([uL[0:1], uL[1:E], uL[0:1]], dim=0)
    else:
        left = torch.cat([ghost(prob, 0, uL[0:1]), uR[0:E - 1], uR[E - 1:E]], dim=0)
        right = torch.cat([uL[0:1], uL[1:E], ghost(prob, 1, uR[E - 1:E])], dim=0)
    fI_n = interface_flux(prob, torch.einsum("qk,fks->fqs", tt["V"], left), torch.einsum("qk,fks->fqs", tt["V"], right))
    fI = torch.einsum("kq,fqs->fks", tt["Pz"], fI_n) / J
    fIL, fIR = fI[0:E], fI[1:E + 1]
    dfdr = (torch.einsum("jm,emks->ejks", tt["D"], fhat)
            + (fIL - fDL)[:, None] * tt["dhL"][None, :, None, None]
            + (fIR - fDR)[:, None] * tt["dhR"][None, :, None, None])
    return -dfdr


# ---------------------------------------------------------------- limiter (§4.3)

def _pressure_root(prob, ubar, us, eps):
    """Smallest root in [0, 1] of p(ubar + beta (us - ubar)) = eps (the quadratic of
    oracle.capture.pressure_root), as a differentiable expression; us [..., 3]."""
    g1 = prob.gamma - 1.0
    d = us - ubar
    a = g1 * (d[..., 2] * d[..., 0] - 0.5 * d[..., 1] ** 2)
    b = g1 * (ubar[..., 2] * d[..., 0] + ubar[..., 0] * d[..., 2] - ubar[..., 1] * d[..., 1]) - eps * d[..., 0]
    c = g1 * (ubar[..., 2] * ubar[..., 0] - 0.5 * ubar[..., 1] ** 2) - eps * ubar[..., 0]
    disc = torch.clamp(b * b - 4.0 * a * c, min=0.0)
    sq = torch.sqrt(disc)
    # the roots as q/a and c/q, q = -(b + sign(b) sqrt(disc))/2: no cancellation when a is small
    q = -0.5 * (b + torch.copysign(sq, b))
    r1 = q / a
    r2 = torch.where(q != 0.0, c / q, r1)
    lin = -c / b
    in1 = (r1 >= 0.0) & (r1 <= 1.0)
    in2 = (r2 >= 0.0) & (r2 <= 1.0)
    quad = torch.where(in1 & in2, torch.minimum(r1, r2), torch.where(in1, r1, r2))
    return torch.where(torch.abs(a) < 1e-300, lin, quad)


def limit(prob, tt, u):
    """Transcription of oracle.capture.limit for 1D Euler with the scalings differentiable."""
    if prob.equation != "euler" or not prob.limiter:
        return u
    Lp = torch.cat([torch.eye(prob.n1, dtype=torch.float64), tt["lm"][None], tt["lp"][None]], dim=0)
    pts = torch.einsum("lj,qk,ejks->elqs", Lp, tt["V"], u)
    ubar = torch.einsum("j,ejs->es", tt["w"] / 2.0, u[:, :, 0, :])
    out = []
    for e in range(u.shape[0]):
        rb = ubar[e, 0]
        pb = pressure(prob, ubar[e])
        if not (float(rb.detach()) > 0.0 and float(pb.detach()) > 0.0):
            raise FloatingPointError(f"element {e}: mean state not admissible")
        eps = min(1e-8, float(rb.detach()), float(pb.detach()))
        ue = pts[e].reshape(-1, 3)
        rho = ue[:, 0]
        p = pressure(prob, ue)
        rmin = torch.min(rho)
        if not (min(float(rmin.detach()), float(torch.min(p).detach())) < eps):
            out.append(u[e])
            continue
        beta1 = torch.ones((), dtype=torch.float64)
        if float((rb - rmin).detach()) > 0.0:
            b1 = (rb - eps) / (rb - rmin)
            beta1 = b1 if float(b1.detach()) < 1.0 else beta1
        us = torch.cat([(beta1 * (rho - rb) + rb)[:, None], ue[:, 1:]], dim=1)
        ps = pressure(prob, us)
        low = ps < eps
        beta2 = torch.ones((), dtype=torch.float64)
        if bool(torch.any(low)):
            roots = _pressure_root(prob, ubar[e][None, :], us[low], eps)
            rmin2 = torch.min(roots)
            beta2 = rmin2 if float(rmin2.detach()) < 1.0 else beta2
        scale = torch.stack([beta2 * beta1, beta2, beta2])
        onehot = torch.zeros(u.shape[2], dtype=torch.float64)
        onehot[0] = 1.0
        mean_part = onehot[None, :, None] * ubar[e][None, None, :]          # ubar in mode 0 at every point
        out.append(mean_part + scale[None, None, :] * (u[e] - mean_part))
    return torch.stack(out, dim=0)


# ---------------------------------------------------------------- filter (frozen decisions) and step

def _filter(prob, tt, u, dt, flags):
    if prob.filter == "none":
        return u
    lam = _T(capture.filter_strengths(prob, dt))            # [m, k]
    ut = torch.einsum("mj,ejks->emks", tt["Vxinv"], u)
    filt = torch.einsum("jm,emks->ejks", tt["Vx"], ut * lam[None, :, :, None])
    mask = torch.as_tensor(np.asarray(flags, dtype=bool))[:, None, None, None]
    return torch.where(mask, filt, u)


def step(prob, tt, u, dt, flags3):
    """One SSP-RK3 step (oracle.integrate.ssp_rk3_step) with frozen filter decisions."""
    u0 = limit(prob, tt, u)
    u1 = _filter(prob, tt, u0 + dt * rhs(prob, tt, u0), dt, flags3[0])
    v1 = limit(prob, tt, u1)
    u2 = _filter(prob, tt, 0.75 * u0 + 0.25 * (v1 + dt * rhs(prob, tt, v1)), dt, flags3[1])
    v2 = limit(prob, tt, u2)
    return _filter(prob, tt, (1.0 / 3.0) * u0 + (2.0 / 3.0) * (v2 + dt * rhs(prob, tt, v2)), dt, flags3[2])


def vjp(prob, uhat0, dts, flags, lam_T):
    """Final state of the run and lambda_0 = (d u_T / d u_0)^T lam_T for the step sizes
    dts (one per step) and the forward run's filter decisions flags [3 * nsteps][E]."""
    assert prob.dim == 1 and prob.filter != "lasso"
    tt = tabs_torch(prob)
    u0 = torch.tensor(np.asarray(uhat0), dtype=torch.float64, requires_grad=True)
    u = u0
    for n, dt in enumerate(dts):
        u = step(prob, tt, u, dt, flags[3 * n:3 * n + 3])
    (g,) = torch.autograd.grad(u, u0, grad_outputs=torch.as_tensor(np.asarray(lam_T), dtype=torch.float64))
    return np.ascontiguousarray(u.detach().numpy()), np.ascontiguousarray(g.numpy())
