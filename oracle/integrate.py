"""Oracle: initial projection, time step, SSP-RK3 stages with limiter and filter, moments.

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy.

Stage order (§4.3, Eq. 53, stated there for forward Euler and applied here to each
forward-Euler stage of the three-stage strong-stability-preserving Runge-Kutta scheme):
limit the stage input, take the Euler update with the residual of the limited state,
form the SSP convex combination, then run the detector and filter the flagged elements.
"""
import numpy as np

from . import capture, scheme, tables


def project_initial(prob, u0):
    """uhat_k(0, x_j) = <u0(x_j, .) Phi_k> by the random-space quadrature (§2.1, Eq. 6,
    third line, with Eq. 5).  u0(x, z) (1D) or u0(x, y, z) (2D) returns [..., S]."""
    g = tables.gpc_tables(prob.N, prob.Q)
    if prob.dim == 1:
        X = prob.nodes()
        vals = np.stack([np.asarray(u0(X, zq), dtype=np.float64).reshape(prob.E, prob.Np, prob.S)
                         for zq in g["z"]], axis=2)
    else:
        X, Y = prob.nodes()
        vals = np.stack([np.asarray(u0(X, Y, zq), dtype=np.float64).reshape(prob.E, prob.Np, prob.S)
                         for zq in g["z"]], axis=2)
    return np.einsum("kq,ejqs->ejks", g["Pz"], vals)


def max_speed(prob, tabs, uhat):
    """Largest spectral radius over the solution points and z-nodes (both directions in 2D)."""
    u = np.einsum("qk,ejks->ejqs", tabs["z_V"], uhat)
    lam = scheme.wave_speed(prob, u, 0)
    if prob.dim == 2:
        lam = np.maximum(lam, scheme.wave_speed(prob, u, 1))
    return float(np.max(lam))


def cfl_dt(prob, tabs, uhat, cfl):
    """dt = CFL * h / lambda_max with h the smallest element width (the setup tables of §5
    give the CFL number only)."""
    h = prob.dx if prob.dim == 1 else min(prob.dx, prob.dy)
    return cfl * h / max_speed(prob, tabs, uhat)


def _finish_stage(prob, tabs, u, dt, record, replay, stage):
    if replay is not None:
        flags = np.asarray(replay[stage], dtype=bool)
    else:
        flags = capture.filter_decisions(prob, tabs, u)
    if record is not None:
        record.append(flags.copy())
    return capture.apply_filter(prob, tabs, u, dt, flags)


def ssp_rk3_step(prob, tabs, uhat, dt, record=None, replay=None, stage_offset=0):
    """One step of the three-stage SSP Runge-Kutta scheme (Shu-Osher form):
        u1 = F(u0),  u2 = 3/4 u0 + 1/4 F(u1),  u^{n+1} = 1/3 u0 + 2/3 F(u2),
    F(v) = lim(v) + dt L(lim(v)) the forward-Euler step of Eq. 53, u0 = lim(u^n), and
    the detector + filter applied after each combination.  `record` collects the filter
    flags of each stage; `replay` supplies them instead of the detector."""
    L = scheme.rhs
    u0 = capture.limit(prob, tabs, uhat)
    u1 = u0 + dt * L(prob, tabs, u0)
    u1 = _finish_stage(prob, tabs, u1, dt, record, replay, stage_offset + 0)
    v1 = capture.limit(prob, tabs, u1)
    u2 = 0.75 * u0 + 0.25 * (v1 + dt * L(prob, tabs, v1))
    u2 = _finish_stage(prob, tabs, u2, dt, record, replay, stage_offset + 1)
    v2 = capture.limit(prob, tabs, u2)
    u3 = (1.0 / 3.0) * u0 + (2.0 / 3.0) * (v2 + dt * L(prob, tabs, v2))
    u3 = _finish_stage(prob, tabs, u3, dt, record, replay, stage_offset + 2)
    return u3


def rk4_step(prob, tabs, uhat, dt, record=None, replay=None, stage_offset=0):
    """One step of the classical four-stage Runge-Kutta scheme (the integrator of the
    advection study, §5.1 setup table):
        y1 = u0 + dt/2 L(u0),  y2 = u0 + dt/2 L(y1),  y3 = u0 + dt L(y2),
        u^{n+1} = u0 + dt/6 (L(u0) + 2 L(y1) + 2 L(y2) + L(y3)),
    with u0 = lim(u^n).  Each stage is treated like an SSP stage (Eq. 53 per stage): its
    input is limited before L is taken and its output y_i (and u^{n+1}) goes through the
    detector and filter; the weighted sum of the L's is not a state and is not filtered.
    With the filter and limiter off this is the textbook scheme."""
    L = scheme.rhs
    u0 = capture.limit(prob, tabs, uhat)
    k = L(prob, tabs, u0)
    acc = u0 + (dt / 6.0) * k
    y = _finish_stage(prob, tabs, u0 + 0.5 * dt * k, dt, record, replay, stage_offset + 0)
    for i, (cy, cacc) in enumerate(((0.5, 1.0 / 3.0), (1.0, 1.0 / 3.0))):
        v = capture.limit(prob, tabs, y)
        k = L(prob, tabs, v)
        acc = acc + (cacc * dt) * k
        y = _finish_stage(prob, tabs, u0 + (cy * dt) * k, dt, record, replay, stage_offset + 1 + i)
    v = capture.limit(prob, tabs, y)
    u = acc + (dt / 6.0) * L(prob, tabs, v)
    return _finish_stage(prob, tabs, u, dt, record, replay, stage_offset + 3)


def run(prob, uhat, dt, nsteps, record=None, replay=None):
    """nsteps SSP-RK3 steps of size dt."""
    tabs = prob.tabs()
    u = uhat
    for n in range(nsteps):
        u = ssp_rk3_step(prob, tabs, u, dt, record=record, replay=replay, stage_offset=3 * n)
    return u


def moments(uhat):
    """Mean and variance of u over z at each solution point: E[u] = uhat_0 (Phi_0 = 1),
    Var[u] = sum_{k >= 1} uhat_k^2 <Phi_k^2> (orthonormal basis, §2.1 Eq. 3)."""
    mean = uhat[:, :, 0, :].copy()
    var = np.sum(uhat[:, :, 1:, :] ** 2, axis=2)
    return mean, var
