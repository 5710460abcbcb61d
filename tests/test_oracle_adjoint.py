"""Pins for the oracle adjoint (gradients of E and Var of the spatial integral of u at T
w.r.t. the initial gPC coefficients): the torch transcription reproduces the numpy forward,
the gradients match central finite differences of the numpy oracle (filter decisions
replayed), and the closed forms of conservative, periodic schemes hold."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, integrate, tables


def _setup(eq="burgers", filt="exp", nx=12, P=2, N=3):
    prob = oracle.Problem(nx=nx, P=P, N=N, Q=2 * N + 1, equation=eq, x0=0.0, x1=2.0, filter=filt,
                          f_alpha=36.0, f_s=4.0, s0=-2 * np.log10(max(P, 2)), kappa=4.0)
    u0 = integrate.project_initial(prob, lambda x, z: (np.sin(np.pi * x) + 0.1 * z + 0.3)[..., None])
    return prob, u0


def _qoi(prob, u):
    w = tables.fr_tables(prob.P)["w"]
    I = 0.5 * prob.dx * np.einsum("j,ejk->k", w, u[..., 0])
    return I[0], np.sum(I[1:] ** 2)


@pytest.mark.parametrize("eq,filt", [("burgers", "exp"), ("burgers", "none"), ("advection", "none")])
def test_torch_forward_matches_numpy_oracle(eq, filt):
    prob, u0 = _setup(eq, filt)
    dt = 0.1 * prob.dx / 1.3
    rec = []
    ref = integrate.run(prob, u0, dt, 25, record=rec)
    g = adjoint.gradients(prob, u0, dt, 25, rec)
    np.testing.assert_allclose(g["state"], ref, atol=1e-13)


def test_gradients_match_central_differences():
    prob, u0 = _setup("burgers", "exp")
    dt = 0.1 * prob.dx / 1.3
    nsteps = 60          # past shock formation (t ~ 0.7 > 1/pi); some elements filtered
    rec = []
    integrate.run(prob, u0, dt, nsteps, record=rec)
    assert np.any(np.concatenate(rec))
    g = adjoint.gradients(prob, u0, dt, nsteps, rec)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(3):
        v = rng.standard_normal(u0.shape)
        up = integrate.run(prob, u0 + h * v, dt, nsteps, replay=rec)
        um = integrate.run(prob, u0 - h * v, dt, nsteps, replay=rec)
        mp, vp = _qoi(prob, up)
        mm, vm = _qoi(prob, um)
        fd_m = (mp - mm) / (2 * h)
        fd_v = (vp - vm) / (2 * h)
        assert abs(np.sum(g["grad_mean"] * v) - fd_m) < 1e-7 * max(1.0, abs(fd_m))
        assert abs(np.sum(g["grad_var"] * v) - fd_v) < 1e-6 * max(1e-3, abs(fd_v))


def test_closed_forms_of_conservative_periodic_runs():
    """The mean integral is conserved (periodic, conservative FR, filter keeps mode 0), so
    d E/d uhat_{e,j,k}(0) = J w_j for k = 0 and 0 otherwise; for linear advection without a
    filter every I_k is conserved and d Var / d uhat_{e,j,k}(0) = 2 I_k J w_j for k >= 1."""
    prob, u0 = _setup("burgers", "exp")
    dt = 0.1 * prob.dx / 1.3
    rec = []
    integrate.run(prob, u0, dt, 40, record=rec)
    g = adjoint.gradients(prob, u0, dt, 40, rec)
    gm, _ = adjoint.qoi_seeds(prob, u0)
    np.testing.assert_allclose(g["grad_mean"], gm, atol=1e-12)
    prob, u0 = _setup("advection", "none")
    dt = 0.1 * prob.dx
    rec = []
    integrate.run(prob, u0, dt, 40, record=rec)
    g = adjoint.gradients(prob, u0, dt, 40, rec)
    _, gv = adjoint.qoi_seeds(prob, u0)
    np.testing.assert_allclose(g["grad_var"], gv, atol=1e-12)
