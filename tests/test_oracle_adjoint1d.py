"""Pins for the general 1D reverse-mode oracle (oracle.adjoint1d).

The limited states sit on the positivity floor (a point at p = 1e-8), where the sound speed
is so ill-conditioned that central differences of a whole run are not in their linear range.
So the pieces are pinned separately, each against central differences of the numpy oracle:
the limiter's vector-Jacobian product where it acts strictly (the raw projection of the
stochastic-location Sod state); the residual's at generic admissible Euler states (LLF and
HLL; Dirichlet, outflow and reflecting ends) and for Burgers; whole runs where the limiter
stays inactive.  The forward step equals the numpy step where the limiter acts; autograd
composes the pieces."""
import numpy as np
import pytest
import torch

from oracle import adjoint1d, capture, integrate, scheme
from paper_2112_05946_gb300 import workloads
from tests.helpers import oracle_initial, oracle_problem


def _vjp(fn_t, x, lam):
    xt = torch.tensor(x, requires_grad=True)
    (g,) = torch.autograd.grad(fn_t(xt), xt, grad_outputs=torch.tensor(lam))
    return g.numpy()


def _check(fn_np, fn_t, x, seed, rel=1e-6):
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal(x.shape)
    g = _vjp(fn_t, x, lam)
    for _ in range(3):
        v = rng.standard_normal(x.shape)
        h = 1e-6 * np.linalg.norm(x) / np.linalg.norm(v)
        fd = np.sum(lam * (fn_np(x + h * v) - fn_np(x - h * v))) / (2 * h)
        assert np.sum(g * v) == pytest.approx(fd, rel=rel, abs=1e-10 * np.abs(g).sum())


def _sod_location(iflux="llf"):
    wl = workloads.sod_location_1d(nx=12, P=2, N=3, Q=5, filter="l2")
    return wl, oracle_problem(wl, flux=iflux, sensor=False)


def test_limiter_vjp_where_it_acts():
    wl, prob = _sod_location()
    tabs, tt = prob.tabs(), adjoint1d.tabs_torch(prob)
    u0 = oracle_initial(prob, wl)
    rec = []
    capture.limit(prob, tabs, u0, record=rec)
    assert np.sum(rec[0] < 1.0) >= 2
    _check(lambda x: capture.limit(prob, tabs, x), lambda x: adjoint1d.limit(prob, tt, x), u0, 1)


@pytest.mark.parametrize("iflux", ["llf", "hll"])
@pytest.mark.parametrize("bc", [("dirichlet", "dirichlet"), ("outflow", "reflect"), ("periodic", "periodic")])
def test_residual_vjp_euler(iflux, bc):
    wl, prob = _sod_location(iflux)
    prob.bc = bc + ("periodic", "periodic")
    tabs, tt = prob.tabs(), adjoint1d.tabs_torch(prob)
    u = workloads.random_state((prob.E, prob.Np, prob.M, prob.S), seed=4, base=[1.0, 0.3, 2.5], amp=[0.1, 0.3, 0.2])
    _check(lambda x: scheme.rhs(prob, tabs, x), lambda x: adjoint1d.rhs(prob, tt, x), u, 2)


def test_residual_vjp_burgers_outflow():
    wl = workloads.burgers_1d(nx=10, P=2, N=3, Q=6)
    prob = oracle_problem(wl, bc=("outflow", "outflow", "periodic", "periodic"))
    tabs, tt = prob.tabs(), adjoint1d.tabs_torch(prob)
    u = workloads.random_state((prob.E, prob.Np, prob.M, prob.S), seed=5, base=[0.3], amp=[0.5])
    _check(lambda x: scheme.rhs(prob, tabs, x), lambda x: adjoint1d.rhs(prob, tt, x), u, 3)


def test_forward_step_matches_numpy_with_limiter_acting():
    for iflux in ("llf", "hll"):
        wl, prob = _sod_location(iflux)
        tabs, tt = prob.tabs(), adjoint1d.tabs_torch(prob)
        u0 = oracle_initial(prob, wl)
        dt = integrate.cfl_dt(prob, tabs, capture.limit(prob, tabs, u0), 0.1)
        rec = []
        ref = u0
        for n in range(3):
            ref = integrate.ssp_rk3_step(prob, tabs, ref, dt, record=rec, stage_offset=3 * n)
        u = torch.tensor(u0)
        for n in range(3):
            u = adjoint1d.step(prob, tt, u, dt, rec[3 * n:3 * n + 3])
        assert np.max(np.abs(u.numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("case", ["euler_smooth", "burgers_filtered"])
def test_run_vjp_without_active_limiter(case):
    if case == "euler_smooth":
        wl, prob = _sod_location("hll")
        prob.bc = ("periodic",) * 4
        prob.filter = "exp"
        u0 = workloads.random_state((prob.E, prob.Np, prob.M, prob.S), seed=6, base=[1.0, 0.3, 2.5],
                                    amp=[0.05, 0.1, 0.1])
    else:
        wl = workloads.burgers_1d(nx=10, P=3, N=4, Q=8)
        prob = oracle_problem(wl, bc=("outflow", "outflow", "periodic", "periodic"), sensor=False)
        u0 = oracle_initial(prob, wl)
    tabs = prob.tabs()
    dt = integrate.cfl_dt(prob, tabs, u0, 0.1)
    rec = []
    u = u0
    for n in range(3):
        u = integrate.ssp_rk3_step(prob, tabs, u, dt, record=rec, stage_offset=3 * n)
    rng = np.random.default_rng(7)
    lam = rng.standard_normal(u0.shape)
    uT, g = adjoint1d.vjp(prob, u0, [dt] * 3, rec, lam)
    assert np.max(np.abs(uT - u)) <= 1e-13 * np.max(np.abs(u))

    def run(x):
        for n in range(3):
            x = integrate.ssp_rk3_step(prob, tabs, x, dt, replay=rec, stage_offset=3 * n)
        return x
    for _ in range(2):
        v = rng.standard_normal(u0.shape)
        h = 1e-6 * np.linalg.norm(u0) / np.linalg.norm(v)
        fd = np.sum(lam * (run(u0 + h * v) - run(u0 - h * v))) / (2 * h)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)
