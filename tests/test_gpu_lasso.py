"""Lasso filter (§4.1.3) on the CUDA path vs the oracle: the filter alone on random states
(several P, N; scalar and Euler), whole SSP-RK3 runs with the filter on every element in
each 1D launch layout, the Sod tube with the limiter, the FP32 form, conservation of the
mean, and the rejection of 2D contexts."""
import numpy as np
import pytest

from oracle import capture, integrate
from paper_2112_05946_gb300 import frsg, workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _burgers_lasso(nx=40, P=3, N=8, Q=16):
    wl = workloads.burgers_1d(nx=nx, P=P, N=N, Q=Q)
    wl["solver"].update(filter="lasso", sensor=False)
    return wl


@pytest.mark.parametrize("P,N", [(1, 2), (2, 4), (3, 8), (4, 10)])
def test_lasso_filter_alone_scalar(P, N):
    wl = _burgers_lasso(nx=12, P=P, N=N, Q=2 * N)
    prob = oracle_problem(wl)
    s = solver(wl)
    u = workloads.random_state(s.state_shape, seed=P * 10 + N, base=[0.2], amp=[1.0])
    s.set_state(u)
    s.filter(1e-3)
    s.check()
    ref = capture.apply_filter(prob, prob.tabs(), u, 1e-3, np.ones(prob.E, dtype=bool))
    assert rel_l2(s.get_state(), ref) < TOL64


def test_lasso_filter_alone_euler():
    wl = workloads.sod_1d(nx=10, P=2, N=4, Q=8)
    wl["solver"].update(filter="lasso", sensor=False)
    prob = oracle_problem(wl)
    s = solver(wl)
    u = workloads.random_state(s.state_shape, seed=3, base=[1.0, 0.2, 2.5], amp=[0.2, 0.2, 0.3])
    s.set_state(u)
    s.filter(1e-3)
    s.check()
    ref = capture.apply_filter(prob, prob.tabs(), u, 1e-3, np.ones(prob.E, dtype=bool))
    assert rel_l2(s.get_state(), ref) < TOL64


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_lasso_burgers_run(variant):
    wl = _burgers_lasso(nx=64)
    prob = oracle_problem(wl)
    s = solver(wl)
    s.set_variant(variant)
    gpu_initial(s, wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    s.rk_step(dt, 60, graph=True)
    s.check()
    ref = integrate.run(prob, oracle_initial(prob, wl), dt, 60)
    assert rel_l2(s.get_state(), ref) < TOL64


def test_lasso_sod_with_limiter():
    wl = workloads.sod_1d(nx=64)
    wl["solver"].update(filter="lasso", sensor=False)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl)
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    for _ in range(30):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        u = integrate.ssp_rk3_step(prob, tabs, u, dt)
        s.rk_step(dt, 1, graph=False)
    s.check()
    assert rel_l2(s.get_state(), u) < 1e-11


def test_lasso_fp32_burgers():
    wl = _burgers_lasso(nx=64)
    prob = oracle_problem(wl)
    s = solver(wl, precision="fp32")
    gpu_initial(s, wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    s.rk_step(dt, 30)
    s.check()
    ref = integrate.run(prob, oracle_initial(prob, wl), dt, 30)
    assert rel_l2(s.get_state(), ref) < 1e-5


def test_lasso_conserves_mean_on_gpu():
    wl = _burgers_lasso(nx=256)
    prob = oracle_problem(wl)
    s = solver(wl)
    gpu_initial(s, wl)
    w = prob.tabs()["w"]
    u0 = s.get_state()
    m0 = np.sum(w[None, :] * u0[:, :, 0, 0])
    s.rk_step(wl["cfl"] * prob.dx / wl["lam0"], 200)
    s.check()
    u = s.get_state()
    scale = np.sum(np.abs(w[None, :] * u[:, :, 0, 0]))
    assert abs(np.sum(w[None, :] * u[:, :, 0, 0]) - m0) < 1e-14 * scale * 600


def test_lasso_rejected_in_2d():
    wl = workloads.shock_vortex_2d(nx=4, ny=4)
    with pytest.raises(frsg.FrsgError):
        solver(wl, filter="lasso")
