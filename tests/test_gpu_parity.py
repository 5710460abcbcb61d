"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance: relative L2 <= 1e-12 for FP64 results (the paper fixes no precision; the
bound is set by rounding of O(100) flops per coefficient in different order).
Discrete decisions (filter flags, limiter activity) must match exactly.
"""
import numpy as np
import pytest

from oracle import capture, integrate, scheme
from paper_2112_05946_gb300 import workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _torch():
    import torch
    return torch


def _rhs_gpu(s, u):
    torch = _torch()
    dt = torch.float64 if s.fp64 else torch.float32
    ud = torch.tensor(u, dtype=dt, device="cuda")
    out = torch.empty_like(ud)
    s.rhs(ud, out)
    torch.cuda.synchronize()
    s.check()
    return out.double().cpu().numpy()


CASES = [
    ("advection", dict(P=2, N=4, Q=8), [1.0], [0.3]),
    ("burgers", dict(P=1, N=2, Q=4), [0.5], [0.4]),
    ("burgers", dict(P=3, N=8, Q=16), [0.2], [0.5]),
    ("burgers", dict(P=4, N=10, Q=20), [0.2], [0.5]),
    ("burgers", dict(P=2, N=5, Q=7), [0.2], [0.5]),
    ("sod", dict(P=3, N=6, Q=12), [1.0, 0.2, 2.5], [0.05, 0.05, 0.1]),
    ("sod", dict(P=1, N=3, Q=6), [1.0, 0.2, 2.5], [0.05, 0.05, 0.1]),
    ("sod", dict(P=4, N=2, Q=3), [1.0, -0.3, 2.5], [0.05, 0.05, 0.1]),
]


@pytest.mark.parametrize("name,orders,base,amp", CASES)
@pytest.mark.parametrize("tile", [1, 3, 8])
@pytest.mark.parametrize("variant", [0, 1])
def test_rhs_parity(name, orders, base, amp, tile, variant):
    wl = workloads.ALL[name]()
    over = dict(orders, nx=37)
    prob = oracle_problem(wl, **over)
    s = solver(wl, **over)
    s.set_variant(variant)
    if variant == 1 and tile * s.Q * s.Np > 256:
        tile = max(1, 256 // (s.Q * s.Np))
    assert s.set_tile(tile) == tile
    u = workloads.random_state(s.state_shape, seed=11 + tile, base=base, amp=amp)
    ref = scheme.rhs(prob, prob.tabs(), u)
    got = _rhs_gpu(s, u)
    assert rel_l2(got, ref) < TOL64


@pytest.mark.parametrize("bc", [("outflow", "outflow"), ("reflect", "reflect"), ("dirichlet", "outflow")])
@pytest.mark.parametrize("variant", [0, 1])
def test_rhs_boundaries(bc, variant):
    wl = workloads.sod_1d(nx=9, P=2, N=3, Q=6)
    over = dict(bc=bc + ("periodic", "periodic"), nx=9)
    prob = oracle_problem(wl, **over)
    s = solver(wl, **over)
    s.set_variant(variant)
    s.set_tile(3)
    u = workloads.random_state(s.state_shape, seed=3, base=[1.0, 0.4, 2.5], amp=[0.05, 0.05, 0.1])
    got = _rhs_gpu(s, u)
    ref = scheme.rhs(prob, prob.tabs(), u)
    assert rel_l2(got, ref) < TOL64


def test_initial_projection_and_moments():
    wl = workloads.burgers_1d(nx=21)
    prob = oracle_problem(wl)
    s = solver(wl)
    gpu_initial(s, wl)
    ref = oracle_initial(prob, wl)
    got = s.get_state()
    assert rel_l2(got, ref) < 1e-14
    m, v = s.moments()
    rm, rv = integrate.moments(ref)
    assert rel_l2(m, rm) < 1e-14 and rel_l2(v, rv) < 1e-13


@pytest.mark.parametrize("name", ["burgers", "sod"])
def test_cfl_dt(name):
    wl = workloads.ALL[name](nx=50)
    prob = oracle_problem(wl)
    s = solver(wl)
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    assert abs(s.cfl_dt(0.1) / integrate.cfl_dt(prob, prob.tabs(), u, 0.1) - 1) < 1e-13


@pytest.mark.parametrize("tile", [1, 3])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_one_step_burgers_with_filter(tile, variant):
    """One SSP-RK3 step with the detector-switched exponential filter, from a state with
    a steep front so that some elements are flagged and others are not."""
    wl = workloads.burgers_1d(nx=40)
    prob = oracle_problem(wl)
    s = solver(wl)
    s.set_variant(variant)
    s.set_tile(tile)
    x = s.nodes()[0]
    rng = np.random.default_rng(4)
    u = workloads.random_state(s.state_shape, seed=5, base=[0.0], amp=[1e-3])
    u[:, :, 0, 0] += np.tanh((x - 1.0) / 0.03)
    u[:, :, 1, 0] += 0.1 * rng.random()
    s.set_state(u)
    dt = 0.1 * prob.dx / 1.2
    rec = []
    ref = integrate.ssp_rk3_step(prob, prob.tabs(), u, dt, record=rec)
    s.rk_step(dt, 1, graph=False)
    s.check()
    flags, _ = s.decisions()
    assert 0 < np.sum(rec[0]) < prob.E
    np.testing.assert_array_equal(flags, np.array(rec))
    assert rel_l2(s.get_state(), ref) < TOL64


def test_limiter_parity():
    wl = workloads.sod_1d(nx=6, P=2, N=3, Q=6)
    prob = oracle_problem(wl)
    s = solver(wl)
    u = np.zeros(s.state_shape)
    rng = np.random.default_rng(3)
    u[:, :, 0, :] = [1.0, 0.2, 2.5]
    u[:, :, 1:, :] = 0.01 * rng.standard_normal((6, 3, 3, 3))
    u[1, 0, 0, 0] = -0.4
    u[1, 2, 0, 0] = 2.4
    u[2, 1, 0, 2] = 0.002
    u[2, 0, 0, 2] = 4.0
    s.set_state(u)
    s.limit()
    s.check()
    rec = []
    ref = capture.limit(prob, prob.tabs(), u, record=rec)
    _, beta = s.decisions()
    np.testing.assert_allclose(beta[0], rec[0], rtol=1e-12)
    assert rel_l2(s.get_state(), ref) < TOL64


def test_advection_full_run_matches_oracle_and_closed_form():
    """Whole advection workload (32 elements, 320 steps to t = 2), graph replay."""
    wl = workloads.advection_1d()
    prob = oracle_problem(wl)
    s = solver(wl)
    gpu_initial(s, wl)
    u0 = oracle_initial(prob, wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    nsteps = int(round(wl["t_end"] / dt))
    s.rk_step(dt, nsteps, graph=True)
    s.check()
    ref = integrate.run(prob, u0, dt, nsteps)
    got = s.get_state()
    assert rel_l2(got, ref) < TOL64
    exact = integrate.project_initial(prob, wl["exact"](wl["t_end"]))
    assert np.sqrt(np.mean((got - exact) ** 2)) < 2e-5


def test_burgers_run_past_shock_with_replayed_decisions():
    """Burgers (P = 3, N = 8, Q = 16) on 64 elements past shock formation; the oracle's
    filter decisions are replayed on the GPU, and the free-running GPU decisions are
    compared with them as well."""
    wl = workloads.burgers_1d(nx=64)
    prob = oracle_problem(wl)
    u0 = oracle_initial(prob, wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    nsteps = 120   # t ~ 0.34 > 1/pi
    rec = []
    ref = integrate.run(prob, u0, dt, nsteps, record=rec)
    assert np.any(np.concatenate(rec))
    for variant in (0, 1, 2, 3):
        s = solver(wl)
        s.set_variant(variant)
        gpu_initial(s, wl)
        s.set_replay(np.array(rec, dtype=np.uint8))
        s.rk_step(dt, nsteps, graph=True)
        s.check()
        assert rel_l2(s.get_state(), ref) < 1e-11, variant
    # free run: decisions compared stage by stage
    s2 = solver(wl)
    gpu_initial(s2, wl)
    mism = 0
    for n in range(nsteps):
        s2.rk_step(dt, 1, graph=False)
        f, _ = s2.decisions()
        mism += int(np.sum(f != np.array(rec[3 * n:3 * n + 3])))
    assert mism <= 2
    if mism == 0:
        assert rel_l2(s2.get_state(), ref) < 1e-11


def test_sod_run_with_limiter_and_filter():
    wl = workloads.sod_1d(nx=64)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl)
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    for _ in range(40):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        dt_gpu = s.cfl_dt(0.1)
        assert abs(dt_gpu / dt - 1) < 1e-12
        rec = []
        u = integrate.ssp_rk3_step(prob, tabs, u, dt, record=rec)
        s.set_replay(np.array(rec, dtype=np.uint8))
        s.rk_step(dt, 1, graph=False)
    s.check()
    assert rel_l2(s.get_state(), u) < 1e-11


@pytest.mark.parametrize("name", ["burgers", "sod"])
def test_full_size_one_step(name):
    """Full benchmark sizes (Burgers 1024 elements, Sod 4096 elements), one step in the
    graph-replayed launch configuration the benchmark times, every coefficient compared."""
    wl = workloads.ALL[name]()
    prob = oracle_problem(wl)
    s = solver(wl)
    gpu_initial(s, wl)
    u0 = oracle_initial(prob, wl)
    tabs = prob.tabs()
    dt = integrate.cfl_dt(prob, tabs, u0, wl["cfl"])
    rec = []
    ref = integrate.ssp_rk3_step(prob, tabs, u0, dt, record=rec)
    s.rk_step(dt, 1, graph=True)
    s.check()
    flags, _ = s.decisions()
    np.testing.assert_array_equal(flags, np.array(rec))
    assert rel_l2(s.get_state(), ref) < TOL64


def test_conservation_full_size_burgers():
    """Cell integral of the mean (mode 0) stays constant through 200 filtered steps, to
    rounding: 1e-14 of the integral of |u| per stage."""
    wl = workloads.burgers_1d()
    prob = oracle_problem(wl)
    s = solver(wl)
    gpu_initial(s, wl)
    w = prob.tabs()["w"]
    I0 = np.einsum("j,ej->", w, s.get_state()[:, :, 0, 0])
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    s.rk_step(dt, 200, graph=True)
    s.check()
    I1 = np.einsum("j,ej->", w, s.get_state()[:, :, 0, 0])
    scale = np.einsum("j,ej->", w, np.abs(s.get_state()[:, :, 0, 0]))
    assert abs(I1 - I0) < 1e-14 * scale * 600


def test_nonfinite_input_is_reported():
    from paper_2112_05946_gb300 import frsg
    wl = workloads.burgers_1d(nx=8)
    s = solver(wl)
    u = workloads.random_state(s.state_shape, seed=1, base=[0.5], amp=[0.1])
    u[3, 1, 0, 0] = np.nan
    s.set_state(u)
    s.rk_step(1e-3, 1, graph=False)
    with pytest.raises(frsg.FrsgError) as ei:
        s.check()
    assert ei.value.status == frsg.E_NONFINITE
    s.check()   # the error word was cleared


def test_inadmissible_mean_is_reported():
    from paper_2112_05946_gb300 import frsg
    wl = workloads.sod_1d(nx=8, P=2, N=2, Q=4)
    s = solver(wl)
    u = workloads.random_state(s.state_shape, seed=1, base=[1.0, 0.0, 2.5], amp=[0.01, 0.01, 0.01])
    u[4, :, 0, 0] = -1.0
    s.set_state(u)
    s.limit()
    with pytest.raises(frsg.FrsgError) as ei:
        s.check()
    assert ei.value.status == frsg.E_POSITIVITY


@pytest.mark.parametrize("name", ["burgers", "sod"])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("fp32", 1e-5)])
def test_autotuned_choice_keeps_parity(name, precision, tol):
    wl = workloads.ALL[name](nx=64)
    prob = oracle_problem(wl)
    s = solver(wl, precision=precision)
    variant, tile = s.autotune(reps=2)
    assert variant in (0, 1, 2, 3) and tile >= 1
    base = [0.2] if name == "burgers" else [1.0, 0.2, 2.5]
    amp = [0.5] if name == "burgers" else [0.05, 0.05, 0.1]
    u = workloads.random_state(s.state_shape, seed=8, base=base, amp=amp)
    if precision == "fp32":
        u = u.astype(np.float32).astype(np.float64)
    ref = scheme.rhs(prob, prob.tabs(), u)
    assert rel_l2(_rhs_gpu(s, u), ref) < tol
    # a second context of the same shape takes the cached choice
    s2 = solver(wl, precision=precision)
    assert s2.autotune() == (variant, tile)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("fp32", 1e-5)])
def test_one_launch_step_full_size(precision, tol):
    """Variant 2 (three stages in one cooperative launch) on the 1024-element Burgers
    workload: 50 steps against the oracle and against the three-launch path."""
    wl = workloads.burgers_1d()
    prob = oracle_problem(wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    ref = integrate.run(prob, oracle_initial(prob, wl), dt, 50)
    outs = []
    for variant in (2, 0):
        s = solver(wl, precision=precision)
        s.set_variant(variant)
        gpu_initial(s, wl)
        s.rk_step(dt, 50, graph=True)
        s.check()
        outs.append(s.get_state())
        assert rel_l2(outs[-1], ref) < tol
    assert rel_l2(outs[0], outs[1]) < (1e-14 if precision == "fp64" else 1e-6)
