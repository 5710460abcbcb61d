"""Discrete adjoint of 1D Euler runs on the GPU (fr_sg_forward_record / fr_sg_adjoint) against
the reverse-mode oracle (oracle.adjoint1d): the LLF and HLL fluxes, Dirichlet, outflow, reflecting and
periodic ends, the filter (decisions frozen) and the positivity limiter differentiated through
its scalings (the stochastic-location Sod state, where the limiter acts from the first stage)."""
import numpy as np
import pytest

from oracle import adjoint1d, capture, integrate
from paper_2112_05946_gb300 import workloads
from tests.helpers import oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu


def _run_case(wl, prob, u0, nsteps, k):
    import torch
    tabs = prob.tabs()
    dt = integrate.cfl_dt(prob, tabs, capture.limit(prob, tabs, u0), 0.1)
    rec = []
    ref = u0
    for n in range(nsteps):
        ref = integrate.ssp_rk3_step(prob, tabs, ref, dt, record=rec, stage_offset=3 * n)
    s = solver(wl, **{kk: getattr(prob, kk) for kk in ("bc", "filter", "sensor")})
    s.set_state(np.ascontiguousarray(u0))
    s.forward_record(dt, nsteps, k)
    s.check()
    assert rel_l2(s.get_state(), ref) < 1e-12
    rng = np.random.default_rng(11)
    lam = rng.standard_normal(u0.shape)
    _, g_ref = adjoint1d.vjp(prob, u0, [dt] * nsteps, rec, lam)
    g = torch.empty(u0.shape, dtype=torch.float64, device="cuda")
    s.adjoint(torch.tensor(lam, device="cuda"), g)
    s.check()
    assert rel_l2(g.cpu().numpy(), g_ref) < 1e-10
    assert rel_l2(s.get_state(), ref) < 1e-12


@pytest.mark.parametrize("nsteps,k", [(3, 2), (4, 1)])
def test_euler_adjoint_with_active_limiter(nsteps, k):
    wl = workloads.sod_location_1d(nx=16, P=2, N=3, Q=5, filter="l2")
    wl["solver"]["flux"] = "llf"
    wl["solver"]["sensor"] = False
    prob = oracle_problem(wl)
    u0 = oracle_initial(prob, wl)              # raw projection: the limiter acts strictly
    rec = []
    capture.limit(prob, prob.tabs(), u0, record=rec)
    assert np.sum(rec[0] < 1.0) >= 2
    _run_case(wl, prob, u0, nsteps, k)


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("outflow", "reflect"), ("dirichlet", "dirichlet")])
def test_euler_adjoint_smooth_states(bc):
    wl = workloads.sod_location_1d(nx=12, P=3, N=4, Q=8, filter="l2")
    wl["solver"].update(flux="llf", sensor=False, bc=bc + ("periodic", "periodic"))
    prob = oracle_problem(wl)
    u0 = workloads.random_state((prob.E, prob.Np, prob.M, prob.S), seed=6, base=[1.0, 0.3, 2.5],
                                amp=[0.05, 0.1, 0.1])
    _run_case(wl, prob, u0, 3, 2)


@pytest.mark.parametrize("bc", [("dirichlet", "dirichlet"), ("outflow", "reflect"), ("periodic", "periodic")])
def test_euler_adjoint_hll_smooth_states(bc):
    """The HLL flux's transpose, with subsonic faces (the HLL middle state and its signal-speed
    derivatives) and every boundary kind."""
    wl = workloads.sod_location_1d(nx=12, P=3, N=4, Q=8, filter="l2")
    wl["solver"].update(flux="hll", sensor=False, bc=bc + ("periodic", "periodic"))
    prob = oracle_problem(wl)
    u0 = workloads.random_state((prob.E, prob.Np, prob.M, prob.S), seed=8, base=[1.0, 0.3, 2.5],
                                amp=[0.05, 0.1, 0.1])
    _run_case(wl, prob, u0, 3, 2)


@pytest.mark.parametrize("vel", [2.2, -2.2])
def test_euler_adjoint_hll_supersonic(vel):
    """Supersonic flow: every face takes the upwind branch of HLL."""
    wl = workloads.sod_location_1d(nx=10, P=2, N=3, Q=6, filter="l2")
    wl["solver"].update(flux="hll", sensor=False, bc=("periodic",) * 4)
    prob = oracle_problem(wl)
    u0 = workloads.random_state((prob.E, prob.Np, prob.M, prob.S), seed=4, base=[1.0, vel, 4.0],
                                amp=[0.02, 0.05, 0.05])
    _run_case(wl, prob, u0, 2, 1)


@pytest.mark.parametrize("nsteps,k", [(3, 2)])
def test_euler_adjoint_hll_with_active_limiter(nsteps, k):
    wl = workloads.sod_location_1d(nx=16, P=2, N=3, Q=5, filter="l2")
    wl["solver"]["flux"] = "hll"
    wl["solver"]["sensor"] = False
    prob = oracle_problem(wl)
    u0 = oracle_initial(prob, wl)
    rec = []
    capture.limit(prob, prob.tabs(), u0, record=rec)
    assert np.sum(rec[0] < 1.0) >= 2
    _run_case(wl, prob, u0, nsteps, k)


def test_scalar_adjoint_rejects_hll():
    from paper_2112_05946_gb300 import frsg
    wl = workloads.burgers_1d(nx=8)
    s = solver(wl, flux="hll")
    with pytest.raises(frsg.FrsgError):
        s.forward_record(1e-4, 2, 1)
