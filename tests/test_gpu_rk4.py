"""Classical RK4 integrator (the advection study's, §5.1) on the CUDA path vs the oracle:
advection, Burgers with detector + filter, Sod with limiter + filter, the 2D shock-vortex
state, the FP32 form, graph replay, and the paper's accuracy study (Tables 2-3) run on the
GPU at the two finest rows."""
import pathlib

import numpy as np
import pytest

from oracle import integrate
from paper_2112_05946_gb300 import workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _oracle_rk4(prob, u, dt, nsteps, rec=None):
    tabs = prob.tabs()
    for n in range(nsteps):
        u = integrate.rk4_step(prob, tabs, u, dt, record=rec, stage_offset=4 * n)
    return u


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("graph", [False, True])
def test_rk4_advection(variant, graph):
    wl = workloads.advection_1d()
    prob = oracle_problem(wl)
    s = solver(wl)
    s.set_variant(variant)
    gpu_initial(s, wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    s.rk4_step(dt, 40, graph=graph)
    s.check()
    ref = _oracle_rk4(prob, oracle_initial(prob, wl), dt, 40)
    assert rel_l2(s.get_state(), ref) < TOL64


def test_rk4_graph_equals_eager():
    wl = workloads.burgers_1d(nx=48)
    a, b = solver(wl), solver(wl)
    gpu_initial(a, wl)
    gpu_initial(b, wl)
    dt = 2e-3
    a.rk4_step(dt, 7, graph=True)
    b.rk4_step(dt, 7, graph=False)
    np.testing.assert_array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("variant", [0, 1])
def test_rk4_burgers_with_filter_replayed(variant):
    """Burgers (P = 3, N = 8, Q = 16, exponential filter + detector) on 64 elements past
    shock formation, with the oracle's stage decisions replayed."""
    wl = workloads.burgers_1d(nx=64)
    prob = oracle_problem(wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    nsteps = 120
    rec = []
    ref = _oracle_rk4(prob, oracle_initial(prob, wl), dt, nsteps, rec)
    assert np.any(np.concatenate(rec))
    s = solver(wl)
    s.set_variant(variant)
    gpu_initial(s, wl)
    s.set_replay(np.array(rec, dtype=np.uint8))
    s.rk4_step(dt, nsteps)
    s.check()
    assert rel_l2(s.get_state(), ref) < TOL64


def test_rk4_sod_with_limiter_and_filter():
    wl = workloads.sod_1d(nx=64)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl)
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    for _ in range(30):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        rec = []
        u = integrate.rk4_step(prob, tabs, u, dt, record=rec)
        s.set_replay(np.array(rec, dtype=np.uint8))
        s.rk4_step(dt, 1)
    s.check()
    assert rel_l2(s.get_state(), u) < 1e-11


def test_rk4_shock_vortex_2d():
    wl = workloads.shock_vortex_2d(nx=16, ny=8)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl)
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    for _ in range(2):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        rec = []
        u = integrate.rk4_step(prob, tabs, u, dt, record=rec)
        s.set_replay(np.array(rec, dtype=np.uint8))
        s.rk4_step(dt, 1)
    s.check()
    assert rel_l2(s.get_state(), u) < TOL64


def test_rk4_fp32_advection():
    """FP32 form: same stated bound as the FP32 SSP-RK3 runs (1e-5 relative L2)."""
    wl = workloads.advection_1d()
    prob = oracle_problem(wl)
    s = solver(wl, precision="fp32")
    gpu_initial(s, wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    s.rk4_step(dt, 40)
    s.check()
    ref = _oracle_rk4(prob, oracle_initial(prob, wl), dt, 40)
    assert rel_l2(s.get_state(), ref) < 1e-5


GOLDEN = pathlib.Path(__file__).parent / "golden" / "advection_rk4_errors.txt"


@pytest.mark.parametrize("P", [2, 3])
def test_paper_accuracy_study_on_gpu(P):
    """§5.1 setup (x in [-1, 1] periodic, xi ~ U(0.9, 1.1), N_c = 5, N_q = 9, RK4, CFL 0.1,
    t = 50) on the GPU at dx = 0.0625 and 0.03125: the point-count-normalised L1 order
    equals the printed L1 order within 0.1 and the Linf order reaches P + 1."""
    from paper_2112_05946_gb300 import frsg
    rows = [l.split() for l in GOLDEN.read_text().splitlines() if l.strip() and not l.startswith("#")]
    printed = [float(r[3]) for r in rows if int(r[0]) == P][-1]
    errs = []
    for nx in (32, 64):
        s = frsg.Solver(dim=1, nx=nx, x0=-1.0, x1=1.0, bc=("periodic",) * 4, P=P, N=5, Q=9, equation="advection",
                        adv_speed=1.0, filter="none")
        x, z = s.nodes()
        s.set_initial_nodal(workloads.nodal_values(
            lambda xx, zz: ((1.0 + 0.1 * zz) * np.sin(np.pi * xx))[..., None], x, z))
        n = int(round(50.0 / (0.1 * 2.0 / nx)))
        s.rk4_step(50.0 / n, n)
        s.check()
        e = s.get_state()[:, :, 0, 0] - np.sin(np.pi * (x - 50.0))
        errs.append(np.array([np.mean(np.abs(e)), np.max(np.abs(e))]))
    orders = np.log2(errs[0] / errs[1])
    assert abs(orders[0] - printed) < 0.1, (orders, printed)
    assert orders[1] > P + 1 - 0.1, orders
