"""2D tensor-product CUDA path vs the FP64 oracle (shock-vortex workload family)."""
import numpy as np
import pytest

from oracle import capture, integrate, scheme
from paper_2112_05946_gb300 import workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _rhs_gpu(s, u):
    import torch
    dt = torch.float64 if s.fp64 else torch.float32
    ud = torch.tensor(u, dtype=dt, device="cuda")
    out = torch.empty_like(ud)
    s.rhs(ud, out)
    torch.cuda.synchronize()
    s.check()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("P,N,Q", [(1, 2, 4), (2, 3, 6), (3, 4, 8)])
@pytest.mark.parametrize("bc", [("periodic",) * 4, ("dirichlet", "dirichlet", "reflect", "reflect"),
                                ("outflow", "reflect", "outflow", "periodic")])
@pytest.mark.parametrize("tile", [1, 3])
def test_rhs_2d_parity(P, N, Q, bc, tile):
    if bc[2] == "outflow" and bc[3] == "periodic":
        bc = ("outflow", "reflect", "periodic", "periodic")
    wl = workloads.shock_vortex_2d(nx=7, ny=5, P=P, N=N, Q=Q)
    over = dict(bc=bc)
    prob = oracle_problem(wl, **over)
    s = solver(wl, **over)
    assert s.set_tile(tile) == tile
    u = workloads.random_state(s.state_shape, seed=7 + P, base=[1.0, 0.3, -0.2, 2.6],
                               amp=[0.05, 0.05, 0.05, 0.1])
    ref = scheme.rhs(prob, prob.tabs(), u)
    got = _rhs_gpu(s, u)
    assert rel_l2(got, ref) < TOL64


def test_shock_vortex_initial_state_rhs():
    wl = workloads.shock_vortex_2d(nx=16, ny=8)
    prob = oracle_problem(wl)
    s = solver(wl)
    gpu_initial(s, wl)
    u0 = oracle_initial(prob, wl)
    assert rel_l2(s.get_state(), u0) < 1e-14
    got = _rhs_gpu(s, u0)
    ref = scheme.rhs(prob, prob.tabs(), u0)
    assert rel_l2(got, ref) < TOL64


@pytest.mark.parametrize("tile", [1, 4])
def test_shock_vortex_steps_with_filter_and_limiter(tile):
    """Three SSP-RK3 steps on a 16 x 8 mesh with detector + L2 filter and the limiter;
    decisions compared exactly, state to 1e-12."""
    wl = workloads.shock_vortex_2d(nx=16, ny=8)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl)
    s.set_tile(tile)
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    nflag = 0
    for _ in range(3):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        assert abs(s.cfl_dt(0.1) / dt - 1) < 1e-12
        rec = []
        u = integrate.ssp_rk3_step(prob, tabs, u, dt, record=rec)
        s.rk_step(dt, 1, graph=False)
        flags, _ = s.decisions()
        np.testing.assert_array_equal(flags, np.array(rec))
        nflag += int(np.sum(rec))
    s.check()
    assert nflag > 0
    assert rel_l2(s.get_state(), u) < TOL64


def test_limiter_2d_parity():
    wl = workloads.shock_vortex_2d(nx=3, ny=2, P=2, N=2, Q=4)
    prob = oracle_problem(wl)
    s = solver(wl)
    rng = np.random.default_rng(9)
    u = np.zeros(s.state_shape)
    u[:, :, 0, :] = [1.0, 0.2, 0.1, 2.5]
    u[:, :, 1:, :] = 0.01 * rng.standard_normal((6, 9, 2, 4))
    u[1, 0, 0, 0] = -0.5
    u[1, 8, 0, 0] = 2.5
    u[4, 3, 0, 3] = 0.01
    s.set_state(u)
    s.limit()
    s.check()
    rec = []
    ref = capture.limit(prob, prob.tabs(), u, record=rec)
    _, beta = s.decisions()
    assert np.sum(rec[0] < 1) >= 2
    np.testing.assert_allclose(beta[0], rec[0], rtol=1e-12)
    assert rel_l2(s.get_state(), ref) < TOL64
