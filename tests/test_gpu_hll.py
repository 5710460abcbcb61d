"""HLL interface flux (Euler setup tables of §5.3-5.4) on the CUDA path vs the oracle: the
residual for scalar, 1D Euler and 2D Euler states in each launch layout, the stochastic
discontinuity-location Sod tube (HLL + Lasso or L2 + limiter), the 2D shock-vortex steps
with HLL, the FP32 form, and admissibility at the benchmark size."""
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


CASES = [
    ("advection", dict(P=2, N=4, Q=8), [1.0], [0.3]),
    ("burgers", dict(P=3, N=8, Q=16), [0.0], [0.5]),                        # transonic faces
    ("sod", dict(P=3, N=6, Q=12), [1.0, 0.2, 2.5], [0.05, 0.3, 0.1]),
    ("sod", dict(P=2, N=9, Q=17), [1.0, 2.2, 4.0], [0.02, 0.05, 0.05]),     # supersonic to the right
    ("sod", dict(P=2, N=9, Q=17), [1.0, -2.2, 4.0], [0.02, 0.05, 0.05]),    # supersonic to the left
]


@pytest.mark.parametrize("name,orders,base,amp", CASES)
@pytest.mark.parametrize("variant", [0, 1])
def test_rhs_hll_parity(name, orders, base, amp, variant):
    wl = workloads.ALL[name]()
    over = dict(orders, nx=37, flux="hll")
    prob = oracle_problem(wl, **over)
    s = solver(wl, **over)
    s.set_variant(variant)
    u = workloads.random_state(s.state_shape, seed=17, base=base, amp=amp)
    assert rel_l2(_rhs_gpu(s, u), scheme.rhs(prob, prob.tabs(), u)) < TOL64


def test_rhs_hll_parity_2d():
    wl = workloads.shock_vortex_2d(nx=7, ny=5, P=3, N=4, Q=8)
    over = dict(flux="hll")
    prob = oracle_problem(wl, **over)
    s = solver(wl, **over)
    u = workloads.random_state(s.state_shape, seed=9, base=[1.0, 0.3, -0.2, 2.6], amp=[0.05, 0.1, 0.1, 0.1])
    assert rel_l2(_rhs_gpu(s, u), scheme.rhs(prob, prob.tabs(), u)) < TOL64


@pytest.mark.parametrize("filt", ["lasso", "l2"])
def test_sod_stochastic_location_run(filt):
    wl = workloads.sod_location_1d(nx=50, filter=filt)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl)
    gpu_initial(s, wl)
    s.limit()         # the z-discontinuous projection has inadmissible z-node states until limited
    u = capture.limit(prob, tabs, oracle_initial(prob, wl))
    for _ in range(25):
        dt = integrate.cfl_dt(prob, tabs, capture.limit(prob, tabs, u), 0.1)
        rec = []
        u = integrate.ssp_rk3_step(prob, tabs, u, dt, record=rec)
        s.set_replay(np.array(rec, dtype=np.uint8))
        s.rk_step(dt, 1, graph=False)
    s.check()
    assert rel_l2(s.get_state(), u) < 1e-11


def test_shock_vortex_hll_steps():
    wl = workloads.shock_vortex_2d(nx=16, ny=8)
    over = dict(flux="hll")
    prob = oracle_problem(wl, **over)
    tabs = prob.tabs()
    s = solver(wl, **over)
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    for _ in range(3):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        rec = []
        u = integrate.ssp_rk3_step(prob, tabs, u, dt, record=rec)
        s.set_replay(np.array(rec, dtype=np.uint8))
        s.rk_step(dt, 1, graph=False)
    s.check()
    assert rel_l2(s.get_state(), u) < TOL64


def test_sod_location_fp32():
    """FP32 form, stated bound for shock problems (1e-3 relative L2 over 20 steps)."""
    wl = workloads.sod_location_1d(nx=50)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl, precision="fp32")
    gpu_initial(s, wl)
    s.limit()
    u = capture.limit(prob, tabs, oracle_initial(prob, wl))
    for _ in range(20):
        dt = integrate.cfl_dt(prob, tabs, capture.limit(prob, tabs, u), 0.1)
        u = integrate.ssp_rk3_step(prob, tabs, u, dt)
        s.rk_step(dt, 1, graph=False)
    s.check()
    assert rel_l2(s.get_state(), u) < 1e-3


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sod_location_full_size_stays_admissible(precision):
    """4096 elements (the benchmark line): after limiting, every z-node state is admissible
    in the context's precision, dt is finite and steps run without errors; the FP64 limiter
    matches the oracle's on the same state."""
    wl = workloads.sod_location_1d(nx=4096)
    s = solver(wl, precision=precision)
    gpu_initial(s, wl)
    s.limit()
    dt = s.cfl_dt(0.05)
    assert np.isfinite(dt) and dt > 0
    s.rk_step(dt, 5, graph=True)
    s.limit()
    assert np.isfinite(s.cfl_dt(0.05))
    s.check()
    if precision == "fp64":
        prob = oracle_problem(wl)
        ref = capture.limit(prob, prob.tabs(), oracle_initial(prob, wl))
        s2 = solver(wl)
        gpu_initial(s2, wl)
        s2.limit()
        s2.check()
        assert rel_l2(s2.get_state(), ref) < 1e-12
