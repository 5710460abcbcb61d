"""The FP32_TC form: the 2D stage with the Galerkin projection of the residual (§2.1, Eq. 6
with the quadrature of Eq. 5) on the tensor cores (tcgen05, 3xTF32 products accumulated in
FP32), against the FP64 oracle and against the plain FP32 form.

Stated bounds: residual 1e-5 relative L2 against the oracle (as the FP32 form) and 1e-6
against the FP32 form's own residual (the two differ in the projection's rounding only);
three steps with the oracle's filter decisions replayed and the limiter on, 1e-5.  Tiles of 4
and 8 elements, with a ragged last tile (its unused MMA rows are never read).
"""
import numpy as np
import pytest

from oracle import integrate, scheme
from paper_2112_05946_gb300 import frsg, workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu


def _rhs_gpu(s, u):
    import torch
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    out = torch.empty_like(ud)
    s.rhs(ud, out)
    torch.cuda.synchronize()
    s.check()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("nx,ny,tile", [(8, 4, 4), (8, 4, 8), (6, 4, 4), (10, 3, 8)])
@pytest.mark.parametrize("N", [4, 7])
@pytest.mark.parametrize("bc", [("dirichlet", "dirichlet", "reflect", "reflect"), ("periodic",) * 4])
def test_rhs_tc_matches_oracle_and_fp32(nx, ny, tile, N, bc):
    wl = workloads.shock_vortex_2d(nx=nx, ny=ny, N=N, Q=8)
    prob = oracle_problem(wl, bc=bc)
    s = solver(wl, precision="fp32_tc", bc=bc)
    assert s.set_tile(tile) == tile
    s32 = solver(wl, precision="fp32", bc=bc)
    u = workloads.random_state(s.state_shape, seed=nx + N, base=[1.0, 0.3, -0.2, 2.6], amp=[0.05, 0.05, 0.05, 0.1])
    u32 = u.astype(np.float32).astype(np.float64)
    got = _rhs_gpu(s, u32)
    assert rel_l2(got, scheme.rhs(prob, prob.tabs(), u32)) < 1e-5
    assert rel_l2(got, _rhs_gpu(s32, u32)) < 1e-6


@pytest.mark.parametrize("tile", [4, 8])
def test_tc_steps_with_filter_and_limiter(tile):
    wl = workloads.shock_vortex_2d(nx=16, ny=8)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    s = solver(wl, precision="fp32_tc")
    assert s.set_tile(tile) == tile
    gpu_initial(s, wl)
    u = oracle_initial(prob, wl)
    nflag = 0
    for _ in range(3):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        rec = []
        u = integrate.ssp_rk3_step(prob, tabs, u, dt, record=rec)
        s.set_replay(np.array(rec, dtype=np.uint8))
        s.rk_step(dt, 1, graph=False)
        nflag += int(np.sum(rec))
    s.check()
    assert nflag > 0
    assert rel_l2(s.get_state(), u) < 1e-5


def test_tc_graph_replayed_steps_match_fp32_form():
    wl = workloads.shock_vortex_2d(nx=32, ny=16)
    out = {}
    for p in ("fp32", "fp32_tc"):
        s = solver(wl, precision=p)
        s.set_tile(4)
        gpu_initial(s, wl)
        s.rk_step(2e-4, 10, graph=True)
        s.check()
        out[p] = s.get_state()
    assert rel_l2(out["fp32_tc"], out["fp32"]) < 1e-6


def test_tc_rejects_unsupported_shapes_and_tiles():
    wl = workloads.shock_vortex_2d(nx=8, ny=4)
    for over in (dict(P=2, N=4, Q=8), dict(N=4, Q=10), dict(N=8, Q=8)):
        with pytest.raises(frsg.FrsgError) as ei:
            solver(wl, precision="fp32_tc", **over)
        assert ei.value.status == frsg.E_INVAL
    s = solver(wl, precision="fp32_tc")
    for te in (1, 2, 3, 5, 16):
        with pytest.raises(frsg.FrsgError):
            s.set_tile(te)
