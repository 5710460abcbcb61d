"""The allocation-free entry point fr_sg_rk_step_noalloc against fr_sg_rk_step.

fr_sg_rk_step_noalloc serves callers that may not allocate device memory (their GPU memory
belongs to another allocator, or they sit on a latency-critical path where cudaMalloc and
cudaFree would synchronise the device).  It keeps its scratch in a static device array,
so this test checks that two calls in a row, each reusing what the previous call left
in that array, give the same states as the context-based entry point, within the FP64
tolerance of the other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import tables
from paper_2112_05946_gb300 import workloads
from tests.helpers import gpu_initial, rel_l2, solver

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _ghost_modes(wl, M, S, Q):
    g = tables.gpc_tables(M - 1, Q)
    out = np.zeros((4, M, S))
    for side, fn in wl.get("boundary", {}).items():
        out[side] = g["Pz"] @ workloads.boundary_values(fn, g["z"])
    return out


def _workload(name, nx):
    if name == "advection":
        return workloads.advection_1d()
    if name == "sod_location_l2":
        # HLL flux, L2 filter behind the detector, limiter, Dirichlet ends
        return workloads.sod_location_1d(nx=nx, filter="l2")
    return workloads.ALL[name](nx=nx)


@pytest.mark.parametrize("name,nx,nsteps", [("burgers", 1024, 5), ("sod", 512, 3), ("advection", 32, 10),
                                             ("sod_location_l2", 100, 3)])
def test_noalloc_matches_context_path_on_two_calls(name, nx, nsteps):
    import torch
    from paper_2112_05946_gb300 import frsg
    wl = _workload(name, nx)
    s = solver(wl)
    gpu_initial(s, wl)
    u0 = torch.tensor(s.get_state(), dtype=torch.float64, device="cuda")
    dx = (wl["solver"]["x1"] - wl["solver"]["x0"]) / wl["solver"]["nx"]
    dt = wl["cfl"] * dx / (wl["lam0"] or 2.5)
    ghost = _ghost_modes(wl, s.M, s.S, s.Q) if "boundary" in wl else None
    stream = torch.cuda.current_stream().cuda_stream
    out1 = torch.empty_like(u0)
    out2 = torch.empty_like(u0)
    # first call, then a second call that starts from the first call's output
    frsg.rk_step_noalloc(u0, out1, dt, nsteps, ghost_modes=ghost, stream=stream, **wl["solver"])
    frsg.rk_step_noalloc(out1, out2, dt, nsteps, ghost_modes=ghost, stream=stream, **wl["solver"])
    torch.cuda.synchronize()
    s.rk_step(dt, nsteps, graph=False)
    s.check()
    ref1 = s.get_state()
    s.rk_step(dt, nsteps, graph=False)
    s.check()
    ref2 = s.get_state()
    assert rel_l2(out1.cpu().numpy(), ref1) < TOL64
    assert rel_l2(out2.cpu().numpy(), ref2) < TOL64


def test_noalloc_rejects_oversized_problem():
    import torch
    from paper_2112_05946_gb300 import frsg
    wl = workloads.burgers_1d(nx=65536)   # 65536 * 36 values: two stage buffers exceed 8 MiB
    cfg = dict(wl["solver"])
    u = torch.zeros((65536, 4, 9, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(frsg.FrsgError) as ei:
        frsg.rk_step_noalloc(u, u, 1e-4, 1, **cfg)
    assert ei.value.status == frsg.E_INVAL


def test_noalloc_rejects_dirichlet_without_ghost_modes():
    import torch
    from paper_2112_05946_gb300 import frsg
    wl = workloads.sod_1d(nx=64)
    cfg = dict(wl["solver"])
    u = torch.zeros((64, 4, 7, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(frsg.FrsgError) as ei:
        frsg.rk_step_noalloc(u, u, 1e-4, 1, ghost_modes=None, **cfg)
    assert ei.value.status == frsg.E_INVAL
