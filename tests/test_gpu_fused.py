"""Layout 3: one launch per SSP-RK3 step, each tile recomputing a three-element halo.

Per slot the kernel does the point-parallel layout's arithmetic, so its states must equal
layout 1's (FP64 to rounding, in practice bit for bit) and the oracle's (relative L2 1e-12
FP64, 1e-5 FP32), with the same filter decisions.  Cases cover short last tiles, tiles of
one and two elements (several neighbouring tiles read one tile's elements), halos that wrap
onto the tile itself, every 1D boundary kind, replayed decisions, and the benchmark size.
"""
import numpy as np
import pytest

from oracle import integrate
from paper_2112_05946_gb300 import frsg, workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-5}
SAME = {"fp64": 1e-14, "fp32": 1e-6}


def _front_state(s, seed):
    """A steep front on a smooth background: some elements are flagged, others not."""
    x = s.nodes()[0]
    rng = np.random.default_rng(seed)
    u = workloads.random_state(s.state_shape, seed=seed, base=[0.0], amp=[1e-3])
    u[:, :, 0, 0] += np.tanh((x - 1.0) / 0.03)
    u[:, :, 1, 0] += 0.1 * rng.random()
    return u


def _run(wl, variant, tile, u, dt, nsteps, precision="fp64", **over):
    s = solver(wl, precision=precision, **over)
    s.set_variant(variant)
    if tile:
        s.set_tile(tile)
    s.set_state(u)
    flags = []
    l0 = s.launch_count()
    for _ in range(nsteps):
        s.rk_step(dt, 1, graph=True)
        flags.append(s.decisions()[0])
    s.check()
    return s.launch_count() - l0, s.get_state(), np.concatenate(flags)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,tile", [(37, 1), (37, 2), (37, 3), (37, 5), (40, 8), (3, 8), (4, 2)])
def test_fused_step_matches_layout1_and_oracle(precision, nx, tile):
    wl = workloads.burgers_1d(nx=nx)
    prob = oracle_problem(wl, nx=nx)
    s0 = solver(wl, nx=nx)
    u = _front_state(s0, seed=nx + tile)
    if precision == "fp32":
        u = u.astype(np.float32).astype(np.float64)
    dt = 0.1 * prob.dx / 1.2
    nsteps = 3
    n3, got3, f3 = _run(wl, 3, tile, u, dt, nsteps, precision, nx=nx)
    # one launch per step (the float form updates its FP64 cell means inside it); the float form
    # adds, once, the anchoring of the three buffers' means
    assert n3 == (nsteps if precision == "fp64" else nsteps + 3)
    _, got1, f1 = _run(wl, 1, 0, u, dt, nsteps, precision, nx=nx)
    np.testing.assert_array_equal(f3, f1)
    assert rel_l2(got3, got1) < SAME[precision]
    ref, rec = u, []
    for _ in range(nsteps):
        ref = integrate.ssp_rk3_step(prob, prob.tabs(), ref, dt, record=rec)
    assert rel_l2(got3, ref) < TOL[precision]
    if precision == "fp64":
        np.testing.assert_array_equal(f3, np.array(rec))


@pytest.mark.parametrize("bc", [("outflow", "outflow"), ("reflect", "reflect"), ("dirichlet", "outflow"),
                                ("dirichlet", "dirichlet")])
@pytest.mark.parametrize("tile", [1, 4])
@pytest.mark.parametrize("flux", ["llf", "hll"])
def test_fused_step_boundaries(bc, tile, flux):
    """1D Euler (no limiter) with the filter at every kind of physical boundary, with either
    interface flux."""
    over = dict(nx=11, P=2, N=3, Q=6)
    wl = workloads.sod_1d(**over)
    kw = dict(bc=bc + ("periodic", "periodic"), limiter=False, flux=flux, **over)
    prob = oracle_problem(wl, **kw)
    s0 = solver(wl, **kw)
    u = workloads.random_state(s0.state_shape, seed=3 + tile, base=[1.0, 0.3, 2.5], amp=[0.05, 0.05, 0.1])
    dt = 2e-3
    _, got3, f3 = _run(wl, 3, tile, u, dt, 2, **kw)
    _, got1, f1 = _run(wl, 1, 0, u, dt, 2, **kw)
    np.testing.assert_array_equal(f3, f1)
    assert rel_l2(got3, got1) < SAME["fp64"]
    ref = u
    for _ in range(2):
        ref = integrate.ssp_rk3_step(prob, prob.tabs(), ref, dt)
    assert rel_l2(got3, ref) < TOL["fp64"]


def test_fused_step_replays_decisions_past_shock():
    """Burgers (P = 3, N = 8, Q = 16) on 64 elements past shock formation with the oracle's
    filter decisions replayed: one launch per step, the oracle's state."""
    wl = workloads.burgers_1d(nx=64)
    prob = oracle_problem(wl)
    u0 = oracle_initial(prob, wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    nsteps = 120
    rec = []
    ref = integrate.run(prob, u0, dt, nsteps, record=rec)
    s = solver(wl)
    s.set_variant(3)
    gpu_initial(s, wl)
    s.set_replay(np.array(rec, dtype=np.uint8))
    l0 = s.launch_count()
    s.rk_step(dt, nsteps, graph=True)
    s.check()
    assert s.launch_count() - l0 == nsteps
    assert rel_l2(s.get_state(), ref) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_step_full_size(precision):
    """The 1024-element Burgers workload, 50 steps: layout 3 against the oracle and layout 1,
    at the tile the autotuner would time for it."""
    wl = workloads.burgers_1d()
    prob = oracle_problem(wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    ref = integrate.run(prob, oracle_initial(prob, wl), dt, 50)
    outs = []
    for variant in (3, 1):
        s = solver(wl, precision=precision)
        s.set_variant(variant)
        gpu_initial(s, wl)
        s.rk_step(dt, 50, graph=True)
        s.check()
        outs.append(s.get_state())
        assert rel_l2(outs[-1], ref) < TOL[precision]
    assert rel_l2(outs[0], outs[1]) < SAME[precision]


def test_fused_layout_refuses_the_limiter():
    wl = workloads.sod_1d(nx=16, P=2, N=3, Q=6)
    s = solver(wl, nx=16, P=2, N=3, Q=6)
    with pytest.raises(frsg.FrsgError) as ei:
        s.set_variant(3)
    assert ei.value.status == frsg.E_UNSUPPORTED


def test_fused_layout_single_stages_run_layout1():
    """With layout 3 selected (tile 8, too large for layout 1), three single stages
    (fr_sg_stage) still make the oracle's step."""
    wl = workloads.burgers_1d(nx=24)
    prob = oracle_problem(wl, nx=24)
    s = solver(wl, nx=24)
    s.set_variant(3)
    s.set_tile(8)
    u = _front_state(s, seed=9)
    s.set_state(u)
    dt = 0.1 * prob.dx / 1.2
    for st in range(3):
        s.stage(st, dt)
    s.check()
    ref = integrate.ssp_rk3_step(prob, prob.tabs(), u, dt)
    assert rel_l2(s.get_state(), ref) < TOL["fp64"]


def test_fused_step_replays_from_a_captured_graph():
    """The launch takes nothing launch-specific from the host (the tiles' launch counters live
    on the device), so a step captured into a CUDA graph by the caller stays correct when the
    graph is replayed: ten steps equal ten steps of layout 1."""
    import torch
    wl = workloads.burgers_1d(nx=64)
    prob = oracle_problem(wl)
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    stream = torch.cuda.Stream()
    s = solver(wl, stream=stream.cuda_stream)
    s.set_variant(3)
    gpu_initial(s, wl)
    s.rk_step(dt, 1, graph=False)          # dt uploaded, counters set for this tiling
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        s.rk_step(dt, 1, graph=False)      # captured, not run
    for _ in range(9):
        g.replay()
    torch.cuda.synchronize()
    s.check()
    ref = solver(wl)
    ref.set_variant(1)
    gpu_initial(ref, wl)
    ref.rk_step(dt, 10, graph=True)
    ref.check()
    assert rel_l2(s.get_state(), ref.get_state()) < SAME["fp64"]


def test_fused_wait_runs_out_when_a_tile_is_held():
    """The neighbour wait before the final store is bounded: hold one tile's launch counter so
    that its target cannot be reached, with a short bound, and the step reports FRSG_E_TIMEOUT;
    the held tile stores nothing (its elements keep u^n) while every other tile stores the same
    new elements as an ordinary step.  The following step re-zeroes the counters and runs."""
    wl = workloads.burgers_1d(nx=256)
    s = solver(wl)
    s.set_variant(3)
    te = s.set_tile(4)
    u = _front_state(s, seed=5)
    dt = 0.1 * (2.0 / 256) / 1.2
    # reference: an ordinary step of the same layout
    s.set_state(u)
    s.rk_step(dt, 1, graph=False)
    s.check()
    ref = s.get_state()
    hold = 9                                 # elements 36 .. 39
    s.set_state(u)
    s.test_fused_wait(wait_cycles=2_000_000, hold_tile=hold)   # about 1 ms
    s.rk_step(dt, 1, graph=False)
    with pytest.raises(frsg.FrsgError) as ei:
        s.check()
    assert ei.value.status == frsg.E_TIMEOUT
    got = s.get_state()
    mine = np.zeros(256, dtype=bool)
    mine[hold * te:(hold + 1) * te] = True
    np.testing.assert_array_equal(got[mine], u[mine])
    np.testing.assert_array_equal(got[~mine], ref[~mine])
    # the counters are re-zeroed and the next step completes
    s.test_fused_wait(0, -1)
    s.set_state(u)
    s.rk_step(dt, 1, graph=False)
    s.check()
    np.testing.assert_array_equal(s.get_state(), ref)
