"""Batched persistent launch (fr_sg_batch_*) over uneven Burgers problems against the same
problems advanced one context at a time, and against the oracle."""
import numpy as np
import pytest

from oracle import integrate
from paper_2112_05946_gb300 import workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu


def _members(n, e_range, precision, seed=3):
    wls = workloads.burgers_batch(n=n, seed=seed, e_range=e_range)
    out = []
    for wl in wls:
        s = solver(wl, precision=precision)
        gpu_initial(s, wl)
        out.append((wl, s))
    return out


def _dts(members):
    return np.array([wl["cfl"] * (wl["solver"]["x1"] - wl["solver"]["x0"]) / wl["solver"]["nx"] / wl["lam0"]
                     for wl, _ in members])


# FP32: a single context carries its element means in FP64 and shifts the float mean mode to
# them every 8th step; the batch members do not, so the two agree to float rounding only
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 5e-6)])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_single_contexts(precision, tol, graph):
    from paper_2112_05946_gb300 import frsg
    members = _members(24, (20, 300), precision)
    twins = _members(24, (20, 300), precision)
    dts = _dts(members)
    b = frsg.Batch([s for _, s in members])
    b.rk_step(dts, 15, graph=graph)
    for (wl, s), (_, t), dt in zip(members, twins, dts):
        t.rk_step(dt, 15, graph=False)
        s.check()
        t.check()
        assert rel_l2(s.get_state(), t.get_state()) < tol, wl["name"]
    assert b.launch_count() == 45
    info = b.info()
    assert info["tiles"] >= 24 and info["grid"] >= 1


def test_batch_matches_oracle():
    from paper_2112_05946_gb300 import frsg
    members = _members(6, (16, 64), "fp64", seed=5)
    dts = _dts(members)
    b = frsg.Batch([s for _, s in members])
    b.rk_step(dts, 20)
    for (wl, s), dt in zip(members, dts):
        prob = oracle_problem(wl)
        ref = integrate.run(prob, oracle_initial(prob, wl), dt, 20)
        s.check()
        assert rel_l2(s.get_state(), ref) < 1e-12, wl["name"]


def test_full_batch_one_step():
    """All 256 members of the batched workload (uneven 64-2048 elements, P 1-4, N 2-10)."""
    from paper_2112_05946_gb300 import frsg
    members = _members(256, (64, 2048), "fp64", seed=0)
    dts = _dts(members)
    b = frsg.Batch([s for _, s in members])
    before = [s.get_state() for _, s in members[:8]]
    b.rk_step(dts, 1)
    for i, ((wl, s), dt) in enumerate(zip(members[:8], dts)):
        t = solver(wl)
        t.set_state(before[i])
        t.rk_step(dt, 1, graph=False)
        assert rel_l2(s.get_state(), t.get_state()) < 1e-13
    for wl, s in members:
        s.check()
