"""FP64 cell means of the float forms: the element means of the gPC mean mode are carried in
FP64 from stage to stage and moved only by the interface fluxes' mean-mode projections, one
stored value per face, so over a periodic mesh their sum is conserved to FP64 rounding (§4.1:
the filter keeps the mean, Lambda_00 = 1; §4.3: the limiter scales about it; the residual's
mean over an element is the flux difference of its faces, Eq. 21 integrated).  The float
state's mean mode is kept within float rounding of them.

Checked: a periodic FP32 Burgers run with the detector and filter active, 1,000 steps, in
every 1D layout (the stage-wise ones and the two one-launch steps); the 2D shock-vortex on a
periodic mesh with the limiter active, FP32 and FP32_TC; and the FP64 form's means.
"""
import numpy as np
import pytest

from paper_2112_05946_gb300 import workloads
from tests.helpers import gpu_initial, solver

pytestmark = pytest.mark.gpu


def _mass(s, dx_dy):
    m = s.cell_means()               # [E, S]
    return m.sum(axis=0) * dx_dy, np.abs(m).sum(axis=0) * dx_dy


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_burgers_fp32_mean_conserved_to_fp64_rounding(variant):
    wl = workloads.burgers_1d(nx=128)
    s = solver(wl, precision="fp32")
    s.set_variant(variant)
    x, z = s.nodes()
    u0 = np.stack([(0.5 + np.sin(np.pi * x) + 0.1 * zq)[..., None] for zq in z], axis=2)
    s.set_initial_nodal(u0)
    dx = 2.0 / 128
    dt = 0.1 * dx / 1.6
    m0, scale = _mass(s, dx)
    flagged = 0
    for _ in range(10):
        s.rk_step(dt, 100, graph=True)
        flagged += int(s.decisions()[0].sum())
    s.check()
    m1, _ = _mass(s, dx)
    assert flagged > 0, "the filter should act after the shock forms (t = 1)"
    assert np.all(np.abs(m1 - m0) <= 1e-12 * scale), (m0, m1)
    # the float state's own element means follow the FP64 ones within float rounding
    u = s.get_state()
    wx, _ = s.quadrature()
    own = np.einsum("j,ejs->es", wx / 2.0, u[:, :, 0, :])
    assert np.max(np.abs(own - s.cell_means())) < 1e-6 * np.max(np.abs(own))


@pytest.mark.parametrize("precision", ["fp32", "fp32_tc"])
def test_shock_vortex_periodic_means_conserved(precision):
    wl = workloads.shock_vortex_2d(nx=32, ny=16)
    s = solver(wl, precision=precision, bc=("periodic",) * 4)
    gpu_initial(s, wl)
    cell = (2.0 / 32) * (1.0 / 16)
    m0, scale = _mass(s, cell)
    limited = 0
    for _ in range(5):
        s.limit()
        dt = s.cfl_dt(0.05)
        s.rk_step(dt, 20, graph=True)
        limited += int((s.decisions()[1] < 1.0).sum())
    s.check()
    m1, _ = _mass(s, cell)
    assert np.all(np.abs(m1 - m0) <= 1e-12 * scale), (m0, m1)


def test_fp64_cell_means_are_the_state_means():
    wl = workloads.sod_1d(nx=64)
    s = solver(wl)
    gpu_initial(s, wl)
    s.rk_step(1e-4, 3, graph=True)
    u = s.get_state()
    wx, _ = s.quadrature()
    np.testing.assert_allclose(s.cell_means(), np.einsum("j,ejs->es", wx / 2.0, u[:, :, 0, :]), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("name", ["shock_vortex", "sod"])
def test_folded_mean_updates_equal_the_mean_kernel(name):
    """With the limiter on, an SSP step leaves the FP64 mean updates of stages 0 and 1 to the
    limiter launches of stages 1 and 2; stage by stage (fr_sg_stage) each stage keeps its own
    mean launch.  Both orders do the same arithmetic: the means and the state agree bit for bit
    over 16 steps (two of them shifting the float mean mode)."""
    wl = workloads.shock_vortex_2d(nx=24, ny=12) if name == "shock_vortex" else workloads.sod_1d(nx=96)
    runs = []
    for folded in (True, False):
        s = solver(wl, precision="fp32")
        gpu_initial(s, wl)
        dt = 0.5 * s.cfl_dt(0.1)
        for _ in range(16):
            if folded:
                s.rk_step(dt, 1, graph=True)
            else:
                for st in range(3):
                    s.stage(st, dt)
        s.check()
        runs.append((s.cell_means(), s.get_state()))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
