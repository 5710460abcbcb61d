"""Pin of oracle/windows.py: a window's exactly reproduced elements equal the full-mesh run.

The claim rests on the reach of one stage (face neighbours only) and on the element-local
limiter and filter.  It is checked against the oracle's own full-mesh run on meshes small
enough to step whole, with the filter and the limiter active, windows touching every kind of
side, and one or two steps; a window with a margin one element too small must differ.
"""
import numpy as np
import pytest

from oracle import integrate, windows
from paper_2112_05946_gb300 import workloads
from tests.helpers import oracle_problem


def _perturbed(prob, u, seed):
    """Seeded high-mode noise that makes the detector flag elements and the limiter act."""
    rng = np.random.default_rng(seed)
    v = u.copy()
    v[:, :, 1:, :] += 0.02 * rng.standard_normal(v[:, :, 1:, :].shape)
    v[:, 5:, 0, 0] += 0.08 * rng.standard_normal(v[:, 5:, 0, 0].shape)
    return v


@pytest.mark.parametrize("nsteps", [1, 2])
@pytest.mark.parametrize("box", [(0, 9, 0, 8), (6, 16, 3, 12), (7, 16, 0, 12), (2, 14, 4, 12)])
def test_window_matches_full_mesh(nsteps, box):
    wl = workloads.shock_vortex_2d(nx=16, ny=12, N=2, Q=4)
    prob = oracle_problem(wl)
    u = _perturbed(prob, integrate.project_initial(prob, wl["ic"]), seed=nsteps)
    dt = integrate.cfl_dt(prob, prob.tabs(), integrate.project_initial(prob, wl["ic"]), 0.05)
    rec_full = []
    ref = integrate.run(prob, u, dt, nsteps, record=rec_full)
    assert any(f.any() for f in rec_full), "the filter should act somewhere"
    try:
        rec = []
        full, got = windows.run_window(prob, u, box, dt, nsteps, record=rec)
    except ValueError:
        pytest.skip("window too small for this many steps")
    # equal up to the rounding of the window's element size (1/12 is not a binary fraction)
    np.testing.assert_allclose(got, ref[full], rtol=1e-13, atol=1e-14)
    for f_w, f_full in zip(rec, rec_full):
        np.testing.assert_array_equal(f_w, f_full[full])


def test_margin_one_short_differs():
    wl = workloads.shock_vortex_2d(nx=16, ny=12, N=2, Q=4)
    prob = oracle_problem(wl)
    u = _perturbed(prob, integrate.project_initial(prob, wl["ic"]), seed=3)
    dt = integrate.cfl_dt(prob, prob.tabs(), integrate.project_initial(prob, wl["ic"]), 0.05)
    ref = integrate.run(prob, u, dt, 1)
    box = (4, 12, 2, 10)
    pw = windows.window_problem(prob, *box)
    out = integrate.run(pw, windows.window_state(prob, u, *box), dt, 1)
    # elements two rows from the cut (one short of the margin of three) no longer match
    ey, ex = 2 + 2, 4 + 4
    local = (ey - 2) * 8 + (ex - 4)
    assert np.max(np.abs(out[local] - ref[ey * 16 + ex])) > 1e-10
    # and at the margin they do
    ey = 2 + 3
    local = (ey - 2) * 8 + (ex - 4)
    np.testing.assert_allclose(out[local], ref[ey * 16 + ex], rtol=1e-13, atol=1e-14)
