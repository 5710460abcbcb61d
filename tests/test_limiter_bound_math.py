"""The z-bound screen of the limiter for double states (§4.3) is a lower bound.

The kernel clears an element without evaluating it at the z-nodes when lower bounds of rho and
p over all of its points and z-nodes pass the check's thresholds.  That is only sound if the
bounds never exceed the true minima.  On random gPC states (positive and near-vacuum ones, 1D
and 2D, several orders) the bound model of the GPU test, which follows the kernel's formulas, is
checked against the minima of the oracle's own point and z-node evaluation, and shown to be
tight when the higher modes vanish.
"""
import numpy as np
import pytest

from paper_2112_05946_gb300 import workloads
from tests.helpers import oracle_problem
from tests.test_gpu_limiter_bound import _bounds
from oracle import capture

SHAPES = [("2d", dict(nx=3, ny=2, P=3, N=4, Q=8)), ("2d", dict(nx=3, ny=2, P=2, N=3, Q=6)),
          ("1d", dict(nx=6, P=3, N=6, Q=12)), ("1d", dict(nx=6, P=4, N=5, Q=10))]


def _problem(dim, kw):
    wl = workloads.shock_vortex_2d(**kw) if dim == "2d" else workloads.sod_1d(**kw)
    prob = oracle_problem(wl)
    return prob, prob.tabs()


def _true_minima(prob, tabs, u):
    L = capture.limiter_points(prob, tabs)
    v = np.einsum("lj,qk,ejks->elqs", L, tabs["z_V"], u)
    rho = v[..., 0]
    m2 = np.sum(v[..., 1:-1] ** 2, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = (prob.gamma - 1.0) * (v[..., -1] - 0.5 * m2 / rho)
    return rho.reshape(prob.E, -1).min(axis=1), np.where(rho > 0, p, np.inf).reshape(prob.E, -1).min(axis=1), \
        (rho > 0).reshape(prob.E, -1).all(axis=1)


@pytest.mark.parametrize("dim,kw", SHAPES)
@pytest.mark.parametrize("amp", [1e-3, 0.05, 0.4])
def test_bounds_never_exceed_the_minima(dim, kw, amp):
    prob, tabs = _problem(dim, kw)
    rng = np.random.default_rng(int(amp * 1e4) + len(dim))
    E, Np, M, S = prob.E, prob.Np, prob.M, prob.S
    base = np.array([1.0, 0.3, -0.2, 2.5]) if S == 4 else np.array([1.0, 0.3, 2.5])
    c = np.max(np.abs(tabs["z_V"]), axis=0)
    for _ in range(5):
        u = np.zeros((E, Np, M, S))
        u[:, :, 0, :] = base * (1.0 + 0.1 * rng.standard_normal((E, Np, 1)))
        u[:, :, 1:, :] = amp * rng.standard_normal((E, Np, M - 1, S)) * base
        rb, pb = _bounds(prob, tabs, u, c)
        rmin, pmin, pos = _true_minima(prob, tabs, u)
        assert np.all(rb <= rmin + 1e-12)
        # the pressure bound is taken only where the density bound is positive
        ok = rb > 0
        assert np.all(pb[ok] <= pmin[ok] + 1e-12)


@pytest.mark.parametrize("dim,kw", SHAPES)
def test_bounds_are_exact_without_higher_modes(dim, kw):
    """With every mode above the mean zero the state is constant in z; the density bound is then
    the minimum over the points, and the pressure bound the minimum where the momentum's
    bound is the momentum itself (up to the 1e-10 rounding margin)."""
    prob, tabs = _problem(dim, kw)
    rng = np.random.default_rng(5)
    E, Np, M, S = prob.E, prob.Np, prob.M, prob.S
    base = np.array([1.0, 0.3, -0.2, 2.5]) if S == 4 else np.array([1.0, 0.3, 2.5])
    u = np.zeros((E, Np, M, S))
    u[:, :, 0, :] = base * (1.0 + 0.1 * rng.standard_normal((E, Np, 1)))
    c = np.max(np.abs(tabs["z_V"]), axis=0)
    rb, pb = _bounds(prob, tabs, u, c)
    rmin, pmin, _ = _true_minima(prob, tabs, u)
    np.testing.assert_allclose(rb, rmin, rtol=1e-8)
    np.testing.assert_allclose(pb, pmin, rtol=1e-8)
