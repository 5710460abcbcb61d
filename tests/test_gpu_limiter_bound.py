"""The positivity limiter (§4.3, Eqs. 48-52) with its bound screen against the oracle.

Before the z-nodal screen the kernel bounds rho and p over all z-nodes at each point of an
element from the gPC modes (v(z_q) >= v_0 - sum_{k>0} max_q |Phi_k(z_q)| |v_k| at the solution
points, the faces' values from these through ell(+-1), and the pressure from the bounds of
rho, E and |m|), and an element whose bounds clear the screen's margins is left alone without
evaluating it at the z-nodes.  Three kinds of element side by
side, in 1D and 2D, in both precisions:
  smooth   small higher modes: the bounds clear it;
  wide     large higher modes with positive nodal values everywhere: the bounds fail, the
           z-nodal screen clears it, and the limiter must leave it untouched;
  limited  a negative nodal density at one point: the limiter scales it.
The test computes the bounds itself to show that the first two kinds take the two paths.
FP64 results equal the oracle's (beta and state to 1e-12); FP32 leaves every element the
oracle leaves untouched bit for bit, and scales the others by the oracle's beta within 1e-4
(the FP32 limiter aims 1e-5 of the element mean above eps so that the rounded state stays
admissible)."""
import numpy as np
import pytest

from oracle import capture
from paper_2112_05946_gb300 import workloads
from tests.helpers import oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu

CASES = [
    ("2d", dict(nx=8, ny=4, P=3, N=4, Q=8)),    # the shock-vortex shape
    ("2d", dict(nx=6, ny=4, P=2, N=4, Q=8)),
    ("1d", dict(nx=24, P=3, N=6, Q=12)),         # the Sod shape
    ("1d", dict(nx=18, P=2, N=5, Q=10)),
]


def _workload(dim, kw):
    return workloads.shock_vortex_2d(**kw) if dim == "2d" else workloads.sod_1d(**kw)


def _state(prob, tabs, rng):
    """Element e is smooth (e % 3 == 0), wide (1) or limited (2)."""
    E, Np, M, S = prob.E, prob.Np, prob.M, prob.S
    base = np.array([1.0, 0.2, 0.1, 2.5]) if S == 4 else np.array([1.0, 0.2, 2.5])
    V = tabs["z_V"]                                    # [Q, M]
    c = np.max(np.abs(V), axis=0)
    u = np.zeros((E, Np, M, S))
    kind = np.arange(E) % 3
    for e in range(E):
        u[e, :, 0, :] = base * (1.0 + 0.02 * rng.standard_normal((Np, 1)))
        if kind[e] == 0:
            u[e, :, 1:, :] = 1e-3 * rng.standard_normal((Np, M - 1, S)) * base
        elif kind[e] == 1:
            # every variable scaled by f(z) = 1 + 0.45 Phi_1 + 0.3 Phi_2: positive at the nodes,
            # far below zero in the bound
            u[e, :, 1, :] = 0.45 * u[e, :, 0, :]
            u[e, :, 2, :] = 0.30 * u[e, :, 0, :]
        else:
            u[e, :, 1:, :] = 1e-3 * rng.standard_normal((Np, M - 1, S)) * base
            u[e, 0, 1, 0] = 1.2 * u[e, 0, 0, 0] / c[1]
    return u, kind, c


def _bounds(prob, tabs, u, c):
    """Per element the kernel's lower bounds of rho and p over its points and all z-nodes: at a
    solution point the z-spread D = sum_{k>0} c_k |uhat_k| about the mean mode; at a face point
    the interpolated mean mode with the spread sum_a |ell_a| D_a."""
    L = capture.limiter_points(prob, tabs)
    D = np.einsum("k,ejks->ejs", c[1:], np.abs(u[:, :, 1:, :]))
    t0 = np.einsum("lj,ejs->els", L, u[:, :, 0, :])
    dd = np.einsum("lj,ejs->els", np.abs(L), D)
    hi = np.einsum("lj,ejs->els", np.abs(L), np.abs(u[:, :, 0, :]) + D)
    lo = t0 - dd - 1e-10 * hi
    up = np.abs(t0) + dd + 1e-10 * hi
    rho, en = lo[..., 0], lo[..., -1]
    m2 = np.sum(up[..., 1:-1] ** 2, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = np.where(rho > 0, (prob.gamma - 1.0) * (en - 0.5 * m2 / rho), -np.inf)
    return rho.min(axis=1), p.min(axis=1)


def _nodal_min(prob, tabs, u):
    L = capture.limiter_points(prob, tabs)
    v = np.einsum("lj,qk,ejks->elqs", L, tabs["z_V"], u)
    return v[..., 0].reshape(prob.E, -1).min(axis=1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,kw", CASES)
def test_limiter_bound_screen(dim, kw, precision):
    wl = _workload(dim, kw)
    prob = oracle_problem(wl)
    tabs = prob.tabs()
    u, kind, c = _state(prob, tabs, np.random.default_rng(11))
    if precision == "fp32":
        u = u.astype(np.float32).astype(np.float64)

    # the three kinds take the three paths
    rb, pb = _bounds(prob, tabs, u, c)
    nmin = _nodal_min(prob, tabs, u)
    assert np.all(rb[kind == 0] > 0.5) and np.all(pb[kind == 0] > 0.3)
    assert np.all(rb[kind == 1] < 0) and np.all(nmin[kind == 1] > 0.05)
    assert np.all(nmin[kind == 2] < 0)

    s = solver(wl, precision=precision)
    s.set_state(u)
    s.limit()
    s.check()
    _, beta = s.decisions()
    got = s.get_state()
    rec = []
    ref = capture.limit(prob, tabs, u, record=rec)
    bref = np.asarray(rec[0])
    assert np.all(bref[kind < 2] == 1.0) and np.all(bref[kind == 2] < 1.0)
    if precision == "fp64":
        np.testing.assert_allclose(beta[0], bref, rtol=1e-12)
        assert rel_l2(got, ref) < 1e-12
    else:
        keep = bref == 1.0
        assert np.all(beta[0][keep] == 1.0)
        np.testing.assert_array_equal(got[keep], u[keep])
        np.testing.assert_allclose(beta[0][~keep], bref[~keep], rtol=1e-4)
        assert rel_l2(got[~keep], ref[~keep]) < 1e-4
