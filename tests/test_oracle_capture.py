"""Pins for the oracle's detector, filters, limiter and moments (§4).

Modal test data are turned into nodal data with numpy's Legendre evaluation, not with
the oracle's Vandermonde, and the expected detector values use the closed forms
sin(pi/6) = 1/2 and sin(0) = 0 of the detector formula at chosen points.
"""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest
from scipy.optimize import brentq

import oracle
from oracle import capture, integrate, scheme


def _psi(m, x):
    c = np.zeros(m + 1)
    c[m] = np.sqrt(2 * m + 1)
    return npleg.legval(x, c)


def _nodal_from_modal_1d(P, c):
    """c[m, k] (modal in r and z) -> uhat[j, k] (nodal in r, modal in z)."""
    r, _ = npleg.leggauss(P + 1)
    out = np.zeros((P + 1, c.shape[1]))
    for m in range(P + 1):
        out += _psi(m, r)[:, None] * c[m][None, :]
    return out


def _modal_from_nodal_1d(P, u):
    r, _ = npleg.leggauss(P + 1)
    V = np.stack([_psi(m, r) for m in range(P + 1)], 1)
    return np.linalg.solve(V, u)


@pytest.mark.parametrize("P,N", [(1, 2), (2, 4), (3, 8), (4, 3)])
def test_sensor_ratio_and_theta_closed_forms(P, N):
    rng = np.random.default_rng(P * 10 + N)
    c = rng.standard_normal((P + 1, N + 1))
    top = np.zeros_like(c, dtype=bool)
    top[P, :] = True
    top[:, N] = True
    Se = np.sum(c[top] ** 2) / np.sum(c ** 2)
    se = np.log10(Se)
    uh = np.zeros((5, P + 1, N + 1, 1))
    for e in range(5):
        uh[e, :, :, 0] = _nodal_from_modal_1d(P, c)
    kappa = 2.0
    # element-wise different s0 is not possible, so test the five probe points in turn
    for offset, theta_exact in [(0.0, 0.5), (kappa / 3, 0.25), (-kappa / 3, 0.75),
                                (kappa, 0.0), (-kappa, 1.0), (2 * kappa, 0.0), (-2 * kappa, 1.0)]:
        prob = oracle.Problem(nx=5, P=P, N=N, Q=2 * N, equation="burgers", filter="exp",
                              s0=se - offset, kappa=kappa)
        th = capture.sensor_theta(prob, prob.tabs(), uh)
        np.testing.assert_allclose(th, theta_exact, atol=1e-12)


def test_sensor_smooth_cases():
    prob = oracle.Problem(nx=3, P=2, N=3, Q=6, equation="burgers", filter="exp", s0=-1.0, kappa=4.0)
    uh = np.zeros((3, 3, 4, 1))
    uh[1, :, 0, 0] = 2.0          # constant: no top-mode energy -> theta = 1
    th = capture.sensor_theta(prob, prob.tabs(), uh)
    np.testing.assert_array_equal(th, [1.0, 1.0, 1.0])   # element 0, 2: zero state


def test_sensor_2d_top_modes():
    P, N = 2, 3
    rng = np.random.default_rng(5)
    c = rng.standard_normal((P + 1, P + 1, N + 1))   # [mb, ma, k]
    top = np.zeros_like(c, dtype=bool)
    top[P, :, :] = True
    top[:, P, :] = True
    top[:, :, N] = True
    Se = np.sum(c[top] ** 2) / np.sum(c ** 2)
    r, _ = npleg.leggauss(P + 1)
    uh = np.zeros((P + 1, P + 1, N + 1))
    for mb in range(P + 1):
        for ma in range(P + 1):
            uh += _psi(mb, r)[:, None, None] * _psi(ma, r)[None, :, None] * c[mb, ma][None, None, :]
    U = np.zeros((2, (P + 1) ** 2, N + 1, 4))
    U[:, :, :, 0] = uh.reshape(-1, N + 1)[None]
    prob = oracle.Problem(dim=2, nx=2, ny=1, P=P, N=N, Q=2 * N, equation="euler", filter="l2",
                          s0=np.log10(Se) - 1.0 / 3.0, kappa=1.0)
    np.testing.assert_allclose(capture.sensor_theta(prob, prob.tabs(), U), 0.25, atol=1e-12)


@pytest.mark.parametrize("kind", ["exp", "l2"])
def test_filter_acts_diagonally_on_modes(kind):
    P, N, dt = 3, 5, 0.01
    prob = oracle.Problem(nx=2, P=P, N=N, Q=10, equation="burgers", filter=kind,
                          f_alpha=36.0, f_s=4.0, f_eps1=0.6, f_eps2=0.8)
    rng = np.random.default_rng(1)
    c = rng.standard_normal((P + 1, N + 1))
    uh = np.zeros((2, P + 1, N + 1, 1))
    uh[0, :, :, 0] = _nodal_from_modal_1d(P, c)
    uh[1, :, :, 0] = _nodal_from_modal_1d(P, c)
    out = capture.apply_filter(prob, prob.tabs(), uh, dt, np.array([True, False]))
    np.testing.assert_array_equal(out[1], uh[1])           # unflagged: untouched
    cf = _modal_from_nodal_1d(P, out[0, :, :, 0])
    ratio = cf / c
    # closed-form factors at the corners of the mode table
    if kind == "exp":
        top = np.exp(-36.0 * dt)
        expect = {(0, 0): 1.0, (P, 0): top, (0, N): top, (P, N): top * top}
    else:
        expect = {(0, 0): 1.0, (P, 0): 1.0 / (1.0 + 1.0 / 0.6), (0, N): 1.0 / (1.0 + 1.0 / 0.8)}
    for (m, k), v in expect.items():
        np.testing.assert_allclose(ratio[m, k], v, rtol=1e-12)
    # every factor lies in (0, 1] and falls with the degree in each direction
    assert np.all(ratio > 0) and np.all(ratio <= 1 + 1e-13)
    assert np.all(np.diff(ratio, axis=0) <= 1e-13) and np.all(np.diff(ratio, axis=1) <= 1e-13)
    # the cell mean (modal (0, 0)) is untouched
    np.testing.assert_allclose(cf[0, 0], c[0, 0], rtol=1e-13)


# ---------------------------------------------------------------- limiter

def _euler_prob(P=2, N=3):
    return oracle.Problem(nx=4, P=P, N=N, Q=2 * N, equation="euler", limiter=True,
                          x0=0.0, x1=1.0)


def _nodal_values(prob, uh):
    tabs = prob.tabs()
    L = capture.limiter_points(prob, tabs)
    return np.einsum("lj,qk,ejks->elqs", L, tabs["z_V"], uh)


def _make_state(prob, rng, bad_density=False, bad_pressure=False):
    uh = np.zeros((prob.E, prob.Np, prob.M, prob.S))
    uh[:, :, 0, :] = [1.0, 0.2, 2.5]
    uh[:, :, 1:, :] = 0.01 * rng.standard_normal((prob.E, prob.Np, prob.M - 1, prob.S))
    if bad_density:
        uh[1, 0, 0, 0] = -0.4      # one solution point with a strongly negative density
        uh[1, 2, 0, 0] = 2.4       # keep the mean positive
    if bad_pressure:
        uh[2, 1, 0, 2] = 0.002     # energy too low -> negative pressure
        uh[2, 0, 0, 2] = 4.0
    return uh


@pytest.mark.parametrize("case", ["density", "pressure", "both"])
def test_limiter_invariants(case):
    prob = _euler_prob()
    tabs = prob.tabs()
    rng = np.random.default_rng(3)
    uh = _make_state(prob, rng, bad_density=case in ("density", "both"),
                     bad_pressure=case in ("pressure", "both"))
    before = _nodal_values(prob, uh)
    assert np.min(before[..., 0]) < 0 or np.min(scheme.pressure(before, 1.4, 1)) < 0
    rec = []
    out = capture.limit(prob, tabs, uh, record=rec)
    after = _nodal_values(prob, out)
    eps = 1e-8
    assert np.min(after[..., 0]) >= eps * (1 - 1e-6) - 1e-14
    assert np.min(scheme.pressure(after, 1.4, 1)) >= eps * (1 - 1e-6) - 1e-13
    np.testing.assert_allclose(capture.element_mean(prob, tabs, out),
                               capture.element_mean(prob, tabs, uh), atol=1e-14)
    # elements that were admissible are bit-identical
    for e in range(prob.E):
        if min(np.min(before[e, ..., 0]), np.min(scheme.pressure(before[e], 1.4, 1))) >= eps:
            np.testing.assert_array_equal(out[e], uh[e])
            assert rec[0][e] == 1.0
    # the limited elements touch the bound: the extreme point sits at eps
    limited = [e for e in range(prob.E) if rec[0][e] < 1.0]
    assert limited
    for e in limited:
        lo = min(np.min(after[e, ..., 0]), np.min(scheme.pressure(after[e], 1.4, 1)))
        assert abs(lo - eps) < 1e-9


def test_pressure_root_matches_bisection():
    prob = _euler_prob()
    rng = np.random.default_rng(11)
    for _ in range(50):
        ubar = np.array([1.0 + rng.random(), 0.5 * rng.standard_normal(), 3.0 + rng.random()])
        d = rng.standard_normal(3) * np.array([0.5, 2.0, 5.0])
        ustar = ubar + d
        eps = 1e-8
        pstar = scheme.pressure(ustar, 1.4, 1)
        if not (pstar < eps and ustar[0] > 0):
            continue

        def g(b):
            return scheme.pressure(ubar + b * (ustar - ubar), 1.4, 1) - eps

        ref = brentq(g, 0.0, 1.0, xtol=1e-15, rtol=1e-15)
        np.testing.assert_allclose(capture.pressure_root(prob, ubar, ustar, eps), ref, atol=1e-10)


def test_moments_match_quadrature_of_expansion():
    rng = np.random.default_rng(2)
    N = 5
    uh = rng.standard_normal((3, 4, N + 1, 2))
    mean, var = integrate.moments(uh)
    z, w = npleg.leggauss(40)
    w = w / 2
    vals = np.zeros((3, 4, 40, 2))
    for k in range(N + 1):
        vals += uh[:, :, k, None, :] * _psi(k, z)[None, None, :, None]
    m_ref = np.einsum("q,ejqs->ejs", w, vals)
    v_ref = np.einsum("q,ejqs->ejs", w, (vals - m_ref[:, :, None, :]) ** 2)
    np.testing.assert_allclose(mean, m_ref, atol=1e-13)
    np.testing.assert_allclose(var, v_ref, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_pressure_root_nearly_linear_case_matches_bisection(dim):
    """The segment from the mean to a point whose density alone differs (momentum and energy
    equal to the mean's up to rounding) makes the quadratic of Eq. 51 nearly linear: its
    leading coefficient is a rounding-sized number.  The root in [0, 1] must still be the
    exact one (bisection of p(beta) = eps), not the cancellation of two nearly equal terms."""
    S = 3 if dim == 1 else 4
    prob = oracle.Problem(dim=dim, nx=2, ny=1, P=2, N=2, Q=4, equation="euler", limiter=True)
    rng = np.random.default_rng(17)
    for _ in range(40):
        rho_b = 1.0 + rng.random()
        m = rng.standard_normal(S - 2) * 1.5
        E = 0.5 * np.dot(m, m) / rho_b + (0.5 + rng.random()) / (prob.gamma - 1.0)
        ubar = np.concatenate([[rho_b], m, [E]])
        ustar = ubar.copy()
        ustar[0] = 1e-8 + 1e-3 * rng.random()                 # the limited density at the point
        ustar[-1] *= 1.0 + 1e-16 * rng.standard_normal()      # rounding left in the energy
        eps = 1e-8
        if not scheme.pressure(ustar, prob.gamma, dim) < eps:
            continue

        def g(b):
            return scheme.pressure(ubar + b * (ustar - ubar), prob.gamma, dim) - eps

        ref = brentq(g, 0.0, 1.0, xtol=1e-16, rtol=1e-15)
        np.testing.assert_allclose(capture.pressure_root(prob, ubar, ustar, eps), ref, rtol=1e-12)
