"""Oracle pins for the Lasso filter (§4.1.3): the L1 norms of the orthonormal Legendre
functions against closed forms and brute force, the minimiser of Theorem 1 against a
numerical minimisation of the per-coefficient optimality problem, the strength choice
(top physical and top random coefficients set to zero, mean untouched), and conservation
of the mean over a Burgers run with the filter on every element."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle
from oracle import capture, integrate


def _brute_l1(m, n=400001):
    x = np.linspace(-1.0, 1.0, n)
    c = np.zeros(m + 1)
    c[m] = 1.0
    f = np.abs(np.sqrt(2 * m + 1) * np.polynomial.legendre.legval(x, c))
    return 0.5 * np.trapezoid(f, x)


def test_l1_norms_closed_forms_and_brute_force():
    l = capture.legendre_l1_norms(9)
    assert l[0] == pytest.approx(1.0, abs=1e-15)
    assert l[1] == pytest.approx(np.sqrt(3.0) / 2.0, rel=1e-14)                    # sqrt3 * (1/2) int |x|
    assert l[2] == pytest.approx(np.sqrt(5.0) / 2.0 * 4.0 / (3.0 * np.sqrt(3.0)), rel=1e-14)
    for m in range(9):
        assert l[m] == pytest.approx(_brute_l1(m), rel=1e-7)


def _prob(P=3, N=4, S=1):
    return oracle.Problem(nx=1, P=P, N=N, Q=2 * N + 1, equation="burgers" if S == 1 else "euler",
                          x0=0.0, x1=1.0, bc=("outflow",) * 4, filter="lasso")


def test_top_coefficients_zeroed_mean_kept_and_shrinkage():
    rng = np.random.default_rng(11)
    for P, N in [(1, 2), (3, 4), (4, 8)]:
        prob = _prob(P, N)
        ut = rng.standard_normal((5, P + 1, N + 1, 1))
        out = capture.lasso_filter_modal(prob, ut)
        # zero up to the rounding of a1 (a2) times its own denominator
        assert np.all(np.abs(out[:, P, 0, 0]) <= 4e-16 * np.abs(ut[:, P, 0, 0]))
        assert np.all(np.abs(out[:, 0, N, 0]) <= 4e-16 * np.abs(ut[:, 0, N, 0]))
        np.testing.assert_array_equal(out[:, 0, 0, 0], ut[:, 0, 0, 0])
        assert np.all(np.sign(out) * np.sign(ut) >= 0)            # same sign or zero
        assert np.all(np.abs(out) <= np.abs(ut))                  # shrinks


def test_theorem1_minimiser_against_numerical_minimisation():
    """Per coefficient the filtered value must minimise 1/2 (v - u)^2 + lam |v| (the
    separable problem whose optimality condition the proof of Theorem 1 writes down), with
    lam = (a1 m(m+1) + a2 k(k+1)) ||Psi_m Phi_k||_1 and the norms taken by brute force."""
    P, N = 3, 4
    prob = _prob(P, N)
    rng = np.random.default_rng(5)
    ut = rng.standard_normal((3, P + 1, N + 1, 1)) * 0.5
    out = capture.lasso_filter_modal(prob, ut)
    lx = np.array([_brute_l1(m) for m in range(P + 1)])
    lz = np.array([_brute_l1(k) for k in range(N + 1)])
    for e in range(3):
        u = ut[e, :, :, 0]
        a1 = abs(u[P, 0]) / (P * (P + 1) * lx[P] * lz[0])
        a2 = abs(u[0, N]) / (N * (N + 1) * lx[0] * lz[N])
        for m in range(P + 1):
            for k in range(N + 1):
                lam = (a1 * m * (m + 1) + a2 * k * (k + 1)) * lx[m] * lz[k]
                f = lambda v: 0.5 * (v - u[m, k]) ** 2 + lam * abs(v)          # noqa: E731
                r = minimize_scalar(f, bounds=(-3.0, 3.0), method="bounded", options={"xatol": 1e-12})
                best = r.x if f(r.x) < f(0.0) else 0.0
                assert out[e, m, k, 0] == pytest.approx(best, abs=2e-6)


def test_lower_degree_element_untouched():
    P, N = 3, 5
    prob = _prob(P, N)
    ut = np.random.default_rng(2).standard_normal((2, P + 1, N + 1, 1))
    ut[:, P, 0, :] = 0.0
    ut[:, 0, N, :] = 0.0
    np.testing.assert_array_equal(capture.lasso_filter_modal(prob, ut), ut)


def test_lasso_per_variable_for_euler():
    prob = _prob(2, 3, S=3)
    rng = np.random.default_rng(8)
    ut = rng.standard_normal((2, 3, 4, 3))
    out = capture.lasso_filter_modal(prob, ut)
    for s in range(3):
        single = capture.lasso_filter_modal(_prob(2, 3), ut[..., s:s + 1])
        np.testing.assert_array_equal(out[..., s:s + 1], single)


def test_burgers_run_with_lasso_conserves_mean():
    prob = oracle.Problem(nx=16, P=3, N=4, Q=8, equation="burgers", x0=0.0, x1=2.0, filter="lasso",
                          sensor=False)
    u = integrate.project_initial(prob, lambda x, z: (np.sin(np.pi * x) + 0.1 * z)[..., None])
    tabs = prob.tabs()
    w = tabs["w"]
    mass0 = np.sum(w[None, :] * u[:, :, 0, 0])
    dt = 0.1 * prob.dx / 1.1
    for _ in range(60):
        u = integrate.ssp_rk3_step(prob, tabs, u, dt)
    assert np.all(np.isfinite(u))
    assert abs(np.sum(w[None, :] * u[:, :, 0, 0]) - mass0) < 1e-13 * np.sum(np.abs(w[None, :] * u[:, :, 0, 0]))
