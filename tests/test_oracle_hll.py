"""Oracle pins for the HLL interface flux (Euler setup tables of §5.3-5.4): the textbook
special cases (Rusanov flux for symmetric signal speeds, exact upwinding for supersonic
states and for linear advection, consistency), the Rankine-Hugoniot relations across both
signal speeds with the intermediate state, and the deterministic Sod tube against the exact
Riemann solution for both interface fluxes."""
import numpy as np
import pytest

import oracle
from oracle import integrate, scheme
from tests.riemann_exact import sample

G = 1.4


def _euler_states(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 2.0, n)
    v = rng.uniform(-1.5, 1.5, n)
    p = rng.uniform(0.1, 2.0, n)
    return np.stack([rho, rho * v, p / (G - 1) + 0.5 * rho * v * v], axis=-1)


def _prob(eq="euler"):
    return oracle.Problem(equation=eq, gamma=G, flux="hll", adv_speed=0.7)


def test_symmetric_speeds_give_rusanov():
    prob = _prob()
    uL, uR = _euler_states(50, 1), _euler_states(50, 2)
    a = np.maximum(scheme.wave_speed(prob, uL), scheme.wave_speed(prob, uR))
    got = scheme.hll_from_speeds(scheme.flux(prob, uL), scheme.flux(prob, uR), uL, uR, -a, a)
    np.testing.assert_allclose(got, scheme.llf(prob, uL, uR), rtol=1e-13, atol=1e-13)


def test_consistency_and_supersonic_upwinding():
    prob = _prob()
    u = _euler_states(40, 3)
    np.testing.assert_allclose(scheme.hll(prob, u, u), scheme.flux(prob, u), rtol=1e-14, atol=1e-14)
    # both states supersonic to the right: the flux is the left flux exactly (and vice versa)
    rho, v, p = 1.0, 3.0, 0.5
    uL = np.array([[rho, rho * v, p / (G - 1) + 0.5 * rho * v * v]])
    uR = np.array([[0.7, 0.7 * 2.8, 0.4 / (G - 1) + 0.5 * 0.7 * 2.8 ** 2]])
    np.testing.assert_array_equal(scheme.hll(prob, uL, uR), scheme.flux(prob, uL))
    mirror = lambda u: u * np.array([1.0, -1.0, 1.0])                           # noqa: E731
    np.testing.assert_array_equal(scheme.hll(prob, mirror(uR), mirror(uL)), scheme.flux(prob, mirror(uL)))


def test_linear_advection_is_upwind():
    prob = _prob("advection")
    rng = np.random.default_rng(4)
    uL, uR = rng.standard_normal((20, 1)), rng.standard_normal((20, 1))
    np.testing.assert_allclose(scheme.hll(prob, uL, uR), 0.7 * uL, rtol=1e-15)


def test_rankine_hugoniot_across_both_signal_speeds():
    """With the intermediate state U* = (S_R U_R - S_L U_L - (F_R - F_L)) / (S_R - S_L), the HLL
    flux satisfies F = F_L + S_L (U* - U_L) = F_R + S_R (U* - U_R) whenever S_L < 0 < S_R."""
    prob = _prob()
    uL, uR = _euler_states(200, 5), _euler_states(200, 6)
    SL, SR = scheme.signal_speeds(prob, uL, uR)
    sub = (SL < 0) & (SR > 0)
    assert np.sum(sub) > 50
    uL, uR, SL, SR = uL[sub], uR[sub], SL[sub][:, None], SR[sub][:, None]
    fL, fR = scheme.flux(prob, uL), scheme.flux(prob, uR)
    ustar = (SR * uR - SL * uL - (fR - fL)) / (SR - SL)
    F = scheme.hll(prob, uL, uR)
    np.testing.assert_allclose(F, fL + SL * (ustar - uL), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F, fR + SR * (ustar - uR), rtol=1e-12, atol=1e-12)


def test_davis_speeds_for_sod_states():
    """Sod states at rest: the estimates are -c_L and +c_L (c_L = sqrt(1.4) > c_R)."""
    prob = _prob()
    cons = lambda r, v, p: np.array([[r, r * v, p / (G - 1) + 0.5 * r * v * v]])      # noqa: E731
    SL, SR = scheme.signal_speeds(prob, cons(1.0, 0.0, 1.0), cons(0.125, 0.0, 0.1))
    assert SL[0] == pytest.approx(-np.sqrt(1.4), rel=1e-15)
    assert SR[0] == pytest.approx(np.sqrt(1.4), rel=1e-15)


@pytest.mark.parametrize("iflux", ["llf", "hll"])
def test_sod_deterministic_converges_to_exact(iflux):
    """N = 0 (one gPC mode, Q = 1): the SG scheme is the deterministic FR scheme.  Density L1
    error at t = 0.1 against the exact solution falls as the mesh is refined."""
    errs = []
    for nx in (25, 50, 100):
        prob = oracle.Problem(nx=nx, P=2, N=0, Q=1, equation="euler", gamma=G, x0=0.0, x1=1.0,
                              bc=("dirichlet", "dirichlet", "periodic", "periodic"), filter="exp", sensor=True,
                              f_alpha=36.0, f_s=4.0, s0=-3.0 * np.log10(2), kappa=4.0, limiter=True, flux=iflux)
        prob.dirichlet = {0: np.array([[1.0, 0.0, 1.0 / (G - 1)]]), 1: np.array([[0.125, 0.0, 0.1 / (G - 1)]])}
        ic = lambda x, z: np.where((x < 0.5)[..., None], [1.0, 0.0, 1.0 / (G - 1)],              # noqa: E731
                                   [0.125, 0.0, 0.1 / (G - 1)])
        u = integrate.project_initial(prob, ic)
        tabs = prob.tabs()
        t = 0.0
        while t < 0.1 - 1e-14:
            dt = min(integrate.cfl_dt(prob, tabs, u, 0.1), 0.1 - t)
            u = integrate.ssp_rk3_step(prob, tabs, u, dt)
            t += dt
        x = prob.nodes()
        ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), ((x - 0.5) / 0.1).ravel())[:, 0].reshape(x.shape)
        w = tabs["w"]
        errs.append(np.sum(0.5 * prob.dx * w[None, :] * np.abs(u[:, :, 0, 0] - ex)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.01, errs
