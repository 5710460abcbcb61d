"""Pins for the 2D parts of the oracle that the 1D pins do not reach.

- The L2 and exponential filter strengths on tensor-product elements (§4.1.1, Eq. 32;
  §4.1.2, Eqs. 38-39): the damping factor of each corner mode of the (m_a, m_b, k) table
  has a closed form, and the modal data are built and read back with numpy's Legendre
  evaluation, not with the oracle's Vandermonde.
- The 2D positivity limiter (§4.3, Eqs. 48-52): its point set must hold the solution
  points and all four faces, its mean is the (0, 0, 0) modal coefficient.  Each element
  below carries a defect that only one face sees, and every check evaluates the state at
  the faces with numpy's Legendre series.
- A stationary normal shock on an element face (§5.4 setup, Rankine-Hugoniot): the
  residual vanishes away from the shock, and next to it equals the closed form of the
  Lax-Friedrichs dissipation term lifted by the Radau correction (§3.3-3.5).  The
  downstream state is found here by solving the jump conditions numerically.
"""
import math

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest
from scipy.optimize import brentq

import oracle
from oracle import capture, scheme

GAMMA = 1.4


def _psi(m, x):
    """Orthonormal Legendre function sqrt(2m+1) P_m (unit norm under the uniform density)."""
    c = np.zeros(m + 1)
    c[m] = np.sqrt(2 * m + 1)
    return npleg.legval(x, c)


def _eval2d(c, r, s):
    """Series sum_{mb, ma} c[mb, ma, ...] Psi_ma(r) Psi_mb(s) at the points (r[i], s[i])."""
    n = c.shape[0]
    out = 0.0
    for mb in range(n):
        for ma in range(n):
            out = out + (_psi(ma, r) * _psi(mb, s))[(...,) + (None,) * (c.ndim - 2)] * c[mb, ma]
    return out


def _gauss_points_2d(P):
    """Solution points of a tensor element in the library order j = b (P+1) + a."""
    g, _ = npleg.leggauss(P + 1)
    a = np.tile(np.arange(P + 1), P + 1)
    b = np.repeat(np.arange(P + 1), P + 1)
    return g[a], g[b]


def _nodal_2d(c):
    """c [mb, ma, k, S] (modal in r, s and z) -> uhat [Np, k, S] (nodal in r, s)."""
    P = c.shape[0] - 1
    r, s = _gauss_points_2d(P)
    return _eval2d(c, r, s)


def _modal_2d(uh):
    """Inverse of _nodal_2d by a least-squares solve on the Gauss points."""
    n = int(round(math.sqrt(uh.shape[0])))
    r, s = _gauss_points_2d(n - 1)
    V = np.stack([_psi(ma, r) * _psi(mb, s) for mb in range(n) for ma in range(n)], 1)
    flat = np.linalg.solve(V, uh.reshape(n * n, -1))
    return flat.reshape((n, n) + uh.shape[1:])


# ---------------------------------------------------------------- filter strengths (2D)

@pytest.mark.parametrize("P,N", [(1, 3), (2, 4), (3, 4)])
@pytest.mark.parametrize("kind", ["l2", "exp"])
def test_filter_strengths_2d_corner_factors(kind, P, N):
    eps1, eps2, alpha, dt = 0.6, 1.0, 36.0, 0.01
    prob = oracle.Problem(dim=2, nx=2, ny=1, P=P, N=N, Q=2 * N, equation="euler", filter=kind,
                          f_eps1=eps1, f_eps2=eps2, f_alpha=alpha, f_s=4.0,
                          bc=("outflow",) * 4)
    rng = np.random.default_rng(31 + P)
    c = 0.5 + rng.random((P + 1, P + 1, N + 1, 4))          # no zero coefficient
    U = np.zeros((2, (P + 1) ** 2, N + 1, 4))
    U[0] = _nodal_2d(c)
    U[1] = U[0]
    out = capture.apply_filter(prob, prob.tabs(), U, dt, np.array([True, False]))
    np.testing.assert_array_equal(out[1], U[1])              # unflagged: untouched
    ratio = _modal_2d(out[0]) / c                             # [mb, ma, k, S]
    # the factor acts diagonally and the same on every variable
    np.testing.assert_allclose(ratio, ratio[..., :1] * np.ones(4), rtol=1e-11)
    if kind == "l2":
        # alpha1 P^2 (P+1)^2 = 1/eps1 and alpha2 N^2 (N+1)^2 = 1/eps2 (Eq. 39 with N_p = P+1),
        # summed over the directions in which the mode is at the top degree
        e1, e2 = 1.0 / eps1, 1.0 / eps2
        expect = {(0, 0, 0): 1.0, (0, P, 0): 1 / (1 + e1), (P, 0, 0): 1 / (1 + e1),
                  (P, P, 0): 1 / (1 + 2 * e1), (0, 0, N): 1 / (1 + e2),
                  (0, P, N): 1 / (1 + e1 + e2), (P, P, N): 1 / (1 + 2 * e1 + e2)}
    else:
        # product of one factor exp(-alpha dt eta^s) per direction, eta = 1 at the top degree
        t = math.exp(-alpha * dt)
        expect = {(0, 0, 0): 1.0, (0, P, 0): t, (P, 0, 0): t, (P, P, 0): t * t, (0, 0, N): t,
                  (0, P, N): t * t, (P, P, N): t ** 3}
    for (mb, ma, k), v in expect.items():
        np.testing.assert_allclose(ratio[mb, ma, k, 0], v, rtol=1e-11, err_msg=str((mb, ma, k)))
    # symmetric in the two physical directions, monotone in every degree, in (0, 1]
    np.testing.assert_allclose(ratio, np.swapaxes(ratio, 0, 1), rtol=1e-11)
    assert np.all(ratio > 0) and np.all(ratio <= 1 + 1e-12)
    for ax in range(3):
        assert np.all(np.diff(ratio, axis=ax) <= 1e-12)


# ---------------------------------------------------------------- limiter (2D)

def _face_points(P):
    """The four faces' points (r, s): r = -1 / +1 at every s_b, s = -1 / +1 at every r_a."""
    g, _ = npleg.leggauss(P + 1)
    one = np.ones_like(g)
    return [(-one, g), (one, g), (g, -one), (g, one)]


def _all_points(P):
    r, s = _gauss_points_2d(P)
    pts = [(r, s)] + _face_points(P)
    return np.concatenate([p[0] for p in pts]), np.concatenate([p[1] for p in pts])


def _pressure(u):
    return (GAMMA - 1.0) * (u[..., 3] - 0.5 * (u[..., 1] ** 2 + u[..., 2] ** 2) / u[..., 0])


def _values_at(c, r, s, N, Q):
    """Conserved variables at (r_i, s_i, z_q) from modal coefficients c [mb, ma, k, S]."""
    z, _ = npleg.leggauss(Q)
    Vz = np.stack([_psi(k, z) for k in range(N + 1)], 1)      # [q, k]
    modal_x = _eval2d(c, r, s)                                  # [i, k, S]
    return np.einsum("qk,iks->iqs", Vz, modal_x)


def _defect_states(P, N, rng):
    """Eight elements: a linear density or pressure profile that is admissible at every
    solution point but negative on exactly one face (r = -1, r = +1, s = -1, s = +1 in turn),
    plus small random gPC modes in z."""
    n = P + 1
    g, _ = npleg.leggauss(n)
    slope = 0.5 * (1.0 + 1.0 / g[-1])        # 1 - slope * g_max > 0 > 1 - slope
    assert 1.0 - slope * g[-1] > 0 and 1.0 - slope < 0
    out = []
    for var in ("rho", "p"):
        for face in range(4):
            c = np.zeros((n, n, N + 1, 4))
            sign = -1.0 if face in (1, 3) else 1.0           # min on the +1 face for sign -1
            lin = sign * slope / math.sqrt(3.0)              # coefficient of Psi_1 = sqrt(3) x
            if var == "rho":
                c[0, 0, 0] = [1.0, 0.0, 0.0, 2.5]
                if face < 2:
                    c[0, 1, 0, 0] = lin
                else:
                    c[1, 0, 0, 0] = lin
            else:
                c[0, 0, 0] = [1.0, 0.0, 0.0, 1.0 / (GAMMA - 1.0)]
                if face < 2:
                    c[0, 1, 0, 3] = lin / (GAMMA - 1.0)
                else:
                    c[1, 0, 0, 3] = lin / (GAMMA - 1.0)
            c[:, :, 1:, :] += 1e-3 * rng.standard_normal((n, n, N, 4)) * np.array([1, 0, 0, 1])
            out.append(c)
    # two admissible elements, untouched by the limiter
    for _ in range(2):
        c = np.zeros((n, n, N + 1, 4))
        c[0, 0, 0] = [1.0, 0.1, -0.2, 3.0]
        c[:, :, :, :] += 0.004 * rng.standard_normal((n, n, N + 1, 4))
        c[0, 0, 0] = [1.0, 0.1, -0.2, 3.0]
        out.append(c)
    return out


@pytest.mark.parametrize("P,N", [(1, 2), (2, 3), (3, 4)])
def test_limiter_2d_faces_mean_and_bound(P, N):
    Q = 2 * N
    rng = np.random.default_rng(7 + P)
    cs = _defect_states(P, N, rng)
    nx = len(cs)
    prob = oracle.Problem(dim=2, nx=nx, ny=1, P=P, N=N, Q=Q, equation="euler", limiter=True,
                          bc=("outflow",) * 4)
    tabs = prob.tabs()
    U = np.stack([_nodal_2d(c) for c in cs])
    # the defects sit on the faces only
    rs, ss = _gauss_points_2d(P)
    for e, c in enumerate(cs):
        sol = _values_at(c, rs, ss, N, Q)
        assert sol[..., 0].min() > 1e-3 and _pressure(sol).min() > 1e-3
    rec = []
    out = capture.limit(prob, tabs, U, record=rec)
    ra, sa = _all_points(P)
    eps = 1e-8
    for e, c in enumerate(cs):
        before = _values_at(c, ra, sa, N, Q)
        lo_before = min(before[..., 0].min(), _pressure(before).min())
        c_out = _modal_2d(out[e])
        after = _values_at(c_out, ra, sa, N, Q)
        lo_after = min(after[..., 0].min(), _pressure(after).min())
        # the element mean over r, s and z is the (0, 0, 0) coefficient: unchanged, and equal to
        # the oracle's mean
        np.testing.assert_allclose(c_out[0, 0, 0], c[0, 0, 0], atol=1e-13)
        np.testing.assert_allclose(capture.element_mean(prob, tabs, U[e:e + 1])[0], c[0, 0, 0], atol=1e-13)
        if lo_before >= eps:
            np.testing.assert_array_equal(out[e], U[e])
            assert rec[0][e] == 1.0
        else:
            assert rec[0][e] < 1.0, f"element {e}: face defect not seen by the limiter"
            assert lo_after >= eps * (1 - 1e-6) - 1e-13
            assert abs(lo_after - eps) < 1e-9, "the extreme point is moved exactly to eps"
    assert sum(1 for b in rec[0] if b < 1.0) == 8


# ---------------------------------------------------------------- stationary shock (P10)

def _euler_flux_x(rho, u, p):
    E = p / (GAMMA - 1.0) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, 0.0, (E + p) * u])


def _downstream_by_root(rho1, u1, p1):
    """The non-trivial state with the same x-flux as (rho1, u1, p1), v = 0: mass and
    momentum fix rho u = m and p = F - m u, and energy is a quadratic in u whose second root
    is the shock state; it is found here by bracketing away from the upstream root."""
    m = rho1 * u1
    F = rho1 * u1 * u1 + p1
    H = _euler_flux_x(rho1, u1, p1)[3]

    def energy_flux_gap(u):
        p = F - m * u
        rho = m / u
        return _euler_flux_x(rho, u, p)[3] - H

    # the other root lies between the sonic speed of the mass/momentum line and u1
    u2 = brentq(energy_flux_gap, 0.05 * u1, 0.999 * u1, xtol=1e-15, rtol=1e-15)
    return m / u2, u2, F - m * u2


def test_stationary_shock_residual_closed_form():
    P, N, Q = 3, 2, 4
    mach = 1.1
    rho1, p1 = 1.0, 1.0
    u1 = mach * math.sqrt(GAMMA * p1 / rho1)
    rho2, u2, p2 = _downstream_by_root(rho1, u1, p1)
    assert u2 < u1 and rho2 > rho1
    f1, f2 = _euler_flux_x(rho1, u1, p1), _euler_flux_x(rho2, u2, p2)
    np.testing.assert_allclose(f2, f1, rtol=1e-13, atol=1e-13)

    def cons(rho, u, p):
        return np.array([rho, rho * u, 0.0, p / (GAMMA - 1.0) + 0.5 * rho * u * u])

    wup, wdn = cons(rho1, u1, p1), cons(rho2, u2, p2)
    nx, ny = 8, 2                       # [0, 2] x [0, 1]: the face x = 0.5 separates ex = 1 and 2
    M = N + 1
    up_modes = np.zeros((M, 4))
    up_modes[0] = wup
    dn_modes = np.zeros((M, 4))
    dn_modes[0] = wdn
    prob = oracle.Problem(dim=2, nx=nx, ny=ny, x0=0.0, x1=2.0, y0=0.0, y1=1.0, P=P, N=N, Q=Q,
                          equation="euler", bc=("dirichlet", "dirichlet", "reflect", "reflect"),
                          dirichlet={0: up_modes, 1: dn_modes}, flux="llf")
    X, _ = prob.nodes()
    U = np.zeros((prob.E, prob.Np, M, 4))
    U[:, :, 0, :] = np.where((X < 0.5)[..., None], wup, wdn)
    R = scheme.rhs(prob, prob.tabs(), U).reshape(ny, nx, P + 1, P + 1, M, 4)
    # away from the shock face every element is a constant state: no residual
    far = [ex for ex in range(nx) if ex not in (1, 2)]
    assert np.max(np.abs(R[:, far])) < 1e-12
    # no z-dependence appears
    assert np.max(np.abs(R[..., 1:, :])) < 1e-12
    # next to it: the interface flux is f - alpha (w_dn - w_up) / 2 because f(w_up) = f(w_dn),
    # alpha = max(|u| + c) of the two states (pointwise, per z-node); the correction lifts the
    # jump f^I - f^D with h_R'(r_a) = ell_a(1)/w_a (left element) and h_L'(r_a) = -ell_a(-1)/w_a
    # (right element), the derivative of the Radau / DG correction at Gauss points.
    c1, c2 = math.sqrt(GAMMA * p1 / rho1), math.sqrt(GAMMA * p2 / rho2)
    alpha = max(abs(u1) + c1, abs(u2) + c2)
    jump = -0.5 * alpha * (wdn - wup)                 # f^I - f(w) on both sides of the face
    g, w = npleg.leggauss(P + 1)
    ell_p1 = np.array([np.prod([(1.0 - g[k]) / (g[a] - g[k]) for k in range(P + 1) if k != a])
                       for a in range(P + 1)])
    ell_m1 = np.array([np.prod([(-1.0 - g[k]) / (g[a] - g[k]) for k in range(P + 1) if k != a])
                       for a in range(P + 1)])
    hR, hL = ell_p1 / w, -ell_m1 / w
    invJ = 2.0 * nx / 2.0
    left = -invJ * jump[None, :] * hR[:, None]        # [a, S]
    right = -invJ * jump[None, :] * hL[:, None]
    for ey in range(ny):
        for b in range(P + 1):
            np.testing.assert_allclose(R[ey, 1, b, :, 0, :], left, rtol=1e-11, atol=1e-12)
            np.testing.assert_allclose(R[ey, 2, b, :, 0, :], right, rtol=1e-11, atol=1e-12)
