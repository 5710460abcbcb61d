"""Pins for the oracle's residual and time stepping.

- brute-force collocation: with Q = M the SG residual equals Q independent deterministic
  solves, one per z_q; those are computed here by a separately written weak-form nodal
  DG code (FR with Radau correction on Gauss points is nodal DG, Huynh), so the test pins
  the z-transforms, flux, face interpolation, LLF flux, D and the correction together;
- exact Galerkin projection of the Burgers flux by triple products;
- closed-form stochastic advection, its order in x and its spectral convergence in z;
- conservation of the cell integrals of every gPC mode;
- 2D: reductions to the 1D residual and free-stream preservation.
"""
import numpy as np
import numpy.polynomial.legendre as npleg
import numpy.polynomial.polynomial as nppoly
import pytest

import oracle
from oracle import integrate, scheme, tables


# ---------------------------------------------------------------- independent DG solver

def _dg_ops(P):
    r, w = npleg.leggauss(P + 1)
    n = P + 1
    dl = np.zeros((n, n))      # dl[i, j] = ell_i'(r_j)
    lm = np.zeros(n)
    lp = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1
        c = nppoly.polyfit(r, e, P)
        dl[i] = nppoly.polyval(r, nppoly.polyder(c))
        lm[i] = nppoly.polyval(-1.0, c)
        lp[i] = nppoly.polyval(1.0, c)
    return r, w, dl, lm, lp


def _phys_flux(eq, u, gamma=1.4, a=1.0):
    if eq == "advection":
        return a * u
    if eq == "burgers":
        return 0.5 * u * u
    rho, m, E = u[..., 0], u[..., 1], u[..., 2]
    v = m / rho
    p = (gamma - 1) * (E - 0.5 * rho * v * v)
    return np.stack([m, m * v + p, (E + p) * v], -1)


def _speed(eq, u, gamma=1.4, a=1.0):
    if eq == "advection":
        return abs(a) * np.ones(u.shape[:-1])
    if eq == "burgers":
        return np.abs(u[..., 0])
    rho, m, E = u[..., 0], u[..., 1], u[..., 2]
    v = m / rho
    p = (gamma - 1) * (E - 0.5 * rho * v * v)
    return np.abs(v) + np.sqrt(gamma * p / rho)


def _dg_rhs(eq, P, dx, u, left_ghost=None, right_ghost=None):
    """Weak-form nodal DG with collocated Gauss quadrature on a uniform 1D mesh.
    u: [E, n, S] nodal values.  J w_i du_i/dt = sum_j w_j f_j ell_i'(r_j)
    - (ell_i(1) F_{e+1/2} - ell_i(-1) F_{e-1/2}).  Periodic unless ghosts given."""
    r, w, dl, lm, lp = _dg_ops(P)
    E, n, S = u.shape
    J = dx / 2
    out = np.zeros_like(u)
    for e in range(E):
        f = _phys_flux(eq, u[e])
        vol = np.zeros((n, S))
        for i in range(n):
            for j in range(n):
                vol[i] += w[j] * f[j] * dl[i, j]
        uin_L = sum(lm[j] * u[e, j] for j in range(n))
        uin_R = sum(lp[j] * u[e, j] for j in range(n))
        if e > 0:
            uout_L = sum(lp[j] * u[e - 1, j] for j in range(n))
        else:
            uout_L = left_ghost if left_ghost is not None else sum(lp[j] * u[E - 1, j] for j in range(n))
        if e < E - 1:
            uout_R = sum(lm[j] * u[e + 1, j] for j in range(n))
        else:
            uout_R = right_ghost if right_ghost is not None else sum(lm[j] * u[0, j] for j in range(n))

        def lf(a, b):
            al = max(_speed(eq, a[None])[0], _speed(eq, b[None])[0])
            return 0.5 * (_phys_flux(eq, a[None])[0] + _phys_flux(eq, b[None])[0]) - 0.5 * al * (b - a)

        FL = lf(uout_L, uin_L)
        FR = lf(uin_R, uout_R)
        for i in range(n):
            out[e, i] = (vol[i] - (lp[i] * FR - lm[i] * FL)) / (J * w[i])
    return out


def _random_smooth_state(prob, rng, base, amp):
    E, Np, M, S = prob.E, prob.Np, prob.M, prob.S
    u = amp * rng.standard_normal((E, Np, M, S)) / (1.0 + np.arange(M))[None, None, :, None] ** 2
    u[:, :, 0, :] += base
    return u


@pytest.mark.parametrize("eq,P,N", [("burgers", 1, 1), ("burgers", 2, 3), ("burgers", 3, 2),
                                    ("advection", 2, 2), ("euler", 2, 2), ("euler", 3, 1)])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_collocation_equals_pointwise_dg(eq, P, N, bc):
    M = N + 1
    prob = oracle.Problem(nx=5, P=P, N=N, Q=M, equation=eq, x0=0.0, x1=1.0)
    rng = np.random.default_rng(7)
    if eq == "euler":
        base = np.array([1.0, 0.3, 2.5])
        amp = np.array([0.05, 0.05, 0.1])
    else:
        base = np.array([0.7])
        amp = np.array([0.3])
    uh = _random_smooth_state(prob, rng, base, amp)
    gl = gr = None
    if bc == "dirichlet":
        g_left = np.zeros((M, prob.S))
        g_left[0] = base * 1.1
        g_left[min(1, N)] += 0.02
        g_right = np.zeros((M, prob.S))
        g_right[0] = base * 0.9
        prob.bc = ("dirichlet", "dirichlet", "periodic", "periodic")
        prob.dirichlet = {0: g_left, 1: g_right}
    tabs = prob.tabs()
    rsg = scheme.rhs(prob, tabs, uh)
    V = tabs["z_V"]
    for q in range(M):
        unodal = np.einsum("k,ejks->ejs", V[q], uh)
        if bc == "dirichlet":
            gl = V[q] @ prob.dirichlet[0]
            gr = V[q] @ prob.dirichlet[1]
        rdg = _dg_rhs(eq, P, prob.dx, unodal, gl, gr)
        rsg_q = np.einsum("k,ejks->ejs", V[q], rsg)
        np.testing.assert_allclose(rsg_q, rdg, rtol=0, atol=1e-11 * max(1.0, np.abs(rdg).max()))


@pytest.mark.parametrize("N", [2, 4, 8])
def test_burgers_projection_is_exact_galerkin(N):
    """For the quadratic Burgers flux and Q >= (3N+1)/2 the quadrature projection equals
    the exact Galerkin form sum_ij u_i u_j E[Phi_i Phi_j Phi_k]/2; the triple products
    come from numpy's Legendre series product, integrated exactly (only the P_0
    coefficient survives the uniform expectation)."""
    Q = int(np.ceil((3 * N + 1) / 2))
    g = tables.gpc_tables(N, Q)
    M = N + 1
    T = np.zeros((M, M, M))
    for i in range(M):
        for j in range(M):
            ci = np.zeros(i + 1)
            ci[i] = np.sqrt(2 * i + 1)
            cj = np.zeros(j + 1)
            cj[j] = np.sqrt(2 * j + 1)
            cij = npleg.legmul(ci, cj)
            for k in range(M):
                ck = np.zeros(k + 1)
                ck[k] = np.sqrt(2 * k + 1)
                T[i, j, k] = npleg.legmul(cij, ck)[0]
    rng = np.random.default_rng(N)
    for _ in range(3):
        u = rng.standard_normal(M)
        exact = 0.5 * np.einsum("i,j,ijk->k", u, u, T)
        quad = g["Pz"] @ (0.5 * (g["V"] @ u) ** 2)
        np.testing.assert_allclose(quad, exact, atol=1e-13)


# ---------------------------------------------------------------- stochastic advection

def _adv_ic(t):
    return lambda x, z: (1.0 + 0.5 * np.sin(np.pi * (x - t + 0.2 * z)))[..., None]


def _adv_error(nx, P, N, Q, t_end=0.5, cfl=0.1):
    prob = oracle.Problem(nx=nx, P=P, N=N, Q=Q, equation="advection", x0=0.0, x1=2.0)
    uh = integrate.project_initial(prob, _adv_ic(0.0))
    dt = cfl * prob.dx
    nsteps = int(round(t_end / dt))
    dt = t_end / nsteps
    u = integrate.run(prob, uh, dt, nsteps)
    ex = integrate.project_initial(prob, _adv_ic(t_end))
    return np.sqrt(np.mean((u - ex) ** 2)), prob, u


def test_advection_matches_closed_form_and_moments():
    """SG of constant-speed advection is exact mode by mode: uhat_k(x, t) = uhat_k(x - t, 0).
    Mean in closed form: E[u] = 1 + 0.5 sin(pi (x - t)) sin(0.2 pi)/(0.2 pi)."""
    err, prob, u = _adv_error(32, 2, 4, 8, t_end=2.0)
    assert err < 2e-5
    mean, var = integrate.moments(u)
    X = prob.nodes()
    b = 0.2 * np.pi
    emean = 1.0 + 0.5 * np.sin(np.pi * (X - 2.0)) * np.sin(b) / b
    th = np.pi * (X - 2.0)
    e_sin2 = 0.5 - 0.5 * np.cos(2 * th) * np.sin(2 * b) / (2 * b)
    evar = 0.25 * (e_sin2 - (np.sin(th) * np.sin(b) / b) ** 2)
    assert np.abs(mean[:, :, 0] - emean).max() < 5e-5
    assert np.abs(var[:, :, 0] - evar).max() < 5e-5


@pytest.mark.parametrize("P", [1, 2, 3])
def test_advection_order_in_x(P):
    """Observed order about P+1 (§5.1 states third and fourth order for P = 2, 3).
    The time step shrinks for P = 3 so the third-order time error stays below the
    fourth-order space error."""
    cfl = 0.1 if P < 3 else 0.02
    errs = [_adv_error(nx, P, 4, 8, cfl=cfl)[0] for nx in (8, 16, 32)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > P + 1 - 0.35, (errs, orders)


def test_advection_spectral_in_z():
    """Variance error against the closed form decays fast with the gPC degree N."""
    b = 0.2 * np.pi
    errs = []
    for N in (1, 2, 3, 4, 5):
        prob = oracle.Problem(nx=8, P=2, N=N, Q=2 * N + 2, equation="advection")
        uh = integrate.project_initial(prob, _adv_ic(0.0))
        _, var = integrate.moments(uh)
        th = np.pi * prob.nodes()
        e_sin2 = 0.5 - 0.5 * np.cos(2 * th) * np.sin(2 * b) / (2 * b)
        evar = 0.25 * (e_sin2 - (np.sin(th) * np.sin(b) / b) ** 2)
        errs.append(np.abs(var[:, :, 0] - evar).max())
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1] * 0.2), errs
    assert errs[-1] < 1e-8


# ---------------------------------------------------------------- conservation

def _cell_integrals(prob, u):
    w = prob.tabs()["w"]
    if prob.dim == 2:
        w = np.kron(w, w)
        J = 0.25 * prob.dx * prob.dy
    else:
        J = 0.5 * prob.dx
    return J * np.einsum("j,ejks->ks", w, u)


@pytest.mark.parametrize("filt", ["none", "exp", "l2"])
def test_conservation_burgers(filt):
    prob = oracle.Problem(nx=16, P=3, N=4, Q=8, equation="burgers", x0=0.0, x1=2.0,
                          filter=filt, f_alpha=36.0, f_s=4.0, s0=-2 * np.log10(3), kappa=4.0,
                          sensor=(filt == "exp"))
    uh = integrate.project_initial(prob, lambda x, z: (np.sin(np.pi * x) + 0.1 * z)[..., None])
    I0 = _cell_integrals(prob, uh)
    dt = 0.1 * prob.dx / 1.1
    rec = []
    # unfiltered: stop before the shock forms (t ~ 1/pi); filtered: run well past it
    nsteps = 20 if filt == "none" else 200
    u = integrate.run(prob, uh, dt, nsteps, record=rec)
    assert np.all(np.isfinite(u))
    I1 = _cell_integrals(prob, u)
    if filt == "none":
        np.testing.assert_allclose(I1, I0, atol=1e-13)
    else:
        np.testing.assert_allclose(I1[0], I0[0], atol=1e-13)
        assert np.any(np.concatenate(rec))


def test_conservation_euler_with_limiter_and_filter():
    prob = oracle.Problem(nx=12, P=2, N=3, Q=6, equation="euler", x0=0.0, x1=1.0,
                          filter="exp", f_alpha=36.0, f_s=4.0, s0=-3 * np.log10(2), kappa=4.0,
                          limiter=True)

    def ic(x, z):
        rho = np.where(np.abs(x - 0.5) < 0.25, 1.0 + 0.1 * z, 0.125)
        p = np.where(np.abs(x - 0.5) < 0.25, 1.0, 0.1)
        return np.stack([rho, 0 * x, p / 0.4], -1)

    uh = integrate.project_initial(prob, ic)
    I0 = _cell_integrals(prob, uh)
    tabs = prob.tabs()
    u = uh
    for _ in range(30):
        dt = integrate.cfl_dt(prob, tabs, u, 0.1)
        u = integrate.ssp_rk3_step(prob, tabs, u, dt)
    I1 = _cell_integrals(prob, u)
    np.testing.assert_allclose(I1[0], I0[0], atol=1e-13)


# ---------------------------------------------------------------- 2D

def _euler2d_prob(nx, ny, P, N):
    return oracle.Problem(dim=2, nx=nx, ny=ny, P=P, N=N, Q=2 * N, equation="euler",
                          x0=0.0, x1=1.0, y0=0.0, y1=0.5)


@pytest.mark.parametrize("direction", [0, 1])
def test_2d_reduces_to_1d(direction):
    """A 2D Euler state that varies along one axis only, with no velocity across it,
    gives the 1D Euler residual along that axis on every line of elements."""
    P, N = 2, 2
    nx, ny = (6, 3) if direction == 0 else (3, 6)
    p2 = _euler2d_prob(nx, ny, P, N)
    n = P + 1
    p1 = oracle.Problem(nx=(nx if direction == 0 else ny), P=P, N=N, Q=2 * N, equation="euler",
                        x0=0.0, x1=(1.0 if direction == 0 else 0.5))
    rng = np.random.default_rng(3)
    u1 = _random_smooth_state(p1, rng, np.array([1.0, 0.2, 2.0]), np.array([0.05, 0.05, 0.1]))
    U2 = np.zeros((ny, nx, n, n, p2.M, 4))
    for a in range(n):
        for b in range(n):
            if direction == 0:
                U2[:, :, b, a, :, 0] = u1[None, :, a, :, 0]
                U2[:, :, b, a, :, 1] = u1[None, :, a, :, 1]
                U2[:, :, b, a, :, 3] = u1[None, :, a, :, 2]
            else:
                U2[:, :, b, a, :, 0] = u1[:, None, b, :, 0]
                U2[:, :, b, a, :, 2] = u1[:, None, b, :, 1]
                U2[:, :, b, a, :, 3] = u1[:, None, b, :, 2]
    r2 = scheme.rhs(p2, p2.tabs(), U2.reshape(p2.E, p2.Np, p2.M, 4)).reshape(ny, nx, n, n, p2.M, 4)
    r1 = scheme.rhs(p1, p1.tabs(), u1)
    vel = 1 if direction == 0 else 2
    other = 2 if direction == 0 else 1
    for a in range(n):
        for b in range(n):
            ref = r1[None, :, a] if direction == 0 else r1[:, None, b]
            ref = np.broadcast_to(ref, (ny, nx) + ref.shape[2:])
            np.testing.assert_allclose(r2[:, :, b, a, :, 0], ref[..., 0], atol=1e-11)
            np.testing.assert_allclose(r2[:, :, b, a, :, vel], ref[..., 1], atol=1e-11)
            np.testing.assert_allclose(r2[:, :, b, a, :, 3], ref[..., 2], atol=1e-11)
            np.testing.assert_allclose(r2[:, :, b, a, :, other], 0.0, atol=1e-11)


def test_2d_free_stream_and_reflect_walls():
    p2 = _euler2d_prob(4, 3, 3, 2)
    U = np.zeros((p2.E, p2.Np, p2.M, 4))
    U[:, :, 0, :] = [1.2, 0.3, -0.2, 2.7]
    U[:, :, 1, 0] = 0.05            # z-dependent but x,y-uniform state
    r = scheme.rhs(p2, p2.tabs(), U)
    np.testing.assert_allclose(r, 0.0, atol=1e-12)
    # gas at rest between reflecting walls stays at rest
    p2.bc = ("reflect", "reflect", "reflect", "reflect")
    U[:, :, 0, :] = [1.2, 0.0, 0.0, 2.7]
    r = scheme.rhs(p2, p2.tabs(), U)
    np.testing.assert_allclose(r, 0.0, atol=1e-12)
