"""Pins for the oracle's tables (quadrature, Lagrange, Radau correction, gPC, Vandermonde).

Each check compares against a library routine (numpy.polynomial), a closed form, or
an exact polynomial identity - never against a retyped copy of the oracle's formula.
"""
import numpy as np
import numpy.polynomial.legendre as npleg
import numpy.polynomial.polynomial as nppoly
import pytest

from oracle import tables


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12, 16, 17, 20, 22])
def test_gauss_legendre_matches_numpy(n):
    x, w = tables.gauss_legendre(n)
    xr, wr = npleg.leggauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, wr, rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", [0, 1, 2, 5, 9])
def test_legendre_matches_numpy(n):
    x = np.linspace(-1, 1, 37)
    c = np.zeros(n + 1)
    c[n] = 1
    p, dp = tables.legendre(n, x)
    np.testing.assert_allclose(p, npleg.legval(x, c), atol=1e-14)
    np.testing.assert_allclose(dp, npleg.legval(x, npleg.legder(c)), atol=1e-12)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_lagrange_cardinal_and_derivative_exact_on_polynomials(P):
    t = tables.fr_tables(P)
    r = t["r"]
    np.testing.assert_allclose(tables.lagrange_basis(r, r), np.eye(P + 1), atol=1e-14)
    # D differentiates every polynomial of degree <= P exactly
    rng = np.random.default_rng(P)
    for _ in range(5):
        c = rng.standard_normal(P + 1)
        vals = nppoly.polyval(r, c)
        dvals = nppoly.polyval(r, nppoly.polyder(c))
        np.testing.assert_allclose(t["D"] @ vals, dvals, atol=1e-12)
        # interpolation to the faces is exact as well
        np.testing.assert_allclose(t["lm"] @ vals, nppoly.polyval(-1.0, c), atol=1e-13)
        np.testing.assert_allclose(t["lp"] @ vals, nppoly.polyval(1.0, c), atol=1e-13)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_radau_correction_constraints_and_dg_equivalence(P):
    """h_L(-1)=1, h_L(1)=0, h_R(-1)=0, h_R(1)=1, h_L(r)=h_R(-r) (§3.3), and the FR-DG
    equivalence of the Radau correction on Gauss points (Huynh): the derivatives at
    the solution points are the DG lifting coefficients h_R'(r_j) = ell_j(1)/w_j and
    h_L'(r_j) = -ell_j(-1)/w_j."""
    hL, hR, _, _ = tables.radau_correction(P, np.array([-1.0, 1.0]))
    np.testing.assert_allclose(hL, [1.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(hR, [0.0, 1.0], atol=1e-15)
    s = np.linspace(-1, 1, 11)
    a = tables.radau_correction(P, s)
    b = tables.radau_correction(P, -s)
    np.testing.assert_allclose(a[0], b[1], atol=1e-14)
    t = tables.fr_tables(P)
    xr, wr = npleg.leggauss(P + 1)
    # Lagrange cardinal values at +-1 computed independently by a numpy fit
    for j in range(P + 1):
        e = np.zeros(P + 1)
        e[j] = 1
        c = nppoly.polyfit(xr, e, P)
        np.testing.assert_allclose(t["dhR"][j], nppoly.polyval(1.0, c) / wr[j], atol=1e-12)
        np.testing.assert_allclose(t["dhL"][j], -nppoly.polyval(-1.0, c) / wr[j], atol=1e-12)


@pytest.mark.parametrize("N,Q", [(0, 1), (1, 2), (4, 8), (6, 12), (8, 16), (10, 20), (5, 9)])
def test_gpc_orthonormality(N, Q):
    """E[Phi_j Phi_k] = delta_jk (§2.1, Eq. 3) by the discrete expectation (Eq. 5):
    mass matrix = diag of squared norms (= 1)."""
    g = tables.gpc_tables(N, Q)
    Mz = g["V"].T @ np.diag(g["wprob"]) @ g["V"]
    np.testing.assert_allclose(Mz, np.diag(g["norm2"]), atol=1e-13)
    np.testing.assert_allclose(g["wprob"].sum(), 1.0, atol=1e-15)
    # projection of the expansion recovers the coefficients
    np.testing.assert_allclose(g["Pz"] @ g["V"], np.eye(N + 1), atol=1e-13)
    # basis against numpy: Phi_k = sqrt(2k+1) P_k
    for k in range(N + 1):
        c = np.zeros(k + 1)
        c[k] = np.sqrt(2 * k + 1)
        np.testing.assert_allclose(g["V"][:, k], npleg.legval(g["z"], c), atol=1e-13)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_vandermonde_x(P):
    t = tables.fr_tables(P)
    xr, _ = npleg.leggauss(P + 1)
    for m in range(P + 1):
        c = np.zeros(m + 1)
        c[m] = np.sqrt(2 * m + 1)
        np.testing.assert_allclose(t["Vx"][:, m], npleg.legval(xr, c), atol=1e-13)
    np.testing.assert_allclose(t["Vx"] @ t["Vx_inv"], np.eye(P + 1), atol=1e-13)
    # discrete orthonormality of Psi on the Gauss points (exact for degree <= 2P+1)
    np.testing.assert_allclose(t["Vx"].T @ np.diag(t["w"] / 2) @ t["Vx"], np.eye(P + 1), atol=1e-13)
