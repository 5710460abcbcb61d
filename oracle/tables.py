"""Oracle tables: quadrature, Lagrange basis, Radau correction, gPC basis, Vandermonde.

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy; slow on purpose, written so that each
function can be checked against the paper by eye.  The GPU library builds its own
tables in its own code; nothing here is shared with it.

Paper: Xiao, Kusch, Koellermeier, Frank, "A flux reconstruction stochastic Galerkin
scheme for hyperbolic conservation laws" (arXiv 2112.05946).
"""
import numpy as np


def legendre(n, x):
    """Legendre polynomial P_n(x) and its derivative P_n'(x).

    Three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and the
    derivative identity P'_{k+1} = P'_{k-1} + (2k+1) P_k.
    """
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    dp_prev = np.zeros_like(x)
    if n == 0:
        return p_prev, dp_prev
    p = x.copy()
    dp = np.ones_like(x)
    for k in range(1, n):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        dp_next = dp_prev + (2 * k + 1) * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def gauss_legendre(n):
    """n-point Gauss-Legendre nodes (ascending) and weights on [-1, 1].

    Newton iteration on P_n from the classical cosine initial guesses; the
    weights are w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).  Used for the solution
    points in r ("Points: Legendre", tables of §5) and for the random-space
    quadrature of §2.1, Eq. (5).
    """
    if n < 1:
        raise ValueError("need at least one point")
    i = np.arange(1, n + 1, dtype=np.float64)
    x = np.cos(np.pi * (i - 0.25) / (n + 0.5))
    for _ in range(100):
        p, dp = legendre(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def lagrange_basis(nodes, r):
    """ell_j(r) = prod_{k != j} (r - r_k) / (r_j - r_k)  (§3.2, Eq. 13).

    Returns an array of shape [len(r), len(nodes)].
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(r), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                out[:, j] *= (r - nodes[k]) / (nodes[j] - nodes[k])
    return out


def lagrange_derivative_matrix(nodes):
    """D[j, m] = d ell_m / dr evaluated at r_j (the ell'_k(r_j) of §3.4, Eq. 21).

    Product rule on the Lagrange product:
    ell_m'(r) = sum_{l != m} 1/(r_m - r_l) prod_{i != m, l} (r - r_i)/(r_m - r_i).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    D = np.zeros((n, n))
    for j in range(n):
        r = nodes[j]
        for m in range(n):
            total = 0.0
            for l in range(n):
                if l == m:
                    continue
                term = 1.0 / (nodes[m] - nodes[l])
                for i in range(n):
                    if i != m and i != l:
                        term *= (r - nodes[i]) / (nodes[m] - nodes[i])
                total += term
            D[j, m] = total
    return D


def radau_correction(P, r):
    """Radau ("DG") correction functions of degree P+1 and their derivatives at r.

    §3.3, Eq. 18 requires h_L(r) = h_R(-r), h_L(-1) = 1, h_L(1) = 0, h_R(-1) = 0,
    h_R(1) = 1; the right Radau polynomial of degree P+1 meets them:
        h_L(r) = ((-1)^(P+1) / 2) (L_{P+1}(r) - L_P(r)),
        h_R(r) = (1/2) (L_{P+1}(r) + L_P(r)).
    Returns (hL, hR, dhL, dhR), each shaped like r.
    """
    r = np.asarray(r, dtype=np.float64)
    a, da = legendre(P + 1, r)
    b, db = legendre(P, r)
    sgn = (-1.0) ** (P + 1)
    hL = 0.5 * sgn * (a - b)
    hR = 0.5 * (a + b)
    dhL = 0.5 * sgn * (da - db)
    dhR = 0.5 * (da + db)
    return hL, hR, dhL, dhR


def orthonormal_legendre(n, x):
    """Phi_n(x) = sqrt(2n+1) P_n(x): orthonormal w.r.t. the uniform density 1/2 on
    [-1, 1], so E[Phi_j Phi_k] = delta_jk (§2.1, Eq. 3)."""
    p, _ = legendre(n, x)
    return np.sqrt(2.0 * n + 1.0) * p


def gpc_tables(N, Q):
    """Random-space tables for z ~ U(-1, 1) with Legendre gPC of degree N and
    Q Gauss points (§2.1, Eqs. 2-5).

    Returns dict with
      z[q], wprob[q]        nodes and probability weights (sum to 1),
      V[q, k] = Phi_k(z_q)  modal -> nodal evaluation (Eq. 2),
      Pz[k, q] = wprob_q Phi_k(z_q) / <Phi_k^2>   Galerkin projection (Eq. 6 with Eq. 5),
      norm2[k] = <Phi_k^2>  (= 1 for the orthonormal basis).
    """
    M = N + 1
    z, w = gauss_legendre(Q)
    wprob = 0.5 * w
    V = np.zeros((Q, M))
    for k in range(M):
        V[:, k] = orthonormal_legendre(k, z)
    norm2 = np.ones(M)
    Pz = (V * wprob[:, None]).T / norm2[:, None]
    return dict(z=z, wprob=wprob, V=V, Pz=Pz, norm2=norm2)


def fr_tables(P):
    """Physical-space FR tables for degree P on P+1 Gauss-Legendre solution points.

    r[j], w[j]                  solution points and quadrature weights,
    D[j, m] = ell_m'(r_j)       (§3.4, Eq. 21),
    lm[j] = ell_j(-1), lp[j] = ell_j(+1)   interpolation to the element faces (§3.3),
    dhL[j] = h_L'(r_j), dhR[j] = h_R'(r_j) (§3.3-3.4, Radau correction),
    Vx[j, m] = Psi_m(r_j) with Psi orthonormal Legendre  (§4, Eq. 28; nodal = Vx @ modal),
    Vx_inv = inverse of Vx.
    """
    n = P + 1
    r, w = gauss_legendre(n)
    D = lagrange_derivative_matrix(r)
    lm = lagrange_basis(r, [-1.0])[0]
    lp = lagrange_basis(r, [1.0])[0]
    _, _, dhL, dhR = radau_correction(P, r)
    Vx = np.zeros((n, n))
    for m in range(n):
        Vx[:, m] = orthonormal_legendre(m, r)
    Vx_inv = np.linalg.inv(Vx)
    return dict(r=r, w=w, D=D, lm=lm, lp=lp, dhL=dhL, dhR=dhR, Vx=Vx, Vx_inv=Vx_inv)
