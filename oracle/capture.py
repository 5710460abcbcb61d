"""Oracle: discontinuity capturing - detector, modal filters, positivity limiter (§4).

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy following §4 step by step.
"""
import numpy as np

from . import scheme


# ---------------------------------------------------------------- nodal <-> modal in x

def to_modal_x(prob, tabs, uhat):
    """Modal coefficients in physical and random space (§4, Eqs. 26-28).

    The nodal solution is Vx times the modal one (Vx[j, m] = Psi_m(r_j)), so the modal
    coefficients are Vx^{-1} times the nodal ones.  1D: [E, m, k, S];
    2D: [E, mb, ma, k, S] with the tensor-product basis Psi_ma(r) Psi_mb(s).
    """
    Vi = tabs["Vx_inv"]
    if prob.dim == 1:
        return np.einsum("mj,ejks->emks", Vi, uhat)
    n = prob.n1
    U = uhat.reshape(prob.E, n, n, prob.M, prob.S)
    return np.einsum("pb,ma,ebaks->epmks", Vi, Vi, U)


def to_nodal_x(prob, tabs, ut):
    """Inverse of to_modal_x."""
    V = tabs["Vx"]
    if prob.dim == 1:
        return np.einsum("jm,emks->ejks", V, ut)
    out = np.einsum("bp,am,epmks->ebaks", V, V, ut)
    return out.reshape(prob.E, prob.Np, prob.M, prob.S)


def _mode_index_grids(prob):
    """Physical mode degrees (per direction) and random mode degree, broadcastable to the
    modal array of to_modal_x without the variable axis."""
    k = np.arange(prob.M)
    if prob.dim == 1:
        m = np.arange(prob.n1)
        return (m[:, None],), k[None, :]
    m = np.arange(prob.n1)
    return (m[:, None, None], m[None, :, None]), k[None, None, :]


# ---------------------------------------------------------------- detector (§4.2)

def sensor_theta(prob, tabs, uhat):
    """Per-element detector value theta (§4.2, Eqs. 46-47).

    S_e = <u^N - u^{N-1}, u^N - u^{N-1}> / <u^N, u^N> on the first conserved variable.
    u^{N-1} is the expansion with its highest modes dropped: the modes whose physical
    degree (any direction) is P or whose gPC degree is N.  With orthonormal Psi and Phi
    the inner products are plain sums of squared modal coefficients.  s_e = log10 S_e;
    theta = 1 below s0 - kappa, 0 above s0 + kappa, (1 - sin(pi (s_e - s0)/(2 kappa)))/2
    between.  An element with <u, u> = 0 or S_e = 0 is smooth (theta = 1).
    """
    ut = to_modal_x(prob, tabs, uhat)[..., 0]
    phys, k = _mode_index_grids(prob)
    top = (k == prob.N)
    for m in phys:
        top = top | (m == prob.P)
    total = np.sum(ut ** 2, axis=tuple(range(1, ut.ndim)))
    high = np.sum(np.where(top[None], ut ** 2, 0.0), axis=tuple(range(1, ut.ndim)))
    theta = np.ones(prob.E)
    for e in range(prob.E):
        if total[e] <= 0.0 or high[e] <= 0.0:
            continue
        se = np.log10(high[e] / total[e])
        if se < prob.s0 - prob.kappa:
            theta[e] = 1.0
        elif se > prob.s0 + prob.kappa:
            theta[e] = 0.0
        else:
            theta[e] = 0.5 * (1.0 - np.sin(np.pi * (se - prob.s0) / (2.0 * prob.kappa)))
    return theta


# ---------------------------------------------------------------- filters (§4.1)

def filter_strengths(prob, dt):
    """Lambda[m..., k]: damping factor of each modal coefficient.

    'exp' (§4.1.1, Eq. 32 with N_* = 0 as in Appendix A): product over directions of
        exp(-alpha dt eta^s), eta = m/P in physical space and k/N in random space.
    'l2' (§4.1.2, Eqs. 38-39): 1 / (1 + alpha1 sum_dir m^2 (m+1)^2 + alpha2 k^2 (k+1)^2),
        alpha1 = 1/(eps1 Np^2 (Np-1)^2), alpha2 = 1/(eps2 N^2 (N+1)^2), Np = P + 1.
    """
    phys, k = _mode_index_grids(prob)
    if prob.filter == "exp":
        def sig(deg, top):
            if top == 0:
                return np.ones_like(deg, dtype=np.float64)
            return np.exp(-prob.f_alpha * dt * (deg / top) ** prob.f_s)
        lam = sig(k.astype(np.float64), prob.N)
        for m in phys:
            lam = lam * sig(m.astype(np.float64), prob.P)
        return lam
    if prob.filter == "l2":
        Np1 = prob.n1
        a1 = 1.0 / (prob.f_eps1 * Np1 ** 2 * (Np1 - 1) ** 2) if Np1 > 1 else 0.0
        a2 = 1.0 / (prob.f_eps2 * prob.N ** 2 * (prob.N + 1) ** 2) if prob.N > 0 else 0.0
        kf = k.astype(np.float64)
        den = 1.0 + a2 * kf ** 2 * (kf + 1) ** 2
        for m in phys:
            mf = m.astype(np.float64)
            den = den + a1 * mf ** 2 * (mf + 1) ** 2
        return 1.0 / den
    raise ValueError(prob.filter)


def legendre_l1_norms(n):
    """||psi_m||_1 for m < n: the L1 norm, under the uniform probability density on [-1, 1],
    of the orthonormal Legendre function psi_m = sqrt(2m+1) P_m.  Between consecutive roots of
    P_m the integrand is a plain polynomial of degree m, integrated exactly by Gauss
    quadrature on each piece."""
    from numpy.polynomial import legendre as npl
    g, w = np.polynomial.legendre.leggauss(max(n, 2))
    out = np.zeros(n)
    for m in range(n):
        c = np.zeros(m + 1)
        c[m] = 1.0
        roots = np.sort(np.real(npl.legroots(c))) if m > 0 else np.array([])
        edges = np.concatenate([[-1.0], roots, [1.0]])
        total = 0.0
        for a, b in zip(edges[:-1], edges[1:]):
            x = 0.5 * (b - a) * g + 0.5 * (a + b)
            total += 0.5 * (b - a) * np.sum(w * np.abs(npl.legval(x, c)))
        out[m] = 0.5 * np.sqrt(2 * m + 1) * total
    return out


def lasso_filter_modal(prob, ut):
    """Lasso filter (§4.1.3) on the modal coefficients ut [E, m, k, S] of 1D elements.

    Theorem 1 of §4.1.3: u*_{m,k} = ReLU(1 - (a1 m(m+1) + a2 k(k+1)) ||Psi_m Phi_k||_1 / |u_{m,k}|) u_{m,k}
    (a coefficient equal to zero stays zero).  The strengths are chosen per element and
    conserved variable so that the top physical coefficient u_{P,0} and the top random
    coefficient u_{0,N} are set to zero:
        a1 = |u_{P,0}| / (P (P+1) ||Psi_P Phi_0||_1),  a2 = |u_{0,N}| / (N (N+1) ||Psi_0 Phi_N||_1),
    (N_p - 1 = P in the paper's notation), with a2 = 0 when N = 0.  Psi and Phi are the
    orthonormal bases of the element and of the random space, so ||Psi_m Phi_k||_1 =
    ||psi_m||_1 ||psi_k||_1."""
    if prob.dim != 1:
        raise ValueError("the Lasso filter is defined here for 1D elements")
    P, N = prob.P, prob.N
    lx = legendre_l1_norms(P + 1)
    lz = legendre_l1_norms(N + 1)
    norm = lx[:, None] * lz[None, :]                                     # [m, k]
    m = np.arange(P + 1, dtype=np.float64)[:, None]
    k = np.arange(N + 1, dtype=np.float64)[None, :]
    out = np.empty_like(ut)
    for e in range(ut.shape[0]):
        for s in range(ut.shape[3]):
            u = ut[e, :, :, s]
            a1 = abs(u[P, 0]) / (P * (P + 1) * norm[P, 0])
            a2 = abs(u[0, N]) / (N * (N + 1) * norm[0, N]) if N > 0 else 0.0
            thr = (a1 * m * (m + 1) + a2 * k * (k + 1)) * norm
            with np.errstate(divide="ignore", invalid="ignore"):
                factor = np.where(u != 0.0, np.maximum(0.0, 1.0 - thr / np.abs(u)), 0.0)
            out[e, :, :, s] = factor * u
    return out


def apply_filter(prob, tabs, uhat, dt, flags):
    """Filter the flagged elements: uhat <- Vx (Lambda o (Vx^{-1} uhat)) for every
    conserved variable (§4.1, Eq. 34), or the Lasso filter on the modal coefficients
    (§4.1.3).  Unflagged elements are returned unchanged."""
    if prob.filter == "none":
        return uhat.copy()
    ut = to_modal_x(prob, tabs, uhat)
    if prob.filter == "lasso":
        filtered = to_nodal_x(prob, tabs, lasso_filter_modal(prob, ut))
        out = uhat.copy()
        out[flags] = filtered[flags]
        return out
    lam = filter_strengths(prob, dt)
    filtered = to_nodal_x(prob, tabs, ut * lam[None, ..., None])
    out = uhat.copy()
    out[flags] = filtered[flags]
    return out


def filter_decisions(prob, tabs, uhat):
    """Elements to filter: theta < 0.99 (§4.2) when the detector is on, else all."""
    if prob.filter == "none":
        return np.zeros(prob.E, dtype=bool)
    if not prob.sensor:
        return np.ones(prob.E, dtype=bool)
    return sensor_theta(prob, tabs, uhat) < 0.99


# ---------------------------------------------------------------- positivity limiter (§4.3)

def limiter_points(prob, tabs):
    """Interpolation matrix from solution-point values to the solution points followed by
    the flux points on the element faces (§4.3: minima over both point sets)."""
    n = prob.n1
    lm, lp = tabs["lm"], tabs["lp"]
    if prob.dim == 1:
        return np.vstack([np.eye(n), lm[None, :], lp[None, :]])
    rows = [np.eye(n * n)]
    I = np.eye(n)
    rows.append(np.kron(I, lm[None, :]))   # r = -1 face, one row per s_b
    rows.append(np.kron(I, lp[None, :]))   # r = +1 face
    rows.append(np.kron(lm[None, :], I))   # s = -1 face, one row per r_a
    rows.append(np.kron(lp[None, :], I))   # s = +1 face
    return np.vstack(rows)


def element_mean(prob, tabs, uhat):
    """Cell mean over r and z: sum_j (w_j / 2^d) uhat[e, j, 0, :] (Phi_0 = 1, E[Phi_k] = 0)."""
    w = tabs["w"]
    if prob.dim == 2:
        w = np.kron(w, w)
    return np.einsum("j,ejs->es", w / 2.0 ** prob.dim, uhat[:, :, 0, :])


def pressure_root(prob, ubar, ustar, eps):
    """Smallest beta in [0, 1] with p(ubar + beta (ustar - ubar)) = eps (§4.3, Eq. 51).

    rho(beta) p(beta)/(gamma-1) = rho E - |m|^2/2 is quadratic in beta along the segment;
    the equation becomes a beta^2 + b beta + c = 0 with c = rho_bar (p_bar - eps) >= 0
    and a negative value at beta = 1, so exactly one root lies in [0, 1).  The two roots are
    q/a and c/q with q = -(b + sign(b) sqrt(b^2 - 4ac))/2, which never subtracts two nearly
    equal numbers: when only the density differs along the segment, a is a rounding-sized
    number and the textbook (-b +- sqrt(b^2 - 4ac))/(2a) loses the root.
    """
    g1 = prob.gamma - 1.0
    d = ustar - ubar
    rb = ubar[0]
    rd = d[0]
    mb = ubar[1:-1]
    md = d[1:-1]
    Eb = ubar[-1]
    Ed = d[-1]
    a = g1 * (Ed * rd - 0.5 * np.dot(md, md))
    b = g1 * (Eb * rd + rb * Ed - np.dot(mb, md)) - eps * rd
    c = g1 * (Eb * rb - 0.5 * np.dot(mb, mb)) - eps * rb
    if abs(a) < 1e-300:
        return -c / b
    disc = b * b - 4.0 * a * c
    disc = max(disc, 0.0)
    sq = np.sqrt(disc)
    q = -0.5 * (b + np.copysign(sq, b))
    roots = [q / a, c / q if q != 0.0 else q / a]
    cand = [r for r in roots if 0.0 <= r <= 1.0]
    if not cand:
        # numerically at the interval end
        return min(max(min(roots, key=lambda r: min(abs(r), abs(r - 1.0))), 0.0), 1.0)
    return min(cand)


def limit(prob, tabs, uhat, record=None):
    """Positivity-preserving limiter on Euler states (§4.3, Eqs. 48-52; first line of Eq. 53).

    For each element: z-evaluate the state at solution and flux points, element mean
    ubar, eps = min(1e-8, rho_bar, p_bar); if min(rho_min, p_min) < eps, scale density
    toward its mean by beta_1, then all variables by beta_2 = min_l beta_l with beta_l the
    root of p = eps at each point where p < eps.  Both scalings are about the element
    mean with an element-constant factor, so the limited state stays a polynomial and is
    written back as the modal scaling uhat <- ubar e_0 + beta (uhat - ubar e_0).
    Raises FloatingPointError when an element mean is not admissible (rho_bar or
    p_bar not positive).
    """
    if prob.equation != "euler" or not prob.limiter:
        return uhat.copy()
    L = limiter_points(prob, tabs)
    u = np.einsum("lj,qk,ejks->elqs", L, tabs["z_V"], uhat)
    ubar = element_mean(prob, tabs, uhat)
    out = uhat.copy()
    betas = np.ones(prob.E)
    for e in range(prob.E):
        rho_bar = ubar[e, 0]
        p_bar = scheme.pressure(ubar[e], prob.gamma, prob.dim)
        if not (rho_bar > 0.0 and p_bar > 0.0):
            raise FloatingPointError(f"element {e}: mean state not admissible")
        eps = min(1e-8, rho_bar, p_bar)
        ue = u[e].reshape(-1, prob.S)
        rho = ue[:, 0]
        p = scheme.pressure(ue, prob.gamma, prob.dim)
        rho_min = rho.min()
        p_min = p.min()
        if not (min(rho_min, p_min) < eps):
            continue
        beta1 = 1.0
        if rho_bar - rho_min > 0.0:
            beta1 = min((rho_bar - eps) / (rho_bar - rho_min), 1.0)
        ustar = ue.copy()
        ustar[:, 0] = beta1 * (rho - rho_bar) + rho_bar
        pstar = scheme.pressure(ustar, prob.gamma, prob.dim)
        beta2 = 1.0
        for l in range(ustar.shape[0]):
            if pstar[l] < eps:
                beta2 = min(beta2, pressure_root(prob, ubar[e], ustar[l], eps))
        # modal form: density scaled by beta2*beta1 about rho_bar, the rest by beta2
        scale = np.full(prob.S, beta2)
        scale[0] = beta2 * beta1
        mean_part = np.zeros_like(out[e])
        mean_part[:, 0, :] = ubar[e][None, :]
        out[e] = mean_part + scale[None, None, :] * (uhat[e] - mean_part)
        betas[e] = beta2 * beta1
    if record is not None:
        record.append(betas)
    return out
