"""Oracle: the FR-SG semi-discrete residual (steps a2-a7 of the stage).

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy, every step in the paper's order:
evaluate the gPC expansion at the random-space quadrature points (§2.1, Eq. 2),
pointwise flux (§3.2, Eq. 15), Galerkin projection of the flux (§2.1, Eq. 6 with the
quadrature of Eq. 5), Lagrange interpolation of solution and flux to the element faces
(§3.3), a Lax-Friedrichs or HLL interface flux (§3.3; §5 setup tables), and the total-flux derivative with the
Radau correction derivatives (§3.4, Eq. 21; multi-D tensor form §3.5, Eq. 24).

State layout (shared with the library's ABI): uhat[e, j, k, s], e = element
(2D: e = ey*nx + ex), j = solution point (2D: j = b*(P+1) + a with a along x),
k = gPC mode, s = conserved variable.
"""
from dataclasses import dataclass, field

import numpy as np

from . import tables


@dataclass
class Problem:
    """One FR-SG problem: mesh, discretisation orders, equation and capturing options."""
    dim: int = 1
    nx: int = 32
    ny: int = 1
    x0: float = 0.0
    x1: float = 2.0
    y0: float = 0.0
    y1: float = 1.0
    # boundary kinds: x-left, x-right, y-bottom, y-top; 'periodic' | 'dirichlet' | 'outflow' | 'reflect'
    bc: tuple = ("periodic", "periodic", "periodic", "periodic")
    # ghost gPC coefficients [M, S] for 'dirichlet' sides, keyed 0..3 as in bc
    dirichlet: dict = field(default_factory=dict)
    P: int = 2
    N: int = 4
    Q: int = 8
    equation: str = "advection"  # 'advection' | 'burgers' | 'euler'
    adv_speed: float = 1.0
    gamma: float = 1.4
    filter: str = "none"  # 'none' | 'exp' | 'l2' | 'lasso'
    sensor: bool = True  # filter only elements the detector flags (theta < 0.99)
    f_alpha: float = 36.0
    f_s: float = 4.0
    f_eps1: float = 0.6
    f_eps2: float = 0.6
    s0: float = 0.0
    kappa: float = 4.0
    limiter: bool = False
    flux: str = "llf"  # interface flux: 'llf' | 'hll'

    @property
    def E(self):
        return self.nx * (self.ny if self.dim == 2 else 1)

    @property
    def n1(self):
        return self.P + 1

    @property
    def Np(self):
        return self.n1 ** self.dim

    @property
    def M(self):
        return self.N + 1

    @property
    def S(self):
        if self.equation == "euler":
            return 3 if self.dim == 1 else 4
        return 1

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny

    def tabs(self):
        t = tables.fr_tables(self.P)
        t.update({"z_" + k: v for k, v in tables.gpc_tables(self.N, self.Q).items()})
        return t

    def nodes(self):
        """Physical coordinates of the solution points: [E, Np] (1D) or ([E, Np], [E, Np])."""
        r = tables.gauss_legendre(self.n1)[0]
        if self.dim == 1:
            xl = self.x0 + self.dx * np.arange(self.nx)
            return xl[:, None] + 0.5 * self.dx * (r[None, :] + 1.0)
        xl = self.x0 + self.dx * np.arange(self.nx)
        yl = self.y0 + self.dy * np.arange(self.ny)
        X = np.zeros((self.ny, self.nx, self.n1, self.n1))
        Y = np.zeros_like(X)
        for b in range(self.n1):
            for a in range(self.n1):
                X[:, :, b, a] = xl[None, :] + 0.5 * self.dx * (r[a] + 1.0)
                Y[:, :, b, a] = yl[:, None] + 0.5 * self.dy * (r[b] + 1.0)
        return X.reshape(self.E, self.Np), Y.reshape(self.E, self.Np)


# ---------------------------------------------------------------- physical fluxes

def pressure(u, gamma, dim):
    """Ideal-gas pressure p = (gamma-1)(rho E - |rho v|^2 / (2 rho)) (§5.3, §5.4)."""
    rho = u[..., 0]
    if dim == 1:
        m2 = u[..., 1] ** 2
        ener = u[..., 2]
    else:
        m2 = u[..., 1] ** 2 + u[..., 2] ** 2
        ener = u[..., 3]
    return (gamma - 1.0) * (ener - 0.5 * m2 / rho)


def flux(prob, u, direction=0):
    """Physical flux f (direction 0, x) or g (direction 1, y) at every point (§3.2, Eq. 15).

    advection: a u; Burgers: u^2/2; Euler 1D (§5.3): (rho U, rho U^2 + p, (rho E + p) U);
    Euler 2D (§5.4): f = (rho U, rho U^2 + p, rho U V, (rho E + p) U),
                     g = (rho V, rho U V, rho V^2 + p, (rho E + p) V).
    """
    if prob.equation == "advection":
        return prob.adv_speed * u
    if prob.equation == "burgers":
        return 0.5 * u * u
    rho = u[..., 0]
    p = pressure(u, prob.gamma, prob.dim)
    if prob.dim == 1:
        v = u[..., 1] / rho
        return np.stack([u[..., 1], u[..., 1] * v + p, (u[..., 2] + p) * v], axis=-1)
    vx = u[..., 1] / rho
    vy = u[..., 2] / rho
    vn = vx if direction == 0 else vy
    out = np.stack([rho * vn, u[..., 1] * vn, u[..., 2] * vn, (u[..., 3] + p) * vn], axis=-1)
    out[..., 1 + direction] += p
    return out


def wave_speed(prob, u, direction=0):
    """Spectral radius of the flux Jacobian in the given direction: |a|, |u|, |v_n| + c."""
    if prob.equation == "advection":
        return np.abs(prob.adv_speed) * np.ones(u.shape[:-1])
    if prob.equation == "burgers":
        return np.abs(u[..., 0])
    rho = u[..., 0]
    p = pressure(u, prob.gamma, prob.dim)
    c = np.sqrt(prob.gamma * p / rho)
    vn = u[..., 1 + direction] / rho
    return np.abs(vn) + c


def llf(prob, uL, uR, direction=0):
    """Local Lax-Friedrichs interface flux at each z-node (§3.3, named there; the flux of
    every advection/Burgers setup table):
        f^I = (f(uL) + f(uR))/2 - alpha (uR - uL)/2,
    alpha = max(lambda(uL), lambda(uR)) taken pointwise per quadrature node z_q."""
    alpha = np.maximum(wave_speed(prob, uL, direction), wave_speed(prob, uR, direction))
    return 0.5 * (flux(prob, uL, direction) + flux(prob, uR, direction)) - 0.5 * alpha[..., None] * (uR - uL)


def signal_speeds(prob, uL, uR, direction=0):
    """Wave-speed estimates of the HLL flux (Davis): S_L = min of the smallest characteristic
    speed of the two states, S_R = max of the largest.  Characteristic speeds: a (advection),
    u (Burgers), v_n -+ c (Euler)."""
    if prob.equation == "advection":
        lo_l = hi_l = prob.adv_speed * np.ones(uL.shape[:-1])
        lo_r = hi_r = prob.adv_speed * np.ones(uR.shape[:-1])
    elif prob.equation == "burgers":
        lo_l = hi_l = uL[..., 0]
        lo_r = hi_r = uR[..., 0]
    else:
        def speeds(u):
            rho = u[..., 0]
            c = np.sqrt(prob.gamma * pressure(u, prob.gamma, prob.dim) / rho)
            vn = u[..., 1 + direction] / rho
            return vn - c, vn + c
        lo_l, hi_l = speeds(uL)
        lo_r, hi_r = speeds(uR)
    return np.minimum(lo_l, lo_r), np.maximum(hi_l, hi_r)


def hll_from_speeds(fL, fR, uL, uR, SL, SR):
    """HLL flux for given signal speeds: the flux of the single intermediate state that
    conserves the Riemann fan between S_L and S_R; F_L when S_L >= 0, F_R when S_R <= 0,
    else (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L)."""
    SL = SL[..., None]
    SR = SR[..., None]
    with np.errstate(divide="ignore", invalid="ignore"):
        mid = (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL)
    return np.where(SL >= 0.0, fL, np.where(SR <= 0.0, fR, mid))


def hll(prob, uL, uR, direction=0):
    """HLL interface flux at each z-node (the flux of the Euler setup tables, §5.3-5.4)."""
    SL, SR = signal_speeds(prob, uL, uR, direction)
    return hll_from_speeds(flux(prob, uL, direction), flux(prob, uR, direction), uL, uR, SL, SR)


def interface_flux(prob, uL, uR, direction=0):
    """The problem's interface flux: local Lax-Friedrichs or HLL, pointwise per z-node."""
    if prob.flux == "hll":
        return hll(prob, uL, uR, direction)
    return llf(prob, uL, uR, direction)


def ghost(prob, side, interior, direction):
    """Ghost (outside) state for a boundary face, modal in z: [..., M, S]."""
    kind = prob.bc[side]
    if kind == "dirichlet":
        return np.broadcast_to(np.asarray(prob.dirichlet[side], dtype=np.float64), interior.shape).copy()
    if kind == "outflow":
        return interior.copy()
    if kind == "reflect":
        g = interior.copy()
        if prob.equation == "euler":
            g[..., 1 + direction] *= -1.0
        else:
            g *= -1.0
        return g
    raise ValueError(kind)


# ---------------------------------------------------------------- 1D residual

def rhs_1d(prob, tabs, uhat):
    """d uhat / dt for a 1D mesh, steps a2-a7 (§3.1 Eq. 12, §3.2-3.4)."""
    E, Np, M, S = uhat.shape
    J = 0.5 * prob.dx                      # J_i = (x_{i+1/2} - x_{i-1/2})/2 (§3.2)
    Vz, Pz = tabs["z_V"], tabs["z_Pz"]
    # a2: gPC expansion evaluated at z_q (Eq. 2)
    u = np.einsum("qk,ejks->ejqs", Vz, uhat)
    # a3: flux at every solution point and z_q (Eq. 15, before the 1/J)
    f = flux(prob, u)
    # a4: Galerkin projection of the flux (Eq. 6, quadrature Eq. 5), transformed by 1/J (Eq. 15)
    fhat = np.einsum("kq,ejqs->ejks", Pz, f) / J
    # a5: Lagrange interpolation of solution and discontinuous flux to r = -1, +1 (§3.3)
    uL = np.einsum("j,ejks->eks", tabs["lm"], uhat)
    uR = np.einsum("j,ejks->eks", tabs["lp"], uhat)
    fDL = np.einsum("j,ejks->eks", tabs["lm"], fhat)
    fDR = np.einsum("j,ejks->eks", tabs["lp"], fhat)
    # a6: interface states; face i separates element i-1 (left) and element i (right)
    left = np.empty((E + 1, M, S))
    right = np.empty((E + 1, M, S))
    left[1:E] = uR[0:E - 1]
    right[1:E] = uL[1:E]
    if prob.bc[0] == "periodic":
        left[0] = uR[E - 1]
        right[0] = uL[0]
        left[E] = uR[E - 1]
        right[E] = uL[0]
    else:
        right[0] = uL[0]
        left[0] = ghost(prob, 0, uL[0], 0)
        left[E] = uR[E - 1]
        right[E] = ghost(prob, 1, uR[E - 1], 0)
    fI_nodal = interface_flux(prob, np.einsum("qk,fks->fqs", Vz, left), np.einsum("qk,fks->fqs", Vz, right))
    fI = np.einsum("kq,fqs->fks", Pz, fI_nodal) / J
    fIL, fIR = fI[0:E], fI[1:E + 1]
    # a7: total flux derivative at r_j (Eq. 21), residual = -d f / dr (Eq. 12)
    dfdr = (np.einsum("jm,emks->ejks", tabs["D"], fhat)
            + (fIL - fDL)[:, None, :, :] * tabs["dhL"][None, :, None, None]
            + (fIR - fDR)[:, None, :, :] * tabs["dhR"][None, :, None, None])
    return -dfdr


# ---------------------------------------------------------------- 2D residual

def _faces_along(prob, tabs, U, Fh, direction):
    """Correction-flux contribution along one direction of the tensor-product element.

    U, Fh: [ny, nx, b, a, M, S] modal-in-z solution and transformed flux.  Returns the
    derivative of the total flux along r (direction 0) or s (direction 1), §3.5, Eq. 24
    with the 1D correction functions of §3.3 along each line of solution points.
    """
    Vz, Pz = tabs["z_V"], tabs["z_Pz"]
    J = 0.5 * (prob.dx if direction == 0 else prob.dy)
    lm, lp, D = tabs["lm"], tabs["lp"], tabs["D"]
    if direction == 0:
        uL = np.einsum("a,yxbaks->yxbks", lm, U)
        uR = np.einsum("a,yxbaks->yxbks", lp, U)
        fDL = np.einsum("a,yxbaks->yxbks", lm, Fh)
        fDR = np.einsum("a,yxbaks->yxbks", lp, Fh)
        vol = np.einsum("am,yxbmks->yxbaks", D, Fh)
    else:
        uL = np.einsum("b,yxbaks->yxaks", lm, U)
        uR = np.einsum("b,yxbaks->yxaks", lp, U)
        fDL = np.einsum("b,yxbaks->yxaks", lm, Fh)
        fDR = np.einsum("b,yxbaks->yxaks", lp, Fh)
        vol = np.einsum("bm,yxmaks->yxbaks", D, Fh)
    # move the element axis of this direction to the front: [nel, other_el, line, M, S]
    ax = 1 if direction == 0 else 0
    uL = np.moveaxis(uL, ax, 0)
    uR = np.moveaxis(uR, ax, 0)
    nel = uL.shape[0]
    left = np.empty((nel + 1,) + uL.shape[1:])
    right = np.empty_like(left)
    left[1:nel] = uR[:nel - 1]
    right[1:nel] = uL[1:]
    sides = (0, 1) if direction == 0 else (2, 3)
    if prob.bc[sides[0]] == "periodic":
        left[0] = uR[nel - 1]
        right[0] = uL[0]
        left[nel] = uR[nel - 1]
        right[nel] = uL[0]
    else:
        right[0] = uL[0]
        left[0] = ghost(prob, sides[0], uL[0], direction)
        left[nel] = uR[nel - 1]
        right[nel] = ghost(prob, sides[1], uR[nel - 1], direction)
    fI_nodal = interface_flux(prob, np.einsum("qk,...ks->...qs", Vz, left),
                              np.einsum("qk,...ks->...qs", Vz, right), direction)
    fI = np.einsum("kq,...qs->...ks", Pz, fI_nodal) / J
    fIL = np.moveaxis(fI[0:nel], 0, ax)
    fIR = np.moveaxis(fI[1:nel + 1], 0, ax)
    if direction == 0:
        return (vol + (fIL - fDL)[:, :, :, None] * tabs["dhL"][None, None, None, :, None, None]
                + (fIR - fDR)[:, :, :, None] * tabs["dhR"][None, None, None, :, None, None])
    return (vol + (fIL - fDL)[:, :, None, :] * tabs["dhL"][None, None, :, None, None, None]
            + (fIR - fDR)[:, :, None, :] * tabs["dhR"][None, None, :, None, None, None])


def rhs_2d(prob, tabs, uhat):
    """d uhat / dt on an axis-aligned uniform quad mesh (§3.5, Eqs. 23-25, with the
    minus sign of Eq. 12): -( d f^delta/dr + d g^delta/ds ), f^delta = f/J_x, g^delta = g/J_y."""
    n = prob.n1
    U = uhat.reshape(prob.ny, prob.nx, n, n, prob.M, prob.S)
    Vz, Pz = tabs["z_V"], tabs["z_Pz"]
    u = np.einsum("qk,yxbaks->yxbaqs", Vz, U)
    fh = np.einsum("kq,yxbaqs->yxbaks", Pz, flux(prob, u, 0)) / (0.5 * prob.dx)
    gh = np.einsum("kq,yxbaqs->yxbaks", Pz, flux(prob, u, 1)) / (0.5 * prob.dy)
    d = _faces_along(prob, tabs, U, fh, 0) + _faces_along(prob, tabs, U, gh, 1)
    return (-d).reshape(uhat.shape)


def rhs(prob, tabs, uhat):
    """Semi-discrete FR-SG residual for the problem's dimension."""
    return rhs_1d(prob, tabs, uhat) if prob.dim == 1 else rhs_2d(prob, tabs, uhat)
