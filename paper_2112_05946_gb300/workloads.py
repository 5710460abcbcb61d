"""Seeded synthetic workloads: the problem definitions both the CUDA path and the
oracle are run on.

This module holds problem data only - mesh, orders, equation and capturing
parameters, initial and boundary data as functions of (x, z) or (x, y, z), and seeded
random coefficient generators.  It contains none of the scheme's arithmetic: each
side evaluates these functions at its own nodes and projects them itself.

The five workloads follow the paper's experiment families (§5.1 advection, §5.2
Burgers, §5.3 Sod, §5.4 shock-vortex) at the sizes of the benchmark configurations.
"""
import math

import numpy as np

GAMMA = 1.4


def advection_1d():
    """u_t + u_x = 0 on periodic [0, 2], u0 = 1 + 0.5 sin(pi (x + 0.2 z)), z ~ U(-1, 1);
    P = 2, 32 elements, N = 4, Q = 8, LLF, CFL 0.1, t_end = 2."""
    return dict(
        name="advection_E32_P2_N4_Q8",
        solver=dict(dim=1, nx=32, x0=0.0, x1=2.0, bc=("periodic",) * 4, P=2, N=4, Q=8,
                    equation="advection", adv_speed=1.0, filter="none"),
        ic=lambda x, z: (1.0 + 0.5 * np.sin(np.pi * (x + 0.2 * z)))[..., None],
        exact=lambda t: (lambda x, z: (1.0 + 0.5 * np.sin(np.pi * (x - t + 0.2 * z)))[..., None]),
        cfl=0.1, t_end=2.0, lam0=1.0,
    )


def burgers_1d(nx=1024, P=3, N=8, Q=16):
    """u_t + (u^2/2)_x = 0 on periodic [0, 2], u0 = sin(pi x) + 0.1 z; P = 3, 1024 elements,
    N = 8, Q = 16, detector + exponential filter (alpha = 36, order 4) in x and z,
    s0 = -2 log10(P) (§5.2 table with N_p - 1 = P), kappa = 4, t_end = 1."""
    return dict(
        name=f"burgers_E{nx}_P{P}_N{N}_Q{Q}",
        solver=dict(dim=1, nx=nx, x0=0.0, x1=2.0, bc=("periodic",) * 4, P=P, N=N, Q=Q,
                    equation="burgers", filter="exp", sensor=True, f_alpha=36.0, f_s=4.0,
                    s0=-2.0 * math.log10(P), kappa=4.0),
        ic=lambda x, z: (np.sin(np.pi * x) + 0.1 * z)[..., None],
        cfl=0.1, t_end=1.0, lam0=1.1,
    )


def _sod_state(x, z, left):
    rho = (1.0 + 0.1 * z) * np.ones_like(x) if left else 0.125 * np.ones_like(x)
    p = (1.0 if left else 0.1) * np.ones_like(x)
    return np.stack([rho, 0.0 * x, p / (GAMMA - 1.0)], axis=-1)


def sod_1d(nx=4096, P=3, N=6, Q=12):
    """Stochastic Sod tube (§5.3, first case): x in [0, 1], rho_L = 1 + 0.1 z, u = 0,
    p_L = 1; rho_R = 0.125, p_R = 0.1; interface at 0.5; Dirichlet ends holding the
    initial states; P = 3, 4096 elements, N = 6, Q = 12; detector + exponential filter
    (alpha = 36, order 4, s0 = -3 log10 P, kappa = 4) and the positivity limiter; t_end = 0.2."""
    def ic(x, z):
        left = _sod_state(x, z, True)
        right = _sod_state(x, z, False)
        return np.where((x < 0.5)[..., None], left, right)

    return dict(
        name=f"sod_E{nx}_P{P}_N{N}_Q{Q}",
        solver=dict(dim=1, nx=nx, x0=0.0, x1=1.0, bc=("dirichlet", "dirichlet", "periodic", "periodic"),
                    P=P, N=N, Q=Q, equation="euler", gamma=GAMMA, filter="exp", sensor=True,
                    f_alpha=36.0, f_s=4.0, s0=-3.0 * math.log10(P), kappa=4.0, limiter=True),
        ic=ic,
        boundary={0: lambda z: _sod_state(np.zeros(1), z, True)[0],
                  1: lambda z: _sod_state(np.zeros(1), z, False)[0]},
        cfl=0.1, t_end=0.2, lam0=None,
    )


def sod_location_1d(nx=100, P=2, N=9, Q=17, sigma=0.05, filter="lasso"):
    """Sod tube with a stochastic discontinuity location (§5.3, second case, setup table of
    §5.3): rho/u/p = (1, 0, 1) left of x_c = 0.5 + sigma z and (0.125, 0, 0.1) right of it,
    sigma = 0.05; x in [0, 1], 100 elements, N_p = 3 (P = 2), N_c = 9, N_q = 17, HLL flux,
    Dirichlet ends, CFL 0.1, t_end = 0.15; the Lasso filter on every element (or the L2 filter,
    eps1 = 0.6, eps2 = 0.6, behind the detector with s0 = -3 log10(N_p - 1), kappa = 4) and
    the positivity limiter.  SSP-RK3 replaces the paper's Bogacki-Shampine integrator."""
    left = np.array([1.0, 0.0, 1.0 / (GAMMA - 1.0)])
    right = np.array([0.125, 0.0, 0.1 / (GAMMA - 1.0)])

    def ic(x, z):
        return np.where((x < 0.5 + sigma * z)[..., None], left, right)

    solver = dict(dim=1, nx=nx, x0=0.0, x1=1.0, bc=("dirichlet", "dirichlet", "periodic", "periodic"),
                  P=P, N=N, Q=Q, equation="euler", gamma=GAMMA, flux="hll", limiter=True,
                  s0=-3.0 * math.log10(P), kappa=4.0)
    if filter == "lasso":
        solver.update(filter="lasso", sensor=False)
    else:
        solver.update(filter="l2", sensor=True, f_eps1=0.6, f_eps2=0.6)
    return dict(
        name=f"sod_location_E{nx}_P{P}_N{N}_Q{Q}_{filter}",
        solver=solver,
        ic=ic,
        boundary={0: lambda z: left.copy(), 1: lambda z: right.copy()},
        cfl=0.1, t_end=0.15, lam0=None,
    )


def _rh_downstream(ma, rho1=1.0, p1=1.0):
    """Normal-shock jump for upstream Mach number ma (stationary shock, ideal gas)."""
    g = GAMMA
    c1 = math.sqrt(g * p1 / rho1)
    u1 = ma * c1
    rho2 = rho1 * (g + 1.0) * ma * ma / ((g - 1.0) * ma * ma + 2.0)
    p2 = p1 * (1.0 + 2.0 * g / (g + 1.0) * (ma * ma - 1.0))
    u2 = u1 * rho1 / rho2
    return (rho1, u1, p1), (rho2, u2, p2)


def shock_vortex_2d(nx=256, ny=128, P=3, N=4, Q=8, mach=1.1):
    """Stochastic shock-vortex interaction (§5.4 family): [0, 2] x [0, 1], stationary
    normal shock of upstream Mach 1.1 at x = 0.5 (upstream rho = 1, p = 1, T = p/rho;
    downstream from the Rankine-Hugoniot jump), isentropic vortex at (0.25, 0.5), r_c = 0.05,
    mu = 0.204, strength 0.3 (1 + 0.2 z) added on both sides (§5.4 perturbation with
    delta S = 0); Dirichlet inflow / outflow states in x, reflecting walls in y.  Tensor
    FR with P = 3, 256 x 128 elements, N = 4, Q = 8; detector + L2 filter (eps1 = 0.6,
    eps2 = 1, s0 = -3 log10 2 as in the §5.4 table, kappa = 4)."""
    up, down = _rh_downstream(mach)
    g = GAMMA
    xs, xc, yc, rc, mu = 0.5, 0.25, 0.5, 0.05, 0.204

    def prim_to_cons(rho, u, v, p):
        return np.stack([rho, rho * u, rho * v, p / (g - 1.0) + 0.5 * rho * (u * u + v * v)], axis=-1)

    def ic(x, y, z):
        left = x < xs
        rho_b = np.where(left, up[0], down[0])
        u_b = np.where(left, up[1], down[1])
        p_b = np.where(left, up[2], down[2])
        T_b = p_b / rho_b
        zeta = 0.3 * (1.0 + 0.2 * z)
        dx, dy = x - xc, y - yc
        r = np.sqrt(dx * dx + dy * dy)
        eta = r / rc
        amp = zeta * eta * np.exp(mu * (1.0 - eta * eta))
        # (sin theta, -cos theta) with theta the polar angle about the vortex centre
        sin_t = np.where(r > 0, dy / np.where(r > 0, r, 1.0), 0.0)
        cos_t = np.where(r > 0, dx / np.where(r > 0, r, 1.0), 0.0)
        du, dv = amp * sin_t, -amp * cos_t
        dT = -(g - 1.0) * zeta * zeta / (4.0 * mu * g) * np.exp(2.0 * mu * (1.0 - eta * eta))
        T = T_b + dT
        rho = rho_b * (T / T_b) ** (1.0 / (g - 1.0))
        return prim_to_cons(rho, u_b + du, 0.0 * x + dv, rho * T)

    def state(prim):
        return lambda z: prim_to_cons(np.array(prim[0]), np.array(prim[1]), np.array(0.0), np.array(prim[2]))

    return dict(
        name=f"shock_vortex_{nx}x{ny}_P{P}_N{N}_Q{Q}",
        solver=dict(dim=2, nx=nx, ny=ny, x0=0.0, x1=2.0, y0=0.0, y1=1.0,
                    bc=("dirichlet", "dirichlet", "reflect", "reflect"), P=P, N=N, Q=Q, equation="euler",
                    gamma=GAMMA, filter="l2", sensor=True, f_eps1=0.6, f_eps2=1.0,
                    s0=-3.0 * math.log10(2.0), kappa=4.0, limiter=True),
        ic=ic,
        boundary={0: state(up), 1: state(down)},
        cfl=0.1, t_end=1.0, lam0=None,
    )


def splitmix64(state):
    """One step of the SplitMix64 generator: returns (next_state, 64-bit output)."""
    mask = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & mask
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return state, z ^ (z >> 31)


class _Stream:
    def __init__(self, seed):
        self.state = seed & ((1 << 64) - 1)

    def uniform(self):
        self.state, z = splitmix64(self.state)
        return (z >> 11) * (1.0 / (1 << 53))

    def integer(self, lo, hi):
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


def burgers_batch(n=256, seed=0, e_range=(64, 2048), cfl=0.05):
    """Uneven batch of stochastic Burgers problems on periodic [0, 2] (§5.2 family).

    Instance i draws from SplitMix64 seeded with seed * 1000003 + i: E ~ U{64..2048},
    P ~ U{1..4}, N ~ U{2..10}, Q = 2N; half of the instances start from
    A sin(2 pi m x / L + phi) + 0.1 z (A in [0.5, 1], m in {1, 2, 3}, phi in [0, 2 pi)),
    the other half from A exp(-(x - x0)^2 / (2 w^2)) (1 + 0.1 z) (w in [0.05, 0.2]).
    Detector + exponential filter as the single Burgers workload; dt = cfl * dx / (A + 0.1)."""
    out = []
    L = 2.0
    for i in range(n):
        r = _Stream(seed * 1000003 + i)
        E = r.integer(*e_range)
        P = r.integer(1, 4)
        N = r.integer(2, 10)
        A = 0.5 + 0.5 * r.uniform()
        if i % 2 == 0:
            m = r.integer(1, 3)
            phi = 2.0 * math.pi * r.uniform()
            ic = (lambda A, m, phi: (lambda x, z: (A * np.sin(2.0 * math.pi * m * x / L + phi) + 0.1 * z)[..., None]))(
                A, m, phi)
        else:
            x0 = L * r.uniform()
            w = 0.05 + 0.15 * r.uniform()
            ic = (lambda A, x0, w: (lambda x, z: (A * np.exp(-((x - x0) ** 2) / (2.0 * w * w)) * (1.0 + 0.1 * z))[..., None]))(
                A, x0, w)
        solver = dict(dim=1, nx=E, x0=0.0, x1=L, bc=("periodic",) * 4, P=P, N=N, Q=2 * N, equation="burgers",
                      filter="exp", sensor=True, f_alpha=36.0, f_s=4.0, s0=-2.0 * math.log10(P), kappa=4.0)
        out.append(dict(name=f"burgers_batch{seed}_{i}_E{E}_P{P}_N{N}", solver=solver, ic=ic, cfl=cfl, lam0=A + 0.1,
                        t_end=0.5))
    return out


def burgers_batch_member(i, seed=0):
    """Instance i of burgers_batch(seed=seed) alone (each instance has its own seeded stream)."""
    return burgers_batch(n=i + 1, seed=seed)[i]


ALL = {"advection": advection_1d, "burgers": burgers_1d, "sod": sod_1d, "shock_vortex": shock_vortex_2d}


def nodal_values(fn, nodes_x, nodes_z, nodes_y=None):
    """Evaluate an initial-data function at every (solution point, z-node): [E, Np, Q, S]."""
    vals = []
    for zq in nodes_z:
        v = fn(nodes_x, zq) if nodes_y is None else fn(nodes_x, nodes_y, zq)
        vals.append(np.asarray(v, dtype=np.float64))
    return np.ascontiguousarray(np.stack(vals, axis=2))


def boundary_values(fn, nodes_z):
    """Evaluate a boundary-state function at the z-nodes: [Q, S]."""
    return np.ascontiguousarray(np.stack([np.asarray(fn(zq), dtype=np.float64) for zq in nodes_z], 0))


def random_state(shape, seed, base, amp, decay=2.0):
    """Seeded gPC coefficients [E, Np, M, S]: mean `base[s]` in mode 0 plus Gaussian
    perturbations of size amp[s] / (1 + k)^decay in every mode k."""
    E, Np, M, S = shape
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(shape) * np.asarray(amp, dtype=np.float64)[None, None, None, :]
    u /= (1.0 + np.arange(M))[None, None, :, None] ** decay
    u[:, :, 0, :] += np.asarray(base, dtype=np.float64)[None, None, :]
    return u
