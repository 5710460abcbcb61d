"""Oracle pin against the paper's only printed numbers: the advection accuracy study of §5.1
(Tables 2-3, stored in tests/golden/advection_rk4_errors.txt), run with the classical RK4
integrator of that study.

Reading of the tables: the L1 / L2 / Linf orders printed there differ by 1 and 1/2, the
signature of unnormalised sums over the solution points; the absolute values are not
reproducible from the stated setup (the N_x range of the setup table contradicts the dx
column).  What is pinned: (1) the printed orders are self-consistent with their own error
columns; (2) the point-count-normalised L1 order of the oracle between the two finest
rows (dx = 0.0625 -> 0.03125) equals the printed L1 order within 0.1; (3) the pointwise
(Linf) order reaches the design order P + 1 ("third- and fourth-order schemes", §5.1);
(4) RK4 itself is fourth order against the matrix exponential of the linear
semi-discrete advection operator.
"""
import pathlib

import numpy as np
import pytest

import oracle
from oracle import integrate, scheme

GOLDEN = pathlib.Path(__file__).parent / "golden" / "advection_rk4_errors.txt"


def _table():
    rows = [l.split() for l in GOLDEN.read_text().splitlines() if l.strip() and not l.startswith("#")]
    return np.array([[float(v) for v in r] for r in rows])


def _advection_errors(P, nx, t_end=50.0, cfl=0.1):
    prob = oracle.Problem(nx=nx, P=P, N=5, Q=9, equation="advection", adv_speed=1.0, x0=-1.0, x1=1.0,
                          filter="none", sensor=False)
    xi = lambda z: 1.0 + 0.1 * z                                       # noqa: E731  U(0.9, 1.1)
    u = integrate.project_initial(prob, lambda x, z: (xi(z) * np.sin(np.pi * x))[..., None])
    n = int(round(t_end / (cfl * prob.dx)))
    dt = t_end / n
    tabs = prob.tabs()
    for _ in range(n):
        u = integrate.rk4_step(prob, tabs, u, dt)
    e = u[:, :, 0, 0] - np.sin(np.pi * (prob.nodes() - t_end))         # E[xi] = 1
    return np.array([np.mean(np.abs(e)), np.sqrt(np.mean(e ** 2)), np.max(np.abs(e))])


def test_printed_orders_match_printed_errors():
    t = _table()
    for P in (2, 3):
        r = t[t[:, 0] == P]
        for i in range(1, len(r)):
            for c in (2, 4, 6):
                order = np.log(r[i - 1, c] / r[i, c]) / np.log(r[i - 1, 1] / r[i, 1])
                assert abs(order - r[i, c + 1]) < 0.011, (P, i, c)


def test_rk4_order_against_matrix_exponential():
    # linear advection: the semi-discrete system is u' = A u; its exact solution is
    # expm(A t) u0 (scipy), so the integrator's global error must fall as dt^4
    from scipy.linalg import expm
    prob = oracle.Problem(nx=4, P=2, N=1, Q=2, equation="advection", adv_speed=1.0, x0=-1.0, x1=1.0,
                          filter="none", sensor=False)
    tabs = prob.tabs()
    shape = (prob.E, prob.Np, prob.M, prob.S)
    n = int(np.prod(shape))
    A = np.stack([scheme.rhs(prob, tabs, np.eye(n)[i].reshape(shape)).ravel() for i in range(n)], axis=1)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(shape)
    T = 0.5
    exact = expm(A * T) @ u0.ravel()
    errs = []
    for steps in (10, 20, 40):
        u = u0
        for _ in range(steps):
            u = integrate.rk4_step(prob, tabs, u, T / steps)
        errs.append(np.linalg.norm(u.ravel() - exact))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 4.0) < 0.2), orders


@pytest.mark.parametrize("P", [2, 3])
def test_finest_rows_order(P):
    t = _table()
    r = t[t[:, 0] == P]
    coarse = _advection_errors(P, 32)      # dx = 0.0625
    fine = _advection_errors(P, 64)        # dx = 0.03125
    orders = np.log2(coarse / fine)
    assert abs(orders[0] - r[-1, 3]) < 0.1, (orders, r[-1])
    assert orders[2] > P + 1 - 0.1, orders
    assert np.all(fine < coarse)
