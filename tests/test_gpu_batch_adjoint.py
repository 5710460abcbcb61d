"""Batched discrete adjoint (fr_sg_batch_forward_record / fr_sg_batch_adjoint /
fr_sg_batch_integral_moments): gradients of the mean and the variance over z of the integral
of u at the end of the run with respect to every member's initial gPC coefficients, for a batch
of uneven stochastic Burgers problems (E, P, N drawn per member, detector + exponential filter).

Over a periodic mesh E[I] is conserved (the scheme is conservative and the filter keeps the
mean, Lambda_00 = 1), so its gradient is the quadrature weight of mode 0 at any time; Var[I]
decays where the filter damps the x-means of the higher gPC modes.  A seeded random cotangent
exercises the whole transposed run as well.

Checked: the moments and the gradients of both QoIs and of a random cotangent for small
members against the oracle's reverse mode (oracle/adjoint.py: torch autograd through the
oracle's steps with the decisions the oracle's own forward run took); every member of the
256-member workload against central finite differences of both QoIs and of the random
cotangent's functional along a seeded direction, the perturbed runs replaying the recorded
decisions (fr_sg_batch_forward_replay: the frozen-decision map the adjoint differentiates);
several cotangent sets in one call equal to one set at a time; the batched forward record
equal to the plain batched step; rejection of unsupported members.
"""
import numpy as np
import pytest

from oracle import adjoint, integrate
from paper_2112_05946_gb300 import workloads
from tests.helpers import gpu_initial, oracle_initial, oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu


def _members(wls, precision="fp64"):
    out = []
    for wl in wls:
        s = solver(wl, precision=precision)
        gpu_initial(s, wl)
        out.append(s)
    return out


def _dts(wls):
    return np.array([wl["cfl"] * (wl["solver"]["x1"] - wl["solver"]["x0"]) / wl["solver"]["nx"] / wl["lam0"]
                     for wl in wls])


def _grads(b, members, nset=2):
    """Seeds from integral_moments (the two QoIs' gradients at the final state), then the adjoint."""
    import torch
    lam = [[torch.empty(s.state_shape, dtype=torch.float64, device="cuda") for s in members] for _ in range(nset)]
    q = b.integral_moments(lam[0], lam[1] if nset > 1 else None)
    g = [[torch.empty_like(t) for t in ts] for ts in lam]
    b.adjoint(lam, g)
    torch.cuda.synchronize()
    return q, lam, g


def _oracle_vjp(prob, u0, dt, nsteps, flags, lam_T):
    """lambda_T^T (d u(T) / d u(0)) by torch autograd through the oracle's steps."""
    import torch
    tt = adjoint._tabs_torch(prob)
    x0 = torch.tensor(np.asarray(u0)[..., 0], dtype=torch.float64, requires_grad=True)
    x = x0
    for n in range(nsteps):
        x = adjoint.step_torch(prob, tt, x, dt, flags[3 * n:3 * n + 3])
    (g,) = torch.autograd.grad(torch.sum(x * torch.tensor(lam_T[..., 0])), x0)
    return g.numpy()[..., None]


@pytest.mark.parametrize("nsteps,k", [(20, 8), (9, 16)])
def test_batch_adjoint_matches_oracle_adjoint(nsteps, k):
    import torch
    from paper_2112_05946_gb300 import frsg
    wls = workloads.burgers_batch(n=6, seed=5, e_range=(12, 40))
    members = _members(wls)
    dts = _dts(wls)
    b = frsg.Batch(members)
    b.forward_record(dts, nsteps, k)
    q, _, g = _grads(b, members)
    rng = np.random.default_rng(nsteps)
    lam_r = [rng.standard_normal(s.state_shape) for s in members]
    g_r = [torch.empty(s.state_shape, dtype=torch.float64, device="cuda") for s in members]
    b.adjoint([[torch.tensor(x, device="cuda") for x in lam_r]], [g_r])
    for i, (wl, s, dt) in enumerate(zip(wls, members, dts)):
        s.check()
        prob = oracle_problem(wl)
        u0 = oracle_initial(prob, wl)
        rec = []
        integrate.run(prob, u0, dt, nsteps, record=rec)
        ref = adjoint.gradients(prob, u0, dt, nsteps, rec)
        assert rel_l2(s.get_state(), ref["state"]) < 1e-12, i
        assert abs(q[i, 0] - ref["mean"]) <= 1e-13 * abs(ref["mean"]) + 1e-15, (i, q[i, 0], ref["mean"])
        assert abs(q[i, 1] - ref["var"]) <= 1e-11 * abs(ref["var"]), (i, q[i, 1], ref["var"])
        assert rel_l2(g[0][i].cpu().numpy(), ref["grad_mean"]) < 1e-11, i
        assert rel_l2(g[1][i].cpu().numpy(), ref["grad_var"]) < 1e-10, i
        ref_r = _oracle_vjp(prob, u0, dt, nsteps, rec, lam_r[i])
        assert rel_l2(g_r[i].cpu().numpy(), ref_r) < 1e-11, i
    b.close()


def test_batch_adjoint_sets_are_independent_and_state_untouched():
    import torch
    from paper_2112_05946_gb300 import frsg
    wls = workloads.burgers_batch(n=10, seed=7, e_range=(16, 200))
    members = _members(wls)
    b = frsg.Batch(members)
    b.forward_record(_dts(wls), 24, 16)
    final = [s.get_state() for s in members]
    rng = np.random.default_rng(11)
    lam = [[torch.tensor(rng.standard_normal(s.state_shape), device="cuda") for s in members] for _ in range(3)]
    g3 = [[torch.empty_like(t) for t in ts] for ts in lam]
    b.adjoint(lam, g3)
    for c in range(3):
        g1 = [torch.empty_like(t) for t in lam[c]]
        b.adjoint([lam[c]], [g1])
        for i in range(len(members)):
            assert torch.equal(g1[i], g3[c][i]), (c, i)
    for s, u in zip(members, final):
        np.testing.assert_array_equal(s.get_state(), u)
    b.close()


def test_batch_forward_record_equals_batched_steps():
    from paper_2112_05946_gb300 import frsg
    wls = workloads.burgers_batch(n=12, seed=9, e_range=(16, 300))
    a, t = _members(wls), _members(wls)
    dts = _dts(wls)
    ba, bt = frsg.Batch(a), frsg.Batch(t)
    ba.forward_record(dts, 17, 5)
    bt.rk_step(dts, 17, graph=True)
    for s, r in zip(a, t):
        np.testing.assert_array_equal(s.get_state(), r.get_state())
    ba.close()
    bt.close()


def test_batch_adjoint_central_differences_full_workload():
    """All 256 members of the batched workload (E in 64..2048, P in 1..4, N in 2..10): the
    directional derivatives <grad Q, v> of E[I], Var[I] and <lambda, u(T)> (lambda seeded)
    against (Q(u0 + h v) - Q(u0 - h v)) / 2h, v seeded per member, 32 steps with checkpoints
    every 16, the perturbed runs replaying the recorded decisions."""
    import torch
    from paper_2112_05946_gb300 import frsg
    wls = workloads.burgers_batch()
    members = _members(wls)
    dts = _dts(wls)
    u0 = [s.get_state() for s in members]
    rng = np.random.default_rng(2024)
    v = [rng.standard_normal(u.shape) * np.abs(u).max() for u in u0]
    lam_r = [rng.standard_normal(u.shape) for u in u0]
    b = frsg.Batch(members)
    b.forward_record(dts, 32, 16)
    lam = [[torch.empty(s.state_shape, dtype=torch.float64, device="cuda") for s in members] for _ in range(2)]
    q0 = b.integral_moments(lam[0], lam[1])
    lam.append([torch.tensor(x, device="cuda") for x in lam_r])
    g = [[torch.empty_like(t) for t in ts] for ts in lam]
    b.adjoint(lam, g)
    def central(h):
        qs, fs = [], []
        for sign in (1.0, -1.0):
            for s, u, d in zip(members, u0, v):
                s.set_state(u + sign * h * d)
            b.forward_replay(32)
            qs.append(b.integral_moments())
            fs.append(np.array([np.sum(x * s.get_state()) for x, s in zip(lam_r, members)]))
        return np.concatenate([(qs[0] - qs[1]) / (2 * h), ((fs[0] - fs[1]) / (2 * h))[:, None]], axis=1), fs[0]

    # the frozen-decision map is not quadratic (the filtered element means move with the flow):
    # Richardson's combination of h and h / 2 removes the h^2 term of the differences.  It is not
    # smooth everywhere either: the Lax-Friedrichs dissipation max(|u_L|, |u_R|) switches branch
    # where the two speeds cross (everywhere in the flat parts of the Gaussian members, where u
    # is near zero), and a perturbation of every coefficient crosses some of those kinks.  The
    # QoIs see only the x-means of the modes and are held to 1e-6.  The functional of a random
    # cotangent sees every point: measured up to 7.5e-4 on a Gaussian member whose flat parts sit
    # at u = 0, so it is only held to 1e-2 here; the exact check of the same transposed runs is
    # the comparison with the oracle's reverse mode (above, and on the workload's own small
    # members in the next test)
    h = 1e-6
    fd_h, f_ref = central(h)
    fd_h2, _ = central(h / 2)
    fd = (4.0 * fd_h2 - fd_h) / 3.0
    rel = np.zeros((len(members), 3))
    for i, d in enumerate(v):
        dd = torch.tensor(d, device="cuda")
        for c in range(3):
            ad = float(torch.sum(g[c][i] * dd))
            # round-off of Q over the step: about 1e-16 |Q| / (h / 2), times the combination's 5
            noise = 1e-8 * (np.abs(q0[i, c]) if c < 2 else np.abs(f_ref[i]))
            rel[i, c] = max(abs(ad - fd[i, c]) - noise, 0.0) / max(abs(ad), abs(fd[i, c]))
    worst = rel.max(axis=0)
    assert worst[0] < 1e-6 and worst[1] < 1e-6 and worst[2] < 1e-2, (worst, rel.argmax(axis=0))
    b.close()


def test_batch_adjoint_workload_members_match_oracle():
    """The members of the batched workload with at most 160 elements (12 of the 256: P 1..4,
    N 2..10, sine and Gaussian data) as one batch, 32 steps with checkpoints every 16: a seeded
    random cotangent's gradient against the oracle's reverse mode."""
    import torch
    from paper_2112_05946_gb300 import frsg
    wls = [wl for wl in workloads.burgers_batch() if wl["solver"]["nx"] <= 160]
    assert len(wls) >= 10
    members = _members(wls)
    dts = _dts(wls)
    nsteps = 32
    b = frsg.Batch(members)
    b.forward_record(dts, nsteps, 16)
    rng = np.random.default_rng(17)
    lam = [rng.standard_normal(s.state_shape) for s in members]
    g = [torch.empty(s.state_shape, dtype=torch.float64, device="cuda") for s in members]
    b.adjoint([[torch.tensor(x, device="cuda") for x in lam]], [g])
    for i, (wl, s, dt) in enumerate(zip(wls, members, dts)):
        prob = oracle_problem(wl)
        u0 = oracle_initial(prob, wl)
        rec = []
        fin = integrate.run(prob, u0, dt, nsteps, record=rec)
        assert rel_l2(s.get_state(), fin) < 1e-11, (i, wl["name"])
        ref = _oracle_vjp(prob, u0, dt, nsteps, rec, lam[i])
        assert rel_l2(g[i].cpu().numpy(), ref) < 1e-10, (i, wl["name"])
    b.close()


def test_batch_adjoint_rejects_unsupported_members():
    from paper_2112_05946_gb300 import frsg
    wls = workloads.burgers_batch(n=3, seed=1, e_range=(16, 40))
    f32 = _members(wls, precision="fp32")
    b = frsg.Batch(f32)
    with pytest.raises(frsg.FrsgError):
        b.forward_record(_dts(wls), 4, 2)
    b.close()
    members = _members(wls)
    b = frsg.Batch(members)
    with pytest.raises(frsg.FrsgError):        # no recorded run yet
        import torch
        lam = [[torch.zeros(s.state_shape, dtype=torch.float64, device="cuda") for s in members]]
        b.adjoint(lam, [[torch.empty_like(t) for t in lam[0]]])
    b.close()
