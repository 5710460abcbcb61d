"""Hand-written discrete adjoint on the GPU (fr_sg_forward_record / fr_sg_adjoint and the
torch.autograd.Function around them) against the oracle adjoint, central finite
differences and closed forms."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, integrate
from paper_2112_05946_gb300 import workloads
from tests.helpers import oracle_problem, rel_l2, solver

pytestmark = pytest.mark.gpu


def _burgers(nx=24, P=2, N=3, Q=7, filt="exp"):
    wl = workloads.burgers_1d(nx=nx, P=P, N=N, Q=Q)
    wl["solver"]["filter"] = filt
    return wl


def _state(prob, wl):
    return integrate.project_initial(prob, lambda x, z: (np.sin(np.pi * x) + 0.1 * z + 0.3)[..., None])


@pytest.mark.parametrize("nsteps,k", [(40, 16), (17, 5), (9, 1)])
@pytest.mark.parametrize("filt", ["exp", "none"])
def test_adjoint_matches_oracle_adjoint(nsteps, k, filt):
    import torch
    wl = _burgers(filt=filt)
    prob = oracle_problem(wl)
    u0 = _state(prob, wl)
    dt = 0.1 * prob.dx / 1.3
    rec = []
    integrate.run(prob, u0, dt, nsteps, record=rec)
    ref = adjoint.gradients(prob, u0, dt, nsteps, rec)
    s = solver(wl)
    s.set_state(u0)
    s.forward_record(dt, nsteps, k)
    s.check()
    assert rel_l2(s.get_state(), ref["state"]) < 1e-12
    flags = s.decisions()[0]
    gm_seed, gv_seed = adjoint.qoi_seeds(prob, ref["state"])
    for seed, key in [(gm_seed, "grad_mean"), (gv_seed, "grad_var")]:
        lam = torch.tensor(seed, device="cuda")
        g = torch.empty_like(lam)
        s.adjoint(lam, g)
        s.check()
        assert rel_l2(g.cpu().numpy(), ref[key]) < 1e-11, key
    # the context's state is the final state again
    assert rel_l2(s.get_state(), ref["state"]) < 1e-12
    del flags


def test_adjoint_finite_differences_through_the_abi():
    """<grad, v> against (Q(u0 + h v) - Q(u0 - h v)) / 2h with both runs on the GPU and the
    forward run's filter decisions replayed."""
    import torch
    wl = _burgers(nx=32, P=3, N=4, Q=9)
    prob = oracle_problem(wl)
    u0 = _state(prob, wl)
    dt = 0.1 * prob.dx / 1.3
    nsteps = 60
    s = solver(wl)
    s.set_state(u0)
    s.forward_record(dt, nsteps, 16)
    uT = s.get_state()
    # decisions of the recorded run, replayed in the perturbed runs
    rec = []
    integrate.run(prob, u0, dt, nsteps, record=rec)
    _, gv_seed = adjoint.qoi_seeds(prob, uT)
    lam = torch.tensor(gv_seed, device="cuda")
    g = torch.empty_like(lam)
    s.adjoint(lam, g)
    g = g.cpu().numpy()

    def qvar(u):
        w = s.quadrature()[0]
        I = 0.5 * prob.dx * np.einsum("j,ejk->k", w, u[..., 0])
        return np.sum(I[1:] ** 2)

    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(2):
        v = rng.standard_normal(u0.shape)
        vals = []
        for sign in (1, -1):
            s2 = solver(wl)
            s2.set_state(u0 + sign * h * v)
            s2.set_replay(np.array(rec, dtype=np.uint8))
            s2.rk_step(dt, nsteps, graph=False)
            vals.append(qvar(s2.get_state()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(np.sum(g * v) - fd) < 1e-6 * max(abs(fd), 1e-4)


def test_mean_gradient_closed_form():
    """Periodic conservative FR with a mode-0-preserving filter conserves E[int u]: its
    gradient w.r.t. uhat(0) is J w_j on mode 0 and zero elsewhere."""
    import torch
    wl = _burgers(nx=48, P=3, N=8, Q=16)
    prob = oracle_problem(wl)
    u0 = _state(prob, wl)
    s = solver(wl)
    s.set_state(u0)
    s.forward_record(0.1 * prob.dx / 1.3, 100, 16)
    gm_seed, _ = adjoint.qoi_seeds(prob, u0)
    lam = torch.tensor(gm_seed, device="cuda")
    g = torch.empty_like(lam)
    s.adjoint(lam, g)
    np.testing.assert_allclose(g.cpu().numpy(), gm_seed, atol=1e-13)


def test_autograd_function_gives_the_adjoint_gradient():
    import torch
    from paper_2112_05946_gb300.autograd import FRSGRun, qoi_mean_var, quadrature_weights
    wl = _burgers(nx=24)
    prob = oracle_problem(wl)
    u0n = _state(prob, wl)
    dt = 0.1 * prob.dx / 1.3
    s = solver(wl)
    u0 = torch.tensor(u0n, device="cuda", requires_grad=True)
    uT = FRSGRun.apply(u0, s, dt, 40, 16)
    mean, var = qoi_mean_var(quadrature_weights(s), uT)
    (var + 0.5 * mean).backward()
    rec = []
    integrate.run(prob, u0n, dt, 40, record=rec)
    ref = adjoint.gradients(prob, u0n, dt, 40, rec)
    assert rel_l2(u0.grad.cpu().numpy(), ref["grad_var"] + 0.5 * ref["grad_mean"]) < 1e-11


def test_adjoint_rejects_unsupported_contexts():
    """FP32 states, 2D meshes, scalar problems with the HLL flux, the Lasso filter and
    non-periodic scalar problems have no adjoint."""
    from paper_2112_05946_gb300 import frsg
    cases = [
        solver(workloads.sod_1d(nx=8), precision="fp32"),
        solver(workloads.shock_vortex_2d(nx=4, ny=4)),
        solver(_burgers(nx=8), flux="hll"),
        solver(_burgers(nx=8), filter="lasso", sensor=False),
        solver(_burgers(nx=8), bc=("outflow", "outflow", "periodic", "periodic")),
    ]
    for s in cases:
        with pytest.raises(frsg.FrsgError) as ei:
            s.forward_record(1e-4, 2, 1)
        assert ei.value.status == frsg.E_UNSUPPORTED


def test_parameter_gradient_of_uncertainty_magnitude():
    """d QoI / d sigma for u0 = sin(pi x) + 0.3 + sigma z, through FRSGProject -> FRSGRun ->
    a torch QoI.  (a) Var[int u dx] is conserved without a filter (periodic, conservative
    scheme), so its gradient is the closed form 2 sigma L^2 / 3 (int u dx has the gPC
    coefficient I_1 = sigma L / sqrt(3), z = Phi_1 / sqrt(3)); (b) the energy of the mean
    field, sum J w_j E[u]^2 at t_end, against central differences of the FP64 oracle run
    with the filter applied to every element (no detector switching)."""
    import torch
    from paper_2112_05946_gb300.autograd import FRSGProject, FRSGRun, qoi_mean_var, quadrature_weights
    sigma0 = 0.1
    for filt, sensor in [("none", True), ("exp", False)]:
        wl = _burgers(nx=32, P=3, N=4, Q=9, filt=filt)
        wl["solver"]["sensor"] = sensor
        prob = oracle_problem(wl)
        s = solver(wl)
        x, z = s.nodes()
        dt = 0.1 * prob.dx / 1.4
        nsteps = 40
        sig = torch.tensor(sigma0, dtype=torch.float64, device="cuda", requires_grad=True)
        xt = torch.tensor(x, device="cuda")
        zt = torch.tensor(z, device="cuda")
        nodal = (torch.sin(np.pi * xt) + 0.3)[:, :, None, None] + sig * zt[None, None, :, None]
        uT = FRSGRun.apply(FRSGProject.apply(nodal, s), s, dt, nsteps, 8)
        Jw = quadrature_weights(s)
        if filt == "none":
            _, var = qoi_mean_var(Jw, uT)
            (g,) = torch.autograd.grad(var, sig)
            L = prob.x1 - prob.x0
            assert float(g) == pytest.approx(2 * sigma0 * L ** 2 / 3, rel=1e-10)
        else:
            energy = torch.sum(Jw[None, :] * uT[:, :, 0, 0] ** 2)
            (g,) = torch.autograd.grad(energy, sig)

            def oracle_energy(sg):
                u0 = integrate.project_initial(prob, lambda xx, zz: (np.sin(np.pi * xx) + 0.3 + sg * zz)[..., None])
                u = integrate.run(prob, u0, dt, nsteps)
                w = prob.tabs()["w"]
                return float(np.sum(0.5 * prob.dx * w[None, :] * u[:, :, 0, 0] ** 2))
            h = 1e-5
            fd = (oracle_energy(sigma0 + h) - oracle_energy(sigma0 - h)) / (2 * h)
            assert float(g) == pytest.approx(fd, rel=1e-6)
        s.check()
