"""fr_sg_advance: one call from a state to a state must equal fr_sg_set_state, fr_sg_rk_step
and fr_sg_get_state (bit for bit), for host and device arrays, in place, in both precisions."""
import numpy as np
import pytest

from paper_2112_05946_gb300 import frsg, workloads
from tests.helpers import oracle_problem, solver

pytestmark = pytest.mark.gpu


def _front(s, seed):
    x = s.nodes()[0]
    u = workloads.random_state(s.state_shape, seed=seed, base=[0.0], amp=[1e-3])
    u[:, :, 0, 0] += np.tanh((x - 1.0) / 0.05)
    return u


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", [0, 1, 3])
def test_advance_equals_set_step_get(precision, variant):
    import torch
    wl = workloads.burgers_1d(nx=40)
    prob = oracle_problem(wl, nx=40)
    dt = 0.1 * prob.dx / 1.2
    ref_s = solver(wl, precision=precision)
    ref_s.set_variant(variant)
    u = _front(ref_s, seed=5)
    ref_s.set_state(u)
    ref_s.rk_step(dt, 3, graph=True)
    ref_s.check()
    ref = ref_s.get_state()

    s = solver(wl, precision=precision)
    s.set_variant(variant)
    out = np.empty_like(u)
    s.advance(u, out, dt, 3)
    s.check()
    np.testing.assert_array_equal(out, ref)
    np.testing.assert_array_equal(s.get_state(), ref)    # the context holds the result too

    inplace = u.copy()
    s.advance(inplace, inplace, dt, 3)
    np.testing.assert_array_equal(inplace, ref)

    # pinned host memory (read and written in place by the FP32 conversion kernels)
    pin_in = torch.tensor(u, dtype=torch.float64).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    s.advance(pin_in.numpy(), pin_out.numpy(), dt, 3)
    np.testing.assert_array_equal(pin_out.numpy(), ref)
    s.advance(pin_in.numpy(), pin_in.numpy(), dt, 3)
    np.testing.assert_array_equal(pin_in.numpy(), ref)

    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    od = torch.empty_like(ud)
    s.advance(ud, od, dt, 3)
    torch.cuda.synchronize()
    s.check()
    np.testing.assert_array_equal(od.cpu().numpy(), ref)


def test_advance_rejects_bad_arguments_and_keeps_the_state():
    wl = workloads.burgers_1d(nx=16)
    s = solver(wl)
    u = _front(s, seed=2)
    s.set_state(u)
    out = np.empty_like(u)
    with pytest.raises(frsg.FrsgError) as ei:
        s.advance(u + 1.0, out, -1e-3, 1)
    assert ei.value.status == frsg.E_INVAL
    with pytest.raises(frsg.FrsgError):
        s.advance(u + 1.0, out, 1e-3, -1)
    np.testing.assert_array_equal(s.get_state(), u)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_advance_native_equals_advance(precision):
    """fr_sg_advance_native with arrays in the form's own precision gives the state fr_sg_advance
    gives (a float form rounds a double input to float anyway; widening back is exact)."""
    import torch
    wl = workloads.burgers_1d(nx=40)
    prob = oracle_problem(wl, nx=40)
    dt = 0.1 * prob.dx / 1.2
    s = solver(wl, precision=precision)
    u = _front(s, seed=9)
    ref = np.empty_like(u)
    s.advance(u, ref, dt, 3)
    dt_np = np.float64 if precision == "fp64" else np.float32
    un = u.astype(dt_np)
    out = np.empty_like(un)
    s.advance_native(un, out, dt, 3)
    s.check()
    np.testing.assert_array_equal(out.astype(np.float64), ref)
    # pinned host memory and device tensors, in place
    tdt = torch.float64 if precision == "fp64" else torch.float32
    pin = torch.tensor(un).pin_memory()
    s.advance_native(pin.numpy(), pin.numpy(), dt, 3)
    np.testing.assert_array_equal(pin.numpy().astype(np.float64), ref)
    dev = torch.tensor(un, device="cuda")
    s.advance_native(dev, dev, dt, 3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dev.cpu().numpy().astype(np.float64), ref)
    # the other precision, or a short array, is rejected before any call
    wrong = u.astype(np.float32 if precision == "fp64" else np.float64)
    with pytest.raises(ValueError):
        s.advance_native(wrong, np.empty_like(wrong), dt, 1)
    with pytest.raises(ValueError):
        s.advance_native(un[:-1], out[:-1], dt, 1)
    assert tdt is not None
    s.close()
