"""Host-side argument checks of rk_step_noalloc: a tensor of the wrong type, device or size,
or ghost modes of the wrong shape, are rejected before the library is called (the kernels
index the caller's arrays by the configuration's sizes)."""
import numpy as np
import pytest
import torch

from paper_2112_05946_gb300 import frsg
from paper_2112_05946_gb300 import workloads


class _FakeCuda:
    """Stands in for a CUDA tensor on a machine without a GPU: only the attributes the
    checks read."""

    def __init__(self, n, dtype=torch.float64, cuda=True, contiguous=True):
        self.dtype, self.is_cuda, self._n, self._c = dtype, cuda, n, contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


def _cfg():
    return dict(workloads.sod_1d(nx=64)["solver"])


def _n(cfg):
    return cfg["nx"] * (cfg["P"] + 1) * (cfg["N"] + 1) * 3


def test_well_formed_arguments_pass():
    cfg = _cfg()
    g = frsg.check_noalloc_args(_FakeCuda(_n(cfg)), _FakeCuda(_n(cfg)), np.zeros((4, cfg["N"] + 1, 3)), cfg)
    assert g.shape == (4, cfg["N"] + 1, 3) and g.flags["C_CONTIGUOUS"]


@pytest.mark.parametrize("bad", ["float32", "cpu", "short", "long", "strided"])
def test_bad_state_rejected_before_launch(bad):
    cfg = _cfg()
    n = _n(cfg)
    t = {"float32": _FakeCuda(n, dtype=torch.float32), "cpu": _FakeCuda(n, cuda=False),
         "short": _FakeCuda(n - 1), "long": _FakeCuda(n + 36), "strided": _FakeCuda(n, contiguous=False)}[bad]
    for args in ((t, _FakeCuda(n)), (_FakeCuda(n), t)):
        with pytest.raises(frsg.FrsgError) as ei:
            frsg.rk_step_noalloc(*args, 1e-4, 1, ghost_modes=np.zeros((4, cfg["N"] + 1, 3)), **cfg)
        assert ei.value.status == frsg.E_INVAL


def test_real_cpu_tensor_rejected():
    cfg = _cfg()
    u = torch.zeros(_n(cfg), dtype=torch.float64)
    with pytest.raises(frsg.FrsgError) as ei:
        frsg.rk_step_noalloc(u, u, 1e-4, 1, **cfg)
    assert ei.value.status == frsg.E_INVAL


@pytest.mark.parametrize("shape", [(4, 7, 1), (3, 7, 3), (4, 6, 3), (28, 3)])
def test_bad_ghost_shape_rejected(shape):
    cfg = _cfg()
    n = _n(cfg)
    with pytest.raises(frsg.FrsgError) as ei:
        frsg.check_noalloc_args(_FakeCuda(n), _FakeCuda(n), np.zeros(shape), cfg)
    assert ei.value.status == frsg.E_INVAL
