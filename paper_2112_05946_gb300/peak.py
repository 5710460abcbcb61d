"""Binding of libfrsg_peak.so: FP64 / FP32 fused multiply-add throughput of the current GPU,
the compute denominators of the stage kernels' roofline (include/frsg_peak.h)."""
import ctypes
import os

from .build import PEAK_OUT


def fma_tflops(fp64, iters=None, reps=5):
    """Measured dense FMA throughput in TFLOP/s (2 flops per FMA) of the current device."""
    if not os.path.exists(PEAK_OUT):
        raise FileNotFoundError(f"{PEAK_OUT} is missing: build it with paper_2112_05946_gb300.build.build()")
    lib = ctypes.CDLL(PEAK_OUT)
    lib.frsg_peak_fma.restype = ctypes.c_int
    lib.frsg_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double()
    if iters is None:
        iters = 200 if fp64 else 4000
    if lib.frsg_peak_fma(1 if fp64 else 0, int(iters), int(reps), ctypes.byref(out)) != 0:
        raise RuntimeError("frsg_peak_fma failed")
    return out.value
