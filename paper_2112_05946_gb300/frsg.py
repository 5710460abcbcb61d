"""Thin ctypes binding of libfrsg (include/frsg.h).  Argument marshalling only.

Every numerical step runs in the CUDA library; this module converts Python values
into the C structures and pointers the C ABI expects, and turns non-zero status
codes into exceptions.  Device buffers are torch tensors (their data_ptr is passed),
host buffers are numpy arrays.  The library must have been built (build.build());
importing this module on a machine without it raises instead of falling back.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfrsg.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_NONFINITE, E_POSITIVITY, E_TIMEOUT, E_UNSUPPORTED = range(8)
BC = {"periodic": 0, "dirichlet": 1, "outflow": 2, "reflect": 3}
EQUATION = {"advection": 0, "burgers": 1, "euler": 2}
FILTER = {"none": 0, "exp": 1, "l2": 2, "lasso": 3}
FLUX = {"llf": 0, "hll": 1}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_tc": 2}
HOST, DEVICE = 0, 1


class FrsgError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"frsg status {status}: {message}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("dim", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4),
        ("P", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("Q", ctypes.c_int32),
        ("equation", ctypes.c_int32),
        ("adv_speed", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("filter", ctypes.c_int32),
        ("sensor", ctypes.c_int32),
        ("f_alpha", ctypes.c_double), ("f_s", ctypes.c_double),
        ("f_eps1", ctypes.c_double), ("f_eps2", ctypes.c_double),
        ("s0", ctypes.c_double), ("kappa", ctypes.c_double),
        ("limiter", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("flux", ctypes.c_int32),
    ]


_lib = None

# (name, restype, argtypes) of every exported entry point in include/frsg.h
_SIGNATURES = [
    ("fr_sg_init", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("fr_sg_destroy", None, [ctypes.c_void_p]),
    ("fr_sg_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("fr_sg_sizes", ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 5),
    ("fr_sg_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("fr_sg_get_nodes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fr_sg_get_quadrature", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fr_sg_set_boundary_nodal", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("fr_sg_set_initial_nodal", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_set_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_get_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_rhs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fr_sg_rk_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    ("fr_sg_rk4_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    ("fr_sg_advance", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int]),
    ("fr_sg_advance_native", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    ("fr_sg_tune_cache_save", ctypes.c_int, [ctypes.c_char_p]),
    ("fr_sg_tune_cache_load", ctypes.c_int, [ctypes.c_char_p]),
    ("fr_sg_project", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_project_transpose", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_stage", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    ("fr_sg_filter", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("fr_sg_limit", ctypes.c_int, [ctypes.c_void_p]),
    ("fr_sg_moments", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_cfl_dt", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    ("fr_sg_get_decisions", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fr_sg_set_replay", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_check", ctypes.c_int, [ctypes.c_void_p]),
    ("fr_sg_launch_count", ctypes.c_uint64, [ctypes.c_void_p]),
    ("fr_sg_set_tile", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("fr_sg_set_variant", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_test_fused_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int]),
    ("fr_sg_set_timing_events", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fr_sg_cell_means", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    ("fr_sg_forward_record", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    ("fr_sg_adjoint", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fr_sg_batch_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    ("fr_sg_batch_destroy", None, [ctypes.c_void_p]),
    ("fr_sg_batch_rk_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("fr_sg_batch_launch_count", ctypes.c_uint64, [ctypes.c_void_p]),
    ("fr_sg_batch_forward_record", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("fr_sg_batch_forward_replay", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("fr_sg_batch_adjoint", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p)]),
    ("fr_sg_batch_integral_moments", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.POINTER(ctypes.c_void_p),
                                                    ctypes.POINTER(ctypes.c_void_p)]),
    ("fr_sg_batch_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_size_t)]),
    ("fr_sg_rk_step_noalloc", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
]


def load_library(path=LIB_PATH):
    """Load libfrsg.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: build it with paper_2112_05946_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_names():
    return [s[0] for s in _SIGNATURES]


def make_config(dim=1, nx=32, ny=1, x0=0.0, x1=2.0, y0=0.0, y1=1.0, bc=("periodic",) * 4, P=2, N=4, Q=8,
                equation="advection", adv_speed=1.0, gamma=1.4, filter="none", sensor=True, f_alpha=36.0,
                f_s=4.0, f_eps1=0.6, f_eps2=0.6, s0=0.0, kappa=4.0, limiter=False, precision="fp64", flux="llf"):
    c = Config()
    c.struct_size = ctypes.sizeof(Config)
    c.dim, c.nx, c.ny = dim, nx, ny
    c.x0, c.x1, c.y0, c.y1 = x0, x1, y0, y1
    for i, b in enumerate(bc):
        c.bc[i] = BC[b] if isinstance(b, str) else int(b)
    c.P, c.N, c.Q = P, N, Q
    c.equation = EQUATION[equation]
    c.adv_speed, c.gamma = adv_speed, gamma
    c.filter = FILTER[filter]
    c.sensor = int(bool(sensor))
    c.f_alpha, c.f_s, c.f_eps1, c.f_eps2, c.s0, c.kappa = f_alpha, f_s, f_eps1, f_eps2, s0, kappa
    c.limiter = int(bool(limiter))
    c.precision = PRECISION[precision]
    c.flux = FLUX[flux] if isinstance(flux, str) else int(flux)
    return c


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():   # torch tensor: the C ABI reads the row-major layout
        raise ValueError("device tensors must be contiguous")
    return a.data_ptr()


def tune_cache_save(path):
    """fr_sg_tune_cache_save: write the autotuner's per-shape choices to a text file."""
    st = load_library().fr_sg_tune_cache_save(os.fsencode(path))
    if st != OK:
        raise FrsgError(st, f"fr_sg_tune_cache_save({path}) failed")


def tune_cache_load(path):
    """fr_sg_tune_cache_load: merge a file written by tune_cache_save into the cache."""
    st = load_library().fr_sg_tune_cache_load(os.fsencode(path))
    if st != OK:
        raise FrsgError(st, f"fr_sg_tune_cache_load({path}) failed")


def check_noalloc_args(u_in, u_out, ghost_modes, cfg):
    """Argument checks of rk_step_noalloc, made before the library is called: both states are
    contiguous CUDA float64 tensors of E*Np*M*S values for the configuration, and the ghost
    modes (when given) have shape (4, M, S).  The kernels index the states by the
    configuration's sizes, so a smaller or mistyped tensor would be read and written out of
    bounds.  Raises FrsgError(E_INVAL) and returns the ghost modes as a contiguous array."""
    P, N = cfg.get("P", 2), cfg.get("N", 4)
    equation = cfg.get("equation", "advection")
    S = 3 if equation == "euler" else 1
    want = int(cfg.get("nx", 32)) * (P + 1) * (N + 1) * S
    for name, t in (("u_in", u_in), ("u_out", u_out)):
        if str(getattr(t, "dtype", None)) != "torch.float64":
            raise FrsgError(E_INVAL, f"rk_step_noalloc: {name} must be a torch.float64 tensor")
        if not getattr(t, "is_cuda", False):
            raise FrsgError(E_INVAL, f"rk_step_noalloc: {name} must be on a CUDA device")
        if not t.is_contiguous() or t.numel() != want:
            raise FrsgError(E_INVAL, f"rk_step_noalloc: {name} must be contiguous with {want} values "
                                     f"(nx*(P+1)*(N+1)*S), got {t.numel()}")
    if ghost_modes is None:
        return None
    g = np.ascontiguousarray(ghost_modes, dtype=np.float64)
    if g.shape != (4, N + 1, S):
        raise FrsgError(E_INVAL, f"rk_step_noalloc: ghost_modes must have shape (4, {N + 1}, {S}), got {g.shape}")
    return g


def rk_step_noalloc(u_in, u_out, dt, nsteps=1, ghost_modes=None, stream=None, **cfg):
    """fr_sg_rk_step_noalloc: nsteps SSP-RK3 steps of a 1D FP64 problem for callers that may
    not allocate device memory; u_in, u_out are device float64 tensors [E, Np, M, S]."""
    g = check_noalloc_args(u_in, u_out, ghost_modes, cfg)
    lib = load_library()
    c = make_config(**cfg)
    st = lib.fr_sg_rk_step_noalloc(ctypes.byref(c), _ptr(g), _ptr(u_in), _ptr(u_out), float(dt), int(nsteps),
                                   ctypes.c_void_p(stream or 0))
    if st != OK:
        raise FrsgError(st, "fr_sg_rk_step_noalloc failed (details on stderr)")


class Solver:
    """One FR-SG context (fr_sg_init ... fr_sg_destroy)."""

    def __init__(self, stream=None, **cfg):
        self.lib = load_library()
        self.cfg_kwargs = dict(cfg)
        self.cfg = make_config(**cfg)
        h = ctypes.c_void_p()
        st = self.lib.fr_sg_init(ctypes.byref(self.cfg), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != OK:
            raise FrsgError(st, "fr_sg_init rejected the configuration (details on stderr)")
        self.h = h
        E, Np, M, S, Q = (ctypes.c_int() for _ in range(5))
        self.lib.fr_sg_sizes(self.h, ctypes.byref(E), ctypes.byref(Np), ctypes.byref(M), ctypes.byref(S),
                             ctypes.byref(Q))
        self.E, self.Np, self.M, self.S, self.Q = E.value, Np.value, M.value, S.value, Q.value
        self.fp64 = self.cfg.precision == 0

    # ------------------------------------------------------------------ plumbing
    def _ck(self, st, what):
        if st != OK:
            msg = self.lib.fr_sg_last_error(self.h)
            raise FrsgError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.fr_sg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def state_shape(self):
        return (self.E, self.Np, self.M, self.S)

    def set_stream(self, stream):
        self._ck(self.lib.fr_sg_set_stream(self.h, ctypes.c_void_p(stream or 0)), "set_stream")

    # ------------------------------------------------------------------ data
    def nodes(self):
        x = np.zeros((self.E, self.Np))
        y = np.zeros((self.E, self.Np))
        z = np.zeros(self.Q)
        self._ck(self.lib.fr_sg_get_nodes(self.h, _ptr(x), _ptr(y), _ptr(z)), "get_nodes")
        return (x, z) if self.cfg.dim == 1 else (x, y, z)

    def quadrature(self):
        """(wx[Np], wz[Q]): reference-element Gauss weights and z probability weights."""
        wx = np.zeros(self.Np)
        wz = np.zeros(self.Q)
        self._ck(self.lib.fr_sg_get_quadrature(self.h, _ptr(wx), _ptr(wz)), "get_quadrature")
        return wx, wz

    def set_boundary_nodal(self, side, g):
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(self.Q, self.S)
        self._ck(self.lib.fr_sg_set_boundary_nodal(self.h, side, _ptr(g)), "set_boundary_nodal")

    def set_initial_nodal(self, u0):
        if isinstance(u0, np.ndarray):
            u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(self.E, self.Np, self.Q, self.S)
            self._ck(self.lib.fr_sg_set_initial_nodal(self.h, _ptr(u0), HOST), "set_initial_nodal")
        else:
            self._ck(self.lib.fr_sg_set_initial_nodal(self.h, _ptr(u0), DEVICE), "set_initial_nodal")

    def set_state(self, uhat):
        if isinstance(uhat, np.ndarray):
            uhat = np.ascontiguousarray(uhat, dtype=np.float64).reshape(self.state_shape)
            self._ck(self.lib.fr_sg_set_state(self.h, _ptr(uhat), HOST), "set_state")
        else:
            self._ck(self.lib.fr_sg_set_state(self.h, _ptr(uhat), DEVICE), "set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.zeros(self.state_shape)
            self._ck(self.lib.fr_sg_get_state(self.h, _ptr(out), HOST), "get_state")
            return out
        if isinstance(out, np.ndarray):
            self._ck(self.lib.fr_sg_get_state(self.h, _ptr(out), HOST), "get_state")
        else:
            self._ck(self.lib.fr_sg_get_state(self.h, _ptr(out), DEVICE), "get_state")
        return out

    # ------------------------------------------------------------------ compute
    def rhs(self, u, dudt):
        """u, dudt: device tensors of the context's precision, shape [E, Np, M, S]."""
        self._ck(self.lib.fr_sg_rhs(self.h, _ptr(u), _ptr(dudt)), "rhs")

    def rk_step(self, dt, nsteps=1, graph=True):
        self._ck(self.lib.fr_sg_rk_step(self.h, float(dt), int(nsteps), int(bool(graph))), "rk_step")

    def advance(self, u_in, u_out, dt, nsteps=1, graph=True):
        """fr_sg_advance: state u_in -> nsteps SSP-RK3 steps -> u_out, one call.  numpy float64
        arrays (host, synchronous) or device float64 tensors [E, Np, M, S]; may be the same."""
        host = isinstance(u_in, np.ndarray)
        if host != isinstance(u_out, np.ndarray):
            raise TypeError("u_in and u_out must both be host arrays or both device tensors")
        if host:
            nbytes = 8 * self.E * self.Np * self.M * self.S
            for a in (u_in, u_out):
                if a.dtype != np.float64 or not a.flags.c_contiguous or a.nbytes != nbytes:
                    raise ValueError("host states must be C-contiguous float64 arrays of the state's size")
            pin, pout = u_in.ctypes.data, u_out.ctypes.data
        else:
            pin, pout = _ptr(u_in), _ptr(u_out)
        st = self.lib.fr_sg_advance(self.h, pin, pout, HOST if host else DEVICE, float(dt), int(nsteps),
                                    1 if graph else 0)
        if st != OK:
            self._ck(st, "advance")
        return u_out

    def advance_native(self, u_in, u_out, dt, nsteps=1, graph=True):
        """fr_sg_advance_native: as advance, with the arrays in the context's own precision
        (float64 for fp64, float32 for the float forms); numpy arrays (host, synchronous) or
        contiguous CUDA tensors, of the state's size."""
        host = isinstance(u_in, np.ndarray)
        if host != isinstance(u_out, np.ndarray):
            raise TypeError("u_in and u_out must both be host arrays or both device tensors")
        n = self.E * self.Np * self.M * self.S
        want = "float64" if self.fp64 else "float32"
        for a in (u_in, u_out):
            if host:
                ok = str(a.dtype) == want and a.flags.c_contiguous and a.size == n
            else:
                ok = a.is_cuda and str(a.dtype) == "torch." + want and a.is_contiguous() and a.numel() == n
            if not ok:
                raise ValueError(f"states must be contiguous {want} arrays of {n} values")
        pin, pout = (u_in.ctypes.data, u_out.ctypes.data) if host else (_ptr(u_in), _ptr(u_out))
        self._ck(self.lib.fr_sg_advance_native(self.h, pin, pout, HOST if host else DEVICE, float(dt), int(nsteps),
                                               1 if graph else 0), "advance_native")
        return u_out

    def project(self, u0, uhat):
        """fr_sg_project: device float64 tensors [E, Np, Q, S] -> [E, Np, M, S]."""
        self._ck(self.lib.fr_sg_project(self.h, _ptr(u0), _ptr(uhat), DEVICE), "project")

    def project_transpose(self, gbar, g):
        """fr_sg_project_transpose: device float64 tensors [E, Np, M, S] -> [E, Np, Q, S]."""
        self._ck(self.lib.fr_sg_project_transpose(self.h, _ptr(gbar), _ptr(g), DEVICE), "project_transpose")

    def rk4_step(self, dt, nsteps=1, graph=True):
        """Classical RK4 steps (the advection study's integrator)."""
        self._ck(self.lib.fr_sg_rk4_step(self.h, float(dt), int(nsteps), int(bool(graph))), "rk4_step")

    def set_timing_events(self, before_limiter=None, before_stage=None, after_stage=None):
        """fr_sg_set_timing_events: torch.cuda.Event objects (or None) that stage() records
        around its limiter and stage-kernel launches."""
        def h(ev):
            return ctypes.c_void_p(ev.cuda_event if ev is not None else 0)
        self._ck(self.lib.fr_sg_set_timing_events(self.h, h(before_limiter), h(before_stage), h(after_stage)),
                 "set_timing_events")

    def stage(self, stage, dt):
        self._ck(self.lib.fr_sg_stage(self.h, int(stage), float(dt)), "stage")

    def filter(self, dt):
        self._ck(self.lib.fr_sg_filter(self.h, float(dt)), "filter")

    def limit(self):
        self._ck(self.lib.fr_sg_limit(self.h), "limit")

    def moments(self, mean=None, var=None):
        if mean is None:
            mean = np.zeros((self.E, self.Np, self.S))
            var = np.zeros((self.E, self.Np, self.S))
            self._ck(self.lib.fr_sg_moments(self.h, _ptr(mean), _ptr(var), HOST), "moments")
        else:
            where = HOST if isinstance(mean, np.ndarray) else DEVICE
            self._ck(self.lib.fr_sg_moments(self.h, _ptr(mean), _ptr(var), where), "moments")
        return mean, var

    def cell_means(self):
        """fr_sg_cell_means: FP64 element means of the gPC mean mode, [E, S] (host)."""
        out = np.zeros((self.E, self.S))
        self._ck(self.lib.fr_sg_cell_means(self.h, _ptr(out), HOST), "cell_means")
        return out

    def cfl_dt(self, cfl):
        dt = ctypes.c_double()
        self._ck(self.lib.fr_sg_cfl_dt(self.h, float(cfl), ctypes.byref(dt)), "cfl_dt")
        return dt.value

    def decisions(self):
        flags = np.zeros((3, self.E), dtype=np.uint8)
        beta = np.zeros((3, self.E))
        self._ck(self.lib.fr_sg_get_decisions(self.h, _ptr(flags), _ptr(beta)), "get_decisions")
        return flags.astype(bool), beta

    def set_replay(self, flags):
        if flags is None:
            self._ck(self.lib.fr_sg_set_replay(self.h, None, 0), "set_replay")
            return
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8).reshape(-1, self.E))
        self._ck(self.lib.fr_sg_set_replay(self.h, _ptr(f), f.shape[0]), "set_replay")

    def check(self):
        self._ck(self.lib.fr_sg_check(self.h), "check")

    def forward_record(self, dt, nsteps, checkpoint_every=16):
        self._ck(self.lib.fr_sg_forward_record(self.h, float(dt), int(nsteps), int(checkpoint_every)),
                 "forward_record")

    def adjoint(self, lambda_T, grad_u0):
        """lambda_T, grad_u0: device float64 tensors [E, Np, M, S]."""
        self._ck(self.lib.fr_sg_adjoint(self.h, _ptr(lambda_T), _ptr(grad_u0)), "adjoint")

    def set_tile(self, te):
        """Elements per CTA of the stage kernel (0 = automatic); returns the tile in use."""
        out = ctypes.c_int()
        self._ck(self.lib.fr_sg_set_tile(self.h, int(te), ctypes.byref(out)), "set_tile")
        return out.value

    def launch_count(self):
        return int(self.lib.fr_sg_launch_count(self.h))

    def autotune(self, reps=5):
        """Pick the fastest stage-kernel layout and tile (cached per problem shape)."""
        v, t = ctypes.c_int(), ctypes.c_int()
        self._ck(self.lib.fr_sg_autotune(self.h, int(reps), ctypes.byref(v), ctypes.byref(t)), "autotune")
        return v.value, t.value

    def test_fused_wait(self, wait_cycles=0, hold_tile=-1):
        """fr_sg_test_fused_wait: bound the one-launch step's neighbour wait, and optionally hold
        one tile's launch counter so that its next wait runs out."""
        self._ck(self.lib.fr_sg_test_fused_wait(self.h, int(wait_cycles), int(hold_tile)), "test_fused_wait")

    def set_variant(self, variant):
        """1D layout: 0 thread per (z-node, element), 1 thread per (z-node, point, element),
        2 one cooperative launch per SSP-RK3 step, 3 one launch per step with each tile
        recomputing a three-element halo (2 and 3: no limiter)."""
        self._ck(self.lib.fr_sg_set_variant(self.h, int(variant)), "set_variant")


class Batch:
    """fr_sg_batch_*: many 1D Solver objects advanced by one persistent launch per stage."""

    def __init__(self, solvers, stream=None):
        self.lib = load_library()
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        h = ctypes.c_void_p()
        st = self.lib.fr_sg_batch_create(arr, len(self.solvers), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != OK:
            raise FrsgError(st, "fr_sg_batch_create rejected the members (details on stderr)")
        self.h = h

    def rk_step(self, dts, nsteps=1, graph=True):
        d = np.ascontiguousarray(dts, dtype=np.float64)
        st = self.lib.fr_sg_batch_rk_step(self.h, _ptr(d), int(nsteps), int(bool(graph)))
        if st != OK:
            raise FrsgError(st, "fr_sg_batch_rk_step failed")

    def forward_record(self, dts, nsteps, checkpoint_every):
        """fr_sg_batch_forward_record: nsteps steps of every member, checkpoints every
        checkpoint_every steps and the decisions of every stage kept on the device."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        st = self.lib.fr_sg_batch_forward_record(self.h, _ptr(d), int(nsteps), int(checkpoint_every))
        if st != OK:
            raise FrsgError(st, "fr_sg_batch_forward_record failed (details on stderr)")

    def forward_replay(self, nsteps):
        """fr_sg_batch_forward_replay: nsteps steps from the members' current states with the
        recorded step sizes and filter decisions."""
        st = self.lib.fr_sg_batch_forward_replay(self.h, int(nsteps))
        if st != OK:
            raise FrsgError(st, "fr_sg_batch_forward_replay failed (details on stderr)")

    @staticmethod
    def _ptr_table(tensors):
        for t in tensors:
            if not (t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous()):
                raise ValueError("cotangents and gradients must be contiguous CUDA float64 tensors")
        return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])

    def adjoint(self, lambda_sets, grad_sets):
        """fr_sg_batch_adjoint for len(lambda_sets) cotangent sets; lambda_sets[c][i] and
        grad_sets[c][i] are member i's tensors of the state's shape (CUDA float64)."""
        n = len(self.solvers)
        if len(lambda_sets) != len(grad_sets) or any(len(x) != n for x in list(lambda_sets) + list(grad_sets)):
            raise ValueError("one tensor per member in every set")
        for c in range(len(lambda_sets)):
            for i, sv in enumerate(self.solvers):
                for t in (lambda_sets[c][i], grad_sets[c][i]):
                    if tuple(t.shape) != tuple(sv.state_shape):
                        raise ValueError(f"member {i}: tensor shape {tuple(t.shape)} != {tuple(sv.state_shape)}")
        lam = self._ptr_table([t for ts in lambda_sets for t in ts])
        grd = self._ptr_table([t for ts in grad_sets for t in ts])
        st = self.lib.fr_sg_batch_adjoint(self.h, len(lambda_sets), lam, grd)
        if st != OK:
            raise FrsgError(st, "fr_sg_batch_adjoint failed (details on stderr)")

    def integral_moments(self, dmean=None, dvar=None):
        """fr_sg_batch_integral_moments: [n, 2] array of (E[I], Var[I]), I the integral of u over
        the domain; gradients into the given per-member tensors (CUDA float64, state shape)."""
        n = len(self.solvers)
        q = np.empty((n, 2), dtype=np.float64)
        tabs = []
        for g in (dmean, dvar):
            if g is None:
                tabs.append(None)
                continue
            if len(g) != n or any(tuple(t.shape) != tuple(sv.state_shape) for t, sv in zip(g, self.solvers)):
                raise ValueError("one gradient tensor of the state's shape per member")
            tabs.append(self._ptr_table(list(g)))
        st = self.lib.fr_sg_batch_integral_moments(self.h, _ptr(q), tabs[0], tabs[1])
        if st != OK:
            raise FrsgError(st, "fr_sg_batch_integral_moments failed (details on stderr)")
        return q

    def info(self):
        nt, gr, sm = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        self.lib.fr_sg_batch_info(self.h, ctypes.byref(nt), ctypes.byref(gr), ctypes.byref(sm))
        return dict(tiles=nt.value, grid=gr.value, smem=sm.value)

    def launch_count(self):
        return int(self.lib.fr_sg_batch_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.fr_sg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
