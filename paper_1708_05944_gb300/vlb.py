"""Thin ctypes binding of libvlb (include/vlb.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
and torch tensors to pointers and status codes to exceptions.  Importing it
without the compiled library raises immediately: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvlb.so")

VLB_OK, VLB_ERR_INVALID, VLB_ERR_UNSUPPORTED, VLB_ERR_CUDA, VLB_ERR_NONFINITE, VLB_ERR_TIMEOUT, VLB_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
VLB_FULL, VLB_HALF = 0, 1
VLB_FP64, VLB_FP32_BULK = 0, 1
VLB_BGK, VLB_SHAKHOV = 0, 1
VLB_CHI, VLB_FTILDE, VLB_CARTESIAN = 0, 1, 2
VLB_TAU_KN_OVER_NT, VLB_TAU_AOKI, VLB_TAU_KN_OVER_N = 0, 1, 2

_STATUS = {VLB_ERR_INVALID: "INVALID", VLB_ERR_UNSUPPORTED: "UNSUPPORTED", VLB_ERR_CUDA: "CUDA",
           VLB_ERR_NONFINITE: "NONFINITE", VLB_ERR_TIMEOUT: "TIMEOUT", VLB_ERR_STATE: "STATE"}


class VlbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libvlb {_STATUS.get(status, status)}: {msg}")
        self.status = status


class vlb_model(C.Structure):
    _fields_ = [("kind", C.c_int * 2), ("N", C.c_int * 2), ("Q", C.c_int * 2)]


class vlb_couette_grid(C.Structure):
    _fields_ = [("n_cells", C.c_int), ("r_in", C.c_double), ("r_out", C.c_double),
                ("stretch_A", C.c_double), ("stretch_delta", C.c_double),
                ("cell_begin", C.c_int), ("cell_end", C.c_int)]


class vlb_channel_grid(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("n_xi", C.c_int), ("xi_in", C.c_double), ("xi_out", C.c_double),
                ("re_c", C.c_double), ("stretch_A", C.c_double)]


class vlb_wall(C.Structure):
    _fields_ = [("u_tangential", C.c_double), ("T", C.c_double)]


EXPORTS = {
    "vlb_parse_model": (C.c_int, [C.c_char_p, C.POINTER(vlb_model)]),
    "vlb_quadrature": (C.c_int, [C.POINTER(vlb_model), C.c_int, C.c_void_p, C.c_void_p]),
    "vlb_axis_tables": (C.c_int, [C.POINTER(vlb_model), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vlb_axis_nodes": (C.c_int, [C.POINTER(vlb_model), C.c_int]),
    "vlb_create_couette": (C.c_int, [C.POINTER(vlb_model), C.c_int, C.c_int, C.POINTER(vlb_couette_grid),
                                     C.POINTER(vlb_wall), C.POINTER(vlb_wall), C.POINTER(C.c_double),
                                     C.POINTER(C.c_int), C.c_void_p, C.POINTER(C.c_void_p)]),
    "vlb_create_channel": (C.c_int, [C.POINTER(vlb_model), C.c_int, C.POINTER(vlb_channel_grid), C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_void_p, C.POINTER(C.c_void_p)]),
    "vlb_channel_variants": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "vlb_channel_variant_tensor_cores": (C.c_int, [C.c_void_p, C.c_int]),
    "vlb_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "vlb_set_walls": (C.c_int, [C.c_void_p, C.POINTER(vlb_wall), C.POINTER(vlb_wall)]),
    "vlb_init_equilibrium": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double]),
    "vlb_set_knudsen": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "vlb_set_channel_reservoirs": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double]),
    "vlb_set_channel_flow_rate": (C.c_int, [C.c_void_p, C.c_double]),
    "vlb_set_collision": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "vlb_set_formulation": (C.c_int, [C.c_void_p, C.c_int]),
    "vlb_channel_postprocess": (C.c_int, [C.c_void_p] + [C.c_void_p] * 5),
    "vlb_set_f": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "vlb_read_f": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "vlb_stage": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "vlb_step": (C.c_int, [C.c_void_p, C.c_double, C.c_longlong]),
    "vlb_set_dt": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "vlb_read_moments": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6 + [C.c_int]),
    "vlb_wall_density": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vlb_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vlb_residual_sums": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vlb_halo_bytes": (C.c_longlong, [C.c_void_p]),
    "vlb_read_edge": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "vlb_write_halo": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "vlb_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "vlb_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "vlb_variants": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "vlb_set_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "vlb_autotune": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "vlb_step_static_scratch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_longlong]),
    "vlb_step_graph": (C.c_int, [C.c_void_p, C.c_double, C.c_longlong]),
    "vlb_run_to_steady": (C.c_int, [C.c_void_p, C.c_double, C.c_longlong, C.c_double, C.c_longlong,
                                    C.POINTER(C.c_longlong), C.c_void_p, C.c_void_p]),
    "vlb_init_from_moments": (C.c_int, [C.c_void_p] + [C.c_void_p] * 5 + [C.c_int]),
    "vlb_no_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "vlb_no_num_params": (C.c_longlong, [C.c_void_p]),
    "vlb_no_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vlb_no_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vlb_no_set_target_scaling": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vlb_no_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "vlb_no_loss_and_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                       C.c_void_p]),
    "vlb_no_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                    C.POINTER(C.c_double)]),
    "vlb_no_last_error": (C.c_char_p, [C.c_void_p]),
    "vlb_no_destroy": (None, [C.c_void_p]),
    "vlb_kernel_launches": (C.c_longlong, [C.c_void_p]),
    "vlb_peak_fp64": (C.c_int, [C.POINTER(C.c_double)]),
    "vlb_last_error": (C.c_char_p, [C.c_void_p]),
    "vlb_destroy": (None, [C.c_void_p]),
}


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libvlb is not built ({path} missing): run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _check(status, ctx=None):
    if status != VLB_OK:
        msg = _lib.vlb_last_error(ctx)
        raise VlbError(status, msg.decode() if msg else "")


def _ptr(a):
    """Pointer of a C-contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _on_device(a):
    return int(hasattr(a, "is_cuda") and a.is_cuda)


def vlb_parse_model(text: str) -> vlb_model:
    m = vlb_model()
    _check(_lib.vlb_parse_model(text.encode(), C.byref(m)))
    return m


def vlb_axis_nodes(model: vlb_model, axis: int) -> int:
    n = _lib.vlb_axis_nodes(C.byref(model), axis)
    if n < 0:
        _check(n)
    return n


def vlb_quadrature(model: vlb_model, axis: int):
    nq = vlb_axis_nodes(model, axis)
    p, w = np.zeros(nq), np.zeros(nq)
    _check(_lib.vlb_quadrature(C.byref(model), axis, _ptr(p), _ptr(w)))
    return p, w


def vlb_axis_tables(model: vlb_model, axis: int):
    nq = vlb_axis_nodes(model, axis)
    p, w, K, Kt = np.zeros(nq), np.zeros(nq), np.zeros((nq, nq)), np.zeros((nq, nq))
    _check(_lib.vlb_axis_tables(C.byref(model), axis, _ptr(p), _ptr(w), _ptr(K), _ptr(Kt)))
    return p, w, K, Kt


class _Context:
    """Operations shared by every context kind (Couette instances, channel)."""

    def close(self):
        if getattr(self, "h", None):
            _lib.vlb_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def _sizes(self):
        cells, nv, nb = C.c_longlong(), C.c_int(), C.c_longlong()
        _check(_lib.vlb_sizes(self.h, C.byref(cells), C.byref(nv), C.byref(nb)), self.h)
        self.total_cells, self.nvel, self.f_bytes = cells.value, nv.value, nb.value
        self.nq = (vlb_axis_nodes(self.model, 0), vlb_axis_nodes(self.model, 1))
        self.dtype = np.float64 if self.precision == VLB_FP64 else np.float32

    def f_shape(self):
        return (self.total_cells, 2, self.nq[0], self.nq[1])

    def init_equilibrium(self, n0=1.0, u0=0.0, u1=0.0, T0=1.0):
        _check(_lib.vlb_init_equilibrium(self.h, n0, u0, u1, T0), self.h)

    def set_f(self, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=self.dtype)
        _check(_lib.vlb_set_f(self.h, _ptr(f), _on_device(f)), self.h)

    def read_f(self, out=None):
        if out is None:
            out = np.empty(self.f_shape(), dtype=self.dtype)
        _check(_lib.vlb_read_f(self.h, _ptr(out), _on_device(out)), self.h)
        return out

    def stage(self, dt, k):
        _check(_lib.vlb_stage(self.h, dt, k), self.h)

    def step(self, dt, nsteps=1):
        _check(_lib.vlb_step(self.h, dt, nsteps), self.h)

    def step_graph(self, dt, nsteps=1):
        _check(_lib.vlb_step_graph(self.h, dt, nsteps), self.h)

    def set_dt(self, dt):
        arr = (C.c_double * self.n_inst)(*dt)
        _check(_lib.vlb_set_dt(self.h, arr), self.h)

    def read_moments(self, full=False):
        N = self.total_cells
        n, u0, u1, T = (np.empty(N) for _ in range(4))
        Tab = np.empty((N, 3)) if full else None
        q = np.empty((N, 2)) if full else None
        _check(_lib.vlb_read_moments(self.h, _ptr(n), _ptr(u0), _ptr(u1), _ptr(T), _ptr(Tab), _ptr(q), 0), self.h)
        return (n, u0, u1, T, Tab, q) if full else (n, u0, u1, T)

    def set_collision(self, collision, prandtl=1.0):
        """vlb_set_collision: VLB_BGK, or VLB_SHAKHOV with the given Prandtl number."""
        _check(_lib.vlb_set_collision(self.h, collision, prandtl), self.h)

    def set_knudsen(self, kn, tau_mode=VLB_TAU_KN_OVER_NT):
        _check(_lib.vlb_set_knudsen(self.h, kn, tau_mode), self.h)

    def init_from_moments(self, n, u0, u1, T, q0=None):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (n, u0, u1, T)]
        q = None if q0 is None else np.ascontiguousarray(q0, dtype=np.float64)
        _check(_lib.vlb_init_from_moments(self.h, *[_ptr(a) for a in arrs], _ptr(q), 0), self.h)

    def save(self, path):
        _check(_lib.vlb_save(self.h, path.encode()), self.h)

    def load(self, path):
        _check(_lib.vlb_load(self.h, path.encode()), self.h)

    def variants(self):
        """[(cells per tile, threads, persistent)] of the stage kernel's launch shapes."""
        tc, nt, ps = (np.zeros(16, dtype=np.int32) for _ in range(3))
        n = _lib.vlb_variants(self.h, _ptr(tc), _ptr(nt), _ptr(ps), 16)
        if n < 0:
            _check(n, self.h)
        return [(int(tc[i]), int(nt[i]), int(ps[i])) for i in range(n)]

    def set_variant(self, v):
        _check(_lib.vlb_set_variant(self.h, v), self.h)

    def autotune(self, dt, reps=20):
        ch, ms = C.c_int(), C.c_double()
        _check(_lib.vlb_autotune(self.h, dt, reps, C.byref(ch), C.byref(ms)), self.h)
        return ch.value, ms.value

    def step_static_scratch(self, f_in, f_out, dt, nsteps=1):
        """vlb_step_static_scratch: f_in, f_out are device tensors in the library layout."""
        _check(_lib.vlb_step_static_scratch(self.h, _ptr(f_in), _ptr(f_out), dt, nsteps), self.h)

    def kernel_launches(self):
        return _lib.vlb_kernel_launches(self.h)


class Couette(_Context):
    """A context of circular Couette instances (vlb_create_couette)."""

    def __init__(self, model, precision, grids, inner, outer, kn, tau_mode, stream=None):
        if isinstance(model, str):
            model = vlb_parse_model(model)
        self.model = model
        self.precision = precision
        n = len(grids)
        G = (vlb_couette_grid * n)(*[vlb_couette_grid(g["n_cells"], g.get("r_in", 1.0), g.get("r_out", 2.0),
                                                      g.get("stretch_A", 0.0), g.get("stretch_delta", 0.5),
                                                      g.get("cell_begin", 0), g.get("cell_end", 0))
                                     for g in grids])
        Wi = (vlb_wall * n)(*[vlb_wall(w[0], w[1]) for w in inner])
        Wo = (vlb_wall * n)(*[vlb_wall(w[0], w[1]) for w in outer])
        K = (C.c_double * n)(*kn)
        T = (C.c_int * n)(*tau_mode)
        h = C.c_void_p()
        st = _lib.vlb_create_couette(C.byref(model), precision, n, G, Wi, Wo, K, T,
                                     C.c_void_p(stream) if stream else None, C.byref(h))
        _check(st)
        self.h = h
        self.n_inst = n
        self._sizes()

    def set_formulation(self, formulation):
        """vlb_set_formulation: VLB_CHI or VLB_FTILDE."""
        _check(_lib.vlb_set_formulation(self.h, formulation), self.h)

    def set_walls(self, inner, outer):
        n = self.n_inst
        Wi = (vlb_wall * n)(*[vlb_wall(w[0], w[1]) for w in inner])
        Wo = (vlb_wall * n)(*[vlb_wall(w[0], w[1]) for w in outer])
        _check(_lib.vlb_set_walls(self.h, Wi, Wo), self.h)

    def wall_density(self):
        nw = np.empty((self.n_inst, 2))
        _check(_lib.vlb_wall_density(self.h, _ptr(nw)), self.h)
        return nw

    def run_to_steady(self, dt, check_steps, threshold, max_steps):
        """(steps taken, last residual per instance, first converged step per instance or -1)."""
        taken = C.c_longlong()
        res = np.zeros(self.n_inst)
        conv = np.zeros(self.n_inst, dtype=np.int64)
        _check(_lib.vlb_run_to_steady(self.h, dt, check_steps, threshold, max_steps, C.byref(taken), _ptr(res),
                                      _ptr(conv)), self.h)
        return taken.value, res, conv

    def residual(self):
        a, b, c = (np.empty(self.n_inst) for _ in range(3))
        _check(_lib.vlb_residual(self.h, _ptr(a), _ptr(b), _ptr(c)), self.h)
        return a, b, c

    def residual_sums(self):
        """vlb_residual_sums: the squared norms (u, n, T) per instance, before the root."""
        a, b, c = (np.empty(self.n_inst) for _ in range(3))
        _check(_lib.vlb_residual_sums(self.h, _ptr(a), _ptr(b), _ptr(c)), self.h)
        return a, b, c

    def halo_bytes(self):
        n = _lib.vlb_halo_bytes(self.h)
        if n < 0:
            _check(int(n), self.h)
        return int(n)

    def read_edge(self, inst, end, out=None):
        """vlb_read_edge into out (a host uint8 array or a device tensor of halo_bytes bytes)."""
        if out is None:
            out = np.empty(self.halo_bytes(), dtype=np.uint8)
        _check(_lib.vlb_read_edge(self.h, inst, end, _ptr(out), _on_device(out)), self.h)
        return out

    def write_halo(self, inst, end, rows):
        _check(_lib.vlb_write_halo(self.h, inst, end, _ptr(rows), _on_device(rows)), self.h)


class Channel(_Context):
    """A gradually expanding channel context (vlb_create_channel)."""

    def __init__(self, model, precision, n_lambda, n_xi, kn, n_in=2.0, n_out=1.0, T0=1.0, xi_in=-10.0, xi_out=40.0,
                 re_c=100.0, stretch_A=0.95, stream=None):
        if isinstance(model, str):
            model = vlb_parse_model(model)
        self.model, self.precision = model, precision
        g = vlb_channel_grid(n_lambda, n_xi, xi_in, xi_out, re_c, stretch_A)
        h = C.c_void_p()
        _check(_lib.vlb_create_channel(C.byref(model), precision, C.byref(g), kn, n_in, n_out, T0,
                                       C.c_void_p(stream) if stream else None, C.byref(h)))
        self.h = h
        self.n_inst = 1
        self.n_lambda, self.n_xi = n_lambda, n_xi
        self._sizes()

    def set_reservoirs(self, n_in, n_out, T0=1.0):
        _check(_lib.vlb_set_channel_reservoirs(self.h, n_in, n_out, T0), self.h)

    def set_formulation(self, formulation):
        """vlb_set_formulation: VLB_CHI (vielbein) or VLB_CARTESIAN (the Cartesian-split channel)."""
        _check(_lib.vlb_set_formulation(self.h, formulation), self.h)

    def set_flow_rate(self, q0):
        """vlb_set_channel_flow_rate: the paper's parabolic flow-rate ends with half-channel rate q0."""
        _check(_lib.vlb_set_channel_flow_rate(self.h, q0), self.h)

    def postprocess(self):
        """vlb_channel_postprocess: dict of ux, uy, omega (n_lambda, n_xi), psi (n_lambda + 1, n_xi)
        and pw (n_xi,), rearranged from the library's column-major order."""
        nl, nx = self.n_lambda, self.n_xi
        ux, uy, om = (np.empty(nl * nx) for _ in range(3))
        psi, pw = np.empty((nl + 1) * nx), np.empty(nx)
        _check(_lib.vlb_channel_postprocess(self.h, _ptr(ux), _ptr(uy), _ptr(psi), _ptr(om), _ptr(pw)), self.h)
        col = lambda a, rows: a.reshape(nx, rows).T.copy()
        return dict(ux=col(ux, nl), uy=col(uy, nl), omega=col(om, nl), psi=col(psi, nl + 1), pw=pw)

    def channel_variants(self):
        ts, tp, nt = (np.zeros(8, dtype=np.int32) for _ in range(3))
        n = _lib.vlb_channel_variants(self.h, _ptr(ts), _ptr(tp), _ptr(nt), 8)
        if n < 0:
            _check(n, self.h)
        return [(int(ts[i]), int(tp[i]), int(nt[i])) for i in range(n)]

    def channel_variant_tensor_cores(self, v):
        """vlb_channel_variant_tensor_cores: whether launch shape v contracts the force on the tensor cores."""
        r = _lib.vlb_channel_variant_tensor_cores(self.h, v)
        if r < 0:
            _check(r, self.h)
        return bool(r)

    def wall_density(self):
        nw = np.empty(self.n_xi)
        _check(_lib.vlb_wall_density(self.h, _ptr(nw)), self.h)
        return nw


class NeuralOperator:
    """The learned warm-start operator (vlb_no_*)."""

    def __init__(self, grid_points=64, width=64, modes=32, layers=4, hidden=128, stream=None):
        h = C.c_void_p()
        st = _lib.vlb_no_create(grid_points, width, modes, layers, hidden, C.c_void_p(stream) if stream else None,
                                C.byref(h))
        if st != VLB_OK:
            raise VlbError(st, "vlb_no_create failed")
        self.h = h
        self.grid_points = grid_points
        self.size = _lib.vlb_no_num_params(h)

    def _chk(self, st):
        if st != VLB_OK:
            raise VlbError(st, (_lib.vlb_no_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            _lib.vlb_no_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.size
        self._chk(_lib.vlb_no_set_params(self.h, _ptr(t)))

    def get_params(self):
        t = np.empty(self.size, dtype=np.float32)
        self._chk(_lib.vlb_no_get_params(self.h, _ptr(t)))
        return t

    def set_target_scaling(self, mean, std):
        m = np.ascontiguousarray(mean, dtype=np.float64)
        s = np.ascontiguousarray(std, dtype=np.float64)
        self._chk(_lib.vlb_no_set_target_scaling(self.h, _ptr(m), _ptr(s)))

    def predict(self, cond):
        c = np.ascontiguousarray(cond, dtype=np.float64)
        out = np.empty((c.shape[0], self.grid_points, 4))
        self._chk(_lib.vlb_no_predict(self.h, _ptr(c), c.shape[0], _ptr(out)))
        return out

    def loss_and_grad(self, cond, targets):
        c = np.ascontiguousarray(cond, dtype=np.float64)
        t = np.ascontiguousarray(targets, dtype=np.float64)
        loss = C.c_double()
        g = np.empty(self.size, dtype=np.float32)
        self._chk(_lib.vlb_no_loss_and_grad(self.h, _ptr(c), _ptr(t), c.shape[0], C.byref(loss), _ptr(g)))
        return loss.value, g

    def train_step(self, cond, targets, lr):
        c = np.ascontiguousarray(cond, dtype=np.float64)
        t = np.ascontiguousarray(targets, dtype=np.float64)
        loss = C.c_double()
        self._chk(_lib.vlb_no_train_step(self.h, _ptr(c), _ptr(t), c.shape[0], lr, C.byref(loss)))
        return loss.value


def vlb_peak_fp64():
    """vlb_peak_fp64: measured FP64 fma throughput of the current device, TFLOP/s."""
    t = C.c_double()
    _check(_lib.vlb_peak_fp64(C.byref(t)))
    return t.value
