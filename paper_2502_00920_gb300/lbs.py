"""ctypes binding of liblbs (include/lbs.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  Importing this
module does not load the library; the first call does, and raises
``LbsError`` if ``liblbs.so`` is missing (run ``__graft_entry__.build()``).

Names follow the C ABI: ``Simulation`` wraps an ``lbs_handle``; workloads are
described by ``paper_2502_00920_gb300.inputs.Case``.  Host field arrays are
numpy float64 [ny, nx, 2] (u, v) and [ny, nx, 4] (P11, P12, P21, P22); device
arrays are torch float64 CUDA tensors of the same shapes.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbs.so")
_LOCK = threading.Lock()
_LIB = None

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, EBUSY, ENOTFOUND, ECANCELED = 0, -1, -2, -3, -4, -5, -6, -7, -8
PRECISION = {"fp64": 0, "fp32": 1, "fp16s": 2}
MODEL = {"svk": 0, "nh": 1, "le": 2}
KIND = {"periodic": 0, "dirichlet": 1, "neumann": 2}
EXTRAP = {"own": 0, "linear": 1}  # LBS_EXTRAP_OWN, LBS_EXTRAP_LINEAR
UNIT = {"steps": 0, "time": 1}
SHAPE = {"const": 0, "linear_ramp": 1, "sin2_ramp": 2, "half_sine": 3, "ricker": 4, "disp_ramp": 5}


class LbsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbs error {code}: {msg}")
        self.code = code


class Lattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double), ("tau", ctypes.c_double),
                ("precision", ctypes.c_int32), ("gscale_log2", ctypes.c_int32), ("wall_extrap", ctypes.c_int32)]


class Material(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho0", ctypes.c_double), ("body", ctypes.c_double * 2)]


class EdgeC(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("shape", ctypes.c_int32), ("amp", ctypes.c_double * 2),
                ("t0", ctypes.c_double), ("t1", ctypes.c_double), ("s", ctypes.c_double),
                ("time_unit", ctypes.c_int32)]


class Bcs(ctypes.Structure):
    _fields_ = [("edge", EdgeC * 4)]


class Monitors(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int64), ("nonfinite", ctypes.c_int64), ("max_abs_u", ctypes.c_double),
                ("momentum", ctypes.c_double * 2), ("mass", ctypes.c_double)]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); every declaration of include/lbs.h
SIGNATURES = {
    "lbs_create": (ctypes.c_int, [ctypes.POINTER(Lattice), ctypes.POINTER(Material), ctypes.POINTER(Bcs),
                                  ctypes.POINTER(_vp)]),
    "lbs_destroy": (ctypes.c_int, [_vp]),
    "lbs_set_stream": (ctypes.c_int, [_vp, _vp]),
    "lbs_set_initial": (ctypes.c_int, [_vp, _dp, _dp]),
    "lbs_set_initial_device": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbs_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lbs_sync": (ctypes.c_int, [_vp]),
    "lbs_fields": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbs_fields_device": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbs_fields_static": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbs_probe": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _dp]),
    "lbs_monitor": (ctypes.c_int, [_vp, ctypes.POINTER(Monitors)]),
    "lbs_grid_error": (ctypes.c_int, [_vp, _dp, _dp]),
    "lbs_grid_error_device": (ctypes.c_int, [_vp, ctypes.c_void_p, _dp]),
    "lbs_set_monitor_interval": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lbs_set_graph_chunk": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "lbs_set_variant": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "lbs_iteration": (ctypes.c_int64, [_vp]),
    "lbs_unstable_iteration": (ctypes.c_int64, [_vp]),
    "lbs_cfl_warning": (ctypes.c_int, [_vp]),
    "lbs_device_bytes": (ctypes.c_size_t, [_vp]),
    "lbs_launch_count": (ctypes.c_int64, [_vp]),
    "lbs_params": (ctypes.c_int, [ctypes.POINTER(Lattice), ctypes.POINTER(Material), _dp]),
    "lbs_footprint": (ctypes.c_size_t, [ctypes.POINTER(Lattice)]),
    "lbs_constitutive": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]),
    "lbs_tile_variants": (ctypes.c_int, [ctypes.c_int32, _i32p, _i32p, _i32p]),
    "lbs_tile_variant_kind": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    "lbs_tile_variant_name": (ctypes.c_char_p, [ctypes.c_int32, ctypes.c_int32]),
    "lbs_variant": (ctypes.c_int32, [_vp]),
    "lbs_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, _i32p,
                                                 ctypes.POINTER(ctypes.c_double)]),
    "lbs_checkpoint_bytes": (ctypes.c_size_t, [_vp]),
    "lbs_save": (ctypes.c_int, [_vp, ctypes.c_void_p, ctypes.c_size_t]),
    "lbs_load": (ctypes.c_int, [_vp, ctypes.c_void_p, ctypes.c_size_t]),
    "lbs_set_allocator": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbs_autotune": (ctypes.c_int, [ctypes.POINTER(Lattice), ctypes.POINTER(Material), ctypes.POINTER(Bcs),
                                    ctypes.c_int32, _i32p, ctypes.POINTER(ctypes.c_float)]),
    "lbs_autotune_handle": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "lbs_autotune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "lbs_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "lbs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbs_last_error": (ctypes.c_char_p, []),
}


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("precision", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("max_resident", ctypes.c_int32), ("queue_limit", ctypes.c_int32),
                ("preempt_after_s", ctypes.c_double), ("batch_shape", ctypes.c_int32)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int32), ("iterations", ctypes.c_int64),
                ("nsteps", ctypes.c_int64), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("swaps", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("resident", ctypes.c_int64), ("node_updates", ctypes.c_int64),
                ("busy_seconds", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t), ("hbm_budget", ctypes.c_size_t),
                ("launches", ctypes.c_int64), ("preemptions", ctypes.c_int64), ("batch_shape", ctypes.c_int32),
                ("batch_tx", ctypes.c_int32), ("batch_ty", ctypes.c_int32), ("batch_tunings", ctypes.c_int64)]


# include/lbs_serve.h
SERVE_SIGNATURES = {
    "lbs_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]),
    "lbs_submit": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), ctypes.POINTER(Material), ctypes.POINTER(Bcs),
                                  ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]),
    "lbs_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(TicketInfo)]),
    "lbs_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double]),
    "lbs_result": (ctypes.c_int, [_vp, ctypes.c_uint64, _dp, _dp, _dp]),
    "lbs_server_drain": (ctypes.c_int, [_vp, ctypes.c_double]),
    "lbs_cancel": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "lbs_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)]),
    "lbs_server_destroy": (ctypes.c_int, [_vp]),
}


def lib():
    """Load liblbs.so (once).  Raises LbsError if it has not been built."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise LbsError(ECUDA, f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in {**SIGNATURES, **SERVE_SIGNATURES}.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def check(rc: int) -> int:
    if rc != OK:
        msg = lib().lbs_last_error().decode(errors="replace")
        raise LbsError(rc, msg or lib().lbs_strerror(rc).decode())
    return rc


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def structs(case):
    """(Lattice, Material, Bcs) of a Case."""
    lat = Lattice(int(case.nx), int(case.ny), float(case.dx if case.dx is not None else 1.0 / case.ny),
                  float(case.tau), PRECISION[case.precision], int(getattr(case, "gscale_log2", 0) or 0),
                  EXTRAP[getattr(case, "extrap", "own")])
    mat = Material(MODEL[case.model], float(case.E), float(case.nu), float(case.rho0),
                   (ctypes.c_double * 2)(float(case.body[0]), float(case.body[1])))
    bcs = Bcs()
    for k, e in enumerate(case.edges):
        bcs.edge[k] = EdgeC(KIND[e.kind], SHAPE[e.shape], (ctypes.c_double * 2)(float(e.amp[0]), float(e.amp[1])),
                            float(e.t0), float(e.t1), float(e.s), UNIT[getattr(e, "unit", "steps")])
    return lat, mat, bcs


def params(case) -> dict:
    lat, mat, _ = structs(case)
    out = np.zeros(5)
    check(lib().lbs_params(ctypes.byref(lat), ctypes.byref(mat), _ptr(out)))
    return dict(zip(("mu", "lam", "cs", "c", "dt"), out.tolist()))


def footprint(case) -> int:
    lat, _, _ = structs(case)
    return int(lib().lbs_footprint(ctypes.byref(lat)))


def constitutive(model: str, lam: float, mu: float, H):
    """(P, N) of the kernels' constitutive formulas, evaluated on the host."""
    H = np.ascontiguousarray(H, dtype=np.float64).reshape(4)
    P = np.empty(4)
    N = np.empty(4)
    check(lib().lbs_constitutive(MODEL[model], float(lam), float(mu), _ptr(H), _ptr(P), _ptr(N)))
    return P, N


def tile_variants(precision: str = "fp32"):
    n = ctypes.c_int32()
    tx = (ctypes.c_int32 * 16)()
    ty = (ctypes.c_int32 * 16)()
    check(lib().lbs_tile_variants(PRECISION[precision], ctypes.byref(n), tx, ty))
    return [(tx[i], ty[i]) for i in range(n.value)]


def autotune(case, steps: int = 20):
    """(best variant, per-variant ms per iteration) for a Case (cached per configuration)."""
    lat, mat, bcs = structs(case)
    best = ctypes.c_int32()
    ms = (ctypes.c_float * 16)()
    check(lib().lbs_autotune(ctypes.byref(lat), ctypes.byref(mat), ctypes.byref(bcs), int(steps), ctypes.byref(best), ms))
    return best.value, [ms[i] for i in range(len(tile_variants(case.precision)))]


def autotune_save(path: str):
    check(lib().lbs_autotune_save(str(path).encode()))


def autotune_load(path: str):
    check(lib().lbs_autotune_load(str(path).encode()))


def tile_variant_kind(precision: str, variant: int) -> str:
    k = lib().lbs_tile_variant_kind(PRECISION[precision], int(variant))
    if k < 0:
        check(k)
    return "tma" if k == 1 else "global"


def selftest_bounded_wait(tx_bytes: int, polls: int):
    """(timed_out, seconds) of one bounded wait on a barrier armed for
    tx_bytes that never arrive (see lbs_selftest_bounded_wait)."""
    out, sec = ctypes.c_int32(), ctypes.c_double()
    check(lib().lbs_selftest_bounded_wait(int(tx_bytes), int(polls), ctypes.byref(out), ctypes.byref(sec)))
    return bool(out.value), sec.value


def tile_variant_name(precision: str, variant: int) -> str:
    """Name of the kernel that updates the variant's interior tiles."""
    n = lib().lbs_tile_variant_name(PRECISION[precision], int(variant))
    if n is None:
        raise LbsError(EINVAL, f"unknown tile variant {variant} for {precision}")
    return n.decode()


def _dev_ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("device fields must be contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


class Simulation:
    """One lattice on the GPU (an lbs_handle)."""

    def __init__(self, case, u0=None, v0=None, stream=None, graph_chunk: int | None = None,
                 monitor_interval: int | None = None, variant: int | None = None):
        self.case = case
        self._lat, self._mat, self._bcs = structs(case)
        h = _vp()
        check(lib().lbs_create(ctypes.byref(self._lat), ctypes.byref(self._mat), ctypes.byref(self._bcs),
                               ctypes.byref(h)))
        self._h = h
        if stream is not None:
            self.set_stream(stream)
        if graph_chunk is not None:
            check(lib().lbs_set_graph_chunk(self._h, int(graph_chunk)))
        if monitor_interval is not None:
            check(lib().lbs_set_monitor_interval(self._h, int(monitor_interval)))
        if variant == "auto":
            check(lib().lbs_autotune_handle(self._h, 20))
        elif variant is not None:
            check(lib().lbs_set_variant(self._h, int(variant)))
        if u0 is not None or v0 is not None:
            self.set_initial(u0, v0)

    # -- life cycle
    def close(self):
        if getattr(self, "_h", None):
            lib().lbs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (own stream)."""
        raw = getattr(stream, "cuda_stream", stream)
        check(lib().lbs_set_stream(self._h, _vp(raw) if raw else None))

    def set_initial(self, u0=None, v0=None):
        """Host (numpy) or device (torch CUDA) initial displacement / velocity."""
        dev = any(getattr(a, "is_cuda", False) for a in (u0, v0) if a is not None)
        if dev:
            check(lib().lbs_set_initial_device(self._h, _dev_ptr(u0), _dev_ptr(v0)))
            return
        shape = (self.case.ny, self.case.nx, 2)
        self._u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(shape)
        self._v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64).reshape(shape)
        check(lib().lbs_set_initial(self._h, _ptr(self._u0) if self._u0 is not None else None,
                                    _ptr(self._v0) if self._v0 is not None else None))

    # -- stepping
    def step(self, n: int):
        check(lib().lbs_step(self._h, int(n)))

    def sync(self):
        check(lib().lbs_sync(self._h))

    def set_graph_chunk(self, k: int):
        check(lib().lbs_set_graph_chunk(self._h, int(k)))

    def set_monitor_interval(self, m: int):
        check(lib().lbs_set_monitor_interval(self._h, int(m)))

    def set_variant(self, v: int):
        check(lib().lbs_set_variant(self._h, int(v)))

    @property
    def variant(self) -> int:
        return int(lib().lbs_variant(self._h))

    # -- checkpoint / resume
    def save(self) -> np.ndarray:
        """The state (g, u, boundary side array, iteration) as a uint8 array."""
        buf = np.empty(int(lib().lbs_checkpoint_bytes(self._h)), dtype=np.uint8)
        check(lib().lbs_save(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes))
        return buf

    def load(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lib().lbs_load(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes))

    # -- outputs
    def fields(self, u=True, v=True, P=True):
        """Host copies of u, v, P.  Each argument is True (allocate), False
        (skip) or a C-contiguous float64 array of the right shape to fill
        (e.g. a view of pinned memory)."""
        ny, nx = self.case.ny, self.case.nx
        out = []
        for want, w in ((u, 2), (v, 2), (P, 4)):
            if isinstance(want, np.ndarray):
                if want.shape != (ny, nx, w) or want.dtype != np.float64 or not want.flags.c_contiguous:
                    raise ValueError("field buffer has the wrong shape or layout")
                out.append(want)
            else:
                out.append(np.empty((ny, nx, w)) if want else None)
        check(lib().lbs_fields(self._h, *[_ptr(a) if a is not None else None for a in out]))
        return tuple(out)

    def fields_static(self, u=True, v=True, P=True):
        """As fields(), through lbs_fields_static: no device memory is
        allocated (rows are staged through a fixed 8 MiB device array)."""
        ny, nx = self.case.ny, self.case.nx
        out = [np.empty((ny, nx, w)) if want else None for want, w in ((u, 2), (v, 2), (P, 4))]
        check(lib().lbs_fields_static(self._h, *[_ptr(a) if a is not None else None for a in out]))
        return tuple(out)

    def fields_device(self, u=None, v=None, P=None):
        check(lib().lbs_fields_device(self._h, _dev_ptr(u), _dev_ptr(v), _dev_ptr(P)))

    def probe(self, nodes):
        idx = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1)
        out = np.empty((idx.size, 2))
        check(lib().lbs_probe(self._h, int(idx.size), idx.ctypes.data_as(_i32p), _ptr(out)))
        return out

    def grid_error(self, u_ref) -> tuple:
        """(E2, Einf) of the current u against u_ref (Eq. griderror): a host
        array [ny, nx, 2] or a device tensor of that shape (float64)."""
        out = np.empty(2)
        if hasattr(u_ref, "data_ptr"):
            check(lib().lbs_grid_error_device(self._h, _dev_ptr(u_ref), _ptr(out)))
        else:
            a = np.ascontiguousarray(u_ref, dtype=np.float64)
            check(lib().lbs_grid_error(self._h, _ptr(a), _ptr(out)))
        return float(out[0]), float(out[1])

    def monitor(self) -> dict:
        m = Monitors()
        check(lib().lbs_monitor(self._h, ctypes.byref(m)))
        return dict(iteration=m.iteration, nonfinite=m.nonfinite, max_abs_u=m.max_abs_u,
                    momentum=(m.momentum[0], m.momentum[1]), mass=m.mass)

    @property
    def iteration(self) -> int:
        return int(lib().lbs_iteration(self._h))

    @property
    def unstable_iteration(self) -> int:
        return int(lib().lbs_unstable_iteration(self._h))

    @property
    def cfl_warning(self) -> bool:
        return bool(lib().lbs_cfl_warning(self._h))

    @property
    def device_bytes(self) -> int:
        return int(lib().lbs_device_bytes(self._h))

    @property
    def launch_count(self) -> int:
        return int(lib().lbs_launch_count(self._h))


TICKET_STATES = ("queued", "running", "done", "failed")


class Server:
    """Continuous-batching server (include/lbs_serve.h)."""

    def __init__(self, precision: str = "fp32", hbm_budget: int = 0, chunk: int = 64, max_resident: int = 0,
                 queue_limit: int = 0, preempt_after_s: float = 0.0, batch_shape: int | None = None):
        """batch_shape: None lets the server time its batch tile shapes and
        pick one; 0..3 fixes one."""
        cfg = ServerConfig(int(hbm_budget), PRECISION[precision], int(chunk), int(max_resident), int(queue_limit),
                           float(preempt_after_s), 0 if batch_shape is None else int(batch_shape) + 1)
        h = _vp()
        check(lib().lbs_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.precision = precision
        self._cases = {}

    def submit(self, case) -> int:
        lat, mat, bcs = structs(case)
        t = ctypes.c_uint64()
        check(lib().lbs_submit(self._h, ctypes.byref(lat), ctypes.byref(mat), ctypes.byref(bcs), int(case.nsteps),
                               ctypes.byref(t)))
        self._cases[t.value] = case
        return t.value

    def poll(self, ticket: int) -> dict:
        info = TicketInfo()
        check(lib().lbs_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(info)))
        return dict(state=TICKET_STATES[info.state], error=info.error, iterations=info.iterations,
                    nsteps=info.nsteps, nx=info.nx, ny=info.ny, t_submit=info.t_submit, t_admit=info.t_admit,
                    t_done=info.t_done, device_bytes=info.device_bytes, swaps=info.swaps)

    def wait(self, ticket: int, timeout: float = -1.0):
        check(lib().lbs_wait(self._h, ctypes.c_uint64(ticket), float(timeout)))

    def result(self, ticket: int):
        """(u, v, P, error code) of a finished ticket (a failed one's fields as
        they stood when it stopped, its code: EUNSTABLE, ECANCELED, ENOMEM ...);
        forgets the ticket.  Raises for a ticket that is not finished or not
        known."""
        case = self._cases.pop(ticket)
        ny, nx = case.ny, case.nx
        u, v, P = np.empty((ny, nx, 2)), np.empty((ny, nx, 2)), np.empty((ny, nx, 4))
        rc = lib().lbs_result(self._h, ctypes.c_uint64(ticket), _ptr(u), _ptr(v), _ptr(P))
        if rc in (EBUSY, ENOTFOUND, EINVAL):
            self._cases[ticket] = case
            check(rc)
        return u, v, P, rc

    def cancel(self, ticket: int):
        """Cancel a ticket: a queued one leaves the queue, a running one stops
        at the next scheduling point; it ends failed with ECANCELED."""
        check(lib().lbs_cancel(self._h, ticket))

    def drain(self, timeout: float = -1.0):
        check(lib().lbs_server_drain(self._h, float(timeout)))

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().lbs_server_get_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().lbs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
