"""ctypes wrapper of the C oracle (test infrastructure only).

The oracle is a plain FP64 CPU implementation of Algorithm 1 of the paper
(see oracle.c for the readings it takes).  This wrapper converts a workload
description (any object with the attributes of ``inputs.Case``) into the
oracle's own configuration struct.  It imports nothing from the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

KIND = {"periodic": 0, "dirichlet": 1, "neumann": 2}
SHAPE = {"const": 0, "linear_ramp": 1, "sin2_ramp": 2, "half_sine": 3, "ricker": 4, "disp_ramp": 5}
MODEL = {"svk": 0, "nh": 1, "le": 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (FP contraction off)."""
    with _LOCK:
        fresh = os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
        if force or not fresh:
            tmp = _SO + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                   "-Wall", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _SO)
    return _SO


class _Edge(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("shape", ctypes.c_int), ("amp", ctypes.c_double * 2),
                ("t0", ctypes.c_double), ("t1", ctypes.c_double), ("s", ctypes.c_double),
                ("time_unit", ctypes.c_int)]


class _Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("tau", ctypes.c_double),
                ("model", ctypes.c_int), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho0", ctypes.c_double), ("body", ctypes.c_double * 2), ("edge", _Edge * 4),
                ("order", ctypes.c_int), ("extrap", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _LIB
    if _LIB is None:
        build()
        L = ctypes.CDLL(_SO)
        L.ora_create.restype = ctypes.c_void_p
        L.ora_create.argtypes = [ctypes.POINTER(_Config), _dp, _dp]
        L.ora_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.ora_iteration.restype = ctypes.c_long
        L.ora_iteration.argtypes = [ctypes.c_void_p]
        L.ora_fields.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.ora_destroy.argtypes = [ctypes.c_void_p]
        L.ora_threads.restype = ctypes.c_int
        L.ora_state_size.restype = ctypes.c_long
        L.ora_state_size.argtypes = [ctypes.c_void_p]
        L.ora_get_state.argtypes = [ctypes.c_void_p, _dp]
        L.ora_set_state.argtypes = [ctypes.c_void_p, _dp]
        L.ora_params.argtypes = [ctypes.POINTER(_Config), _dp]
        L.ora_first_piola.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.ora_pi_of_h.argtypes = [ctypes.c_double, _dp, _dp]
        L.ora_equilibrium.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        L.ora_forcing.argtypes = [ctypes.c_double, _dp, _dp]
        L.ora_gradient.argtypes = [ctypes.POINTER(_Config), _dp, _dp]
        L.ora_load.argtypes = [ctypes.POINTER(_Config), ctypes.c_int, ctypes.c_long, _dp]
        L.ora_grid_error.argtypes = [ctypes.c_long, _dp, _dp, _dp]
        L.ora_wall_value.restype = ctypes.c_double
        L.ora_wall_value.argtypes = [ctypes.POINTER(_Config), _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int]
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


ORDER = {"text": 0, "listing": 1}
EXTRAP = {"own": 0, "linear": 1}


def config(case, order: str = "text") -> _Config:
    c = _Config()
    c.order = ORDER[order]
    c.extrap = EXTRAP[getattr(case, "extrap", "own")]
    c.nx, c.ny = int(case.nx), int(case.ny)
    c.dx = float(case.dx if case.dx is not None else 1.0 / case.ny)
    c.tau = float(case.tau)
    c.model = MODEL[case.model]
    c.E, c.nu, c.rho0 = float(case.E), float(case.nu), float(case.rho0)
    c.body[0], c.body[1] = float(case.body[0]), float(case.body[1])
    for k, e in enumerate(case.edges):
        c.edge[k].type = KIND[e.kind]
        c.edge[k].shape = SHAPE[e.shape]
        c.edge[k].amp[0], c.edge[k].amp[1] = float(e.amp[0]), float(e.amp[1])
        c.edge[k].t0, c.edge[k].t1, c.edge[k].s = float(e.t0), float(e.t1), float(e.s)
        c.edge[k].time_unit = {"steps": 0, "time": 1}[getattr(e, "unit", "steps")]
    return c


def params(case) -> dict:
    out = np.zeros(5)
    lib().ora_params(ctypes.byref(config(case)), _ptr(out))
    return dict(zip(("mu", "lam", "cs", "c", "dt"), out.tolist()))


class OracleSim:
    """One simulation on the CPU oracle.  u0, v0: [ny, nx, 2] float64 or None."""

    def __init__(self, case, u0=None, v0=None, order: str = "text"):
        self.case = case
        self._cfg = config(case, order)
        shape = (case.ny, case.nx, 2)
        self._u0 = None if u0 is None else _f64(np.asarray(u0), shape)
        self._v0 = None if v0 is None else _f64(np.asarray(v0), shape)
        L = lib()
        self._h = L.ora_create(ctypes.byref(self._cfg),
                               _ptr(self._u0) if self._u0 is not None else None,
                               _ptr(self._v0) if self._v0 is not None else None)
        if not self._h:
            raise ValueError(f"oracle rejected case {case.name!r}")

    def step(self, n: int) -> None:
        lib().ora_step(self._h, int(n))

    @property
    def iteration(self) -> int:
        return int(lib().ora_iteration(self._h))

    def fields(self):
        """(u, v, P): [ny, nx, 2], [ny, nx, 2], [ny, nx, 4] float64."""
        ny, nx = self.case.ny, self.case.nx
        u = np.empty((ny, nx, 2))
        v = np.empty((ny, nx, 2))
        P = np.empty((ny, nx, 4))
        lib().ora_fields(self._h, _ptr(u), _ptr(v), _ptr(P))
        return u, v, P

    def state(self) -> np.ndarray:
        """The carried state (f, u, P, Pi(H), S) as one float64 vector."""
        x = np.empty(int(lib().ora_state_size(self._h)))
        lib().ora_get_state(self._h, _ptr(x))
        return x

    def set_state(self, x) -> None:
        x = _f64(x)
        assert x.size == int(lib().ora_state_size(self._h))
        lib().ora_set_state(self._h, _ptr(x))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ora_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @staticmethod
    def threads() -> int:
        return int(lib().ora_threads())


def first_piola(model: str, lam: float, mu: float, H) -> np.ndarray:
    H = _f64(H, (4,))
    P = np.empty(4)
    lib().ora_first_piola(MODEL[model], float(lam), float(mu), _ptr(H), _ptr(P))
    return P


def pi_of_h(mu: float, H) -> np.ndarray:
    H = _f64(H, (4,))
    out = np.empty(4)
    lib().ora_pi_of_h(float(mu), _ptr(H), _ptr(out))
    return out


def equilibrium(cs: float, r: float, j, Pi) -> np.ndarray:
    j = _f64(j, (2,))
    Pi = _f64(Pi, (4,))
    out = np.empty(9)
    lib().ora_equilibrium(float(cs), float(r), _ptr(j), _ptr(Pi), _ptr(out))
    return out


def forcing(cs: float, S) -> np.ndarray:
    S = _f64(S, (2,))
    out = np.empty(9)
    lib().ora_forcing(float(cs), _ptr(S), _ptr(out))
    return out


def gradient(case, u) -> np.ndarray:
    u = _f64(u, (case.ny, case.nx, 2))
    H = np.empty((case.ny, case.nx, 4))
    lib().ora_gradient(ctypes.byref(config(case)), _ptr(u), _ptr(H))
    return H


def load(case, edge: int, k: int) -> np.ndarray:
    out = np.empty(2)
    lib().ora_load(ctypes.byref(config(case)), int(edge), int(k), _ptr(out))
    return out


WALL = {None: -1, "left": 0, "right": 1, "bottom": 2, "top": 3}


def wall_value(case, a, x: int, y: int, xwall=None, ywall=None) -> float:
    """The oracle's value of the scalar node field a[ny, nx] at node (x, y)
    carried to the named walls, as its Neumann rule does (case.extrap)."""
    a = _f64(a, (case.ny, case.nx))
    return float(lib().ora_wall_value(ctypes.byref(config(case)), _ptr(a), int(x), int(y), WALL[xwall],
                                      WALL[ywall]))


def grid_error(u, u_ref):
    """(E2, Einf) of Eq. griderror for fields [..., 2] of the same shape."""
    u = _f64(u)
    r = _f64(u_ref)
    assert u.shape == r.shape and u.shape[-1] == 2
    out = np.empty(2)
    lib().ora_grid_error(u.size // 2, _ptr(u), _ptr(r), _ptr(out))
    return float(out[0]), float(out[1])
