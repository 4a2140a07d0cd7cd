"""Seeded synthetic workloads for the moment-chain LBM (no method arithmetic).

This module describes *what* is simulated: lattice sizes, materials, boundary
edges, load histories and seeded initial fields.  It holds none of the
scheme's arithmetic (no moments, equilibria, stresses or time steps) and is
the only module that both the CUDA path's tests and the oracle's tests use.

Workloads follow the paper's test problems (Sect. 4: uniaxial tension, simple
shear, bending wave) at the sizes of this repository's benchmark table, plus a
periodic roofline lattice with a smooth random initial velocity.  Times are in
iterations k (t_k = k dt).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

EDGE_KINDS = ("periodic", "dirichlet", "neumann")
SHAPES = ("const", "linear_ramp", "sin2_ramp", "half_sine", "ricker", "disp_ramp")
MODELS = ("svk", "nh", "le")
PRECISIONS = ("fp64", "fp32", "fp16s")


@dataclass(frozen=True)
class Edge:
    """One lattice edge: its boundary type and the time shape of its value.

    ``kind`` "dirichlet" prescribes the momentum density j* (Eq. bbcon),
    "neumann" the traction T* (Eq. abbcon), "periodic" wraps (must pair).
    ``amp`` is the vector amplitude; for shape "disp_ramp" it is the
    displacement reached linearly over [t0, t1).
    """

    kind: str = "neumann"
    shape: str = "const"
    amp: tuple = (0.0, 0.0)
    t0: float = 0.0
    t1: float = 1.0
    s: float = 1.0
    unit: str = "steps"  # "steps": times are iterations k; "time": t = k dt


PERIODIC = Edge("periodic")
FREE = Edge("neumann")
CLAMPED = Edge("dirichlet")


@dataclass(frozen=True)
class Case:
    """A complete simulation request.  Edge order: left, right, bottom, top."""

    name: str
    nx: int
    ny: int
    nsteps: int
    model: str = "nh"
    E: float = 1.0
    nu: float = 0.3
    rho0: float = 1.0
    tau: float = 0.55
    dx: float | None = None  # default 1 / ny
    body: tuple = (0.0, 0.0)
    edges: tuple = (FREE, FREE, FREE, FREE)
    precision: str = "fp64"
    init: str = "rest"  # "rest" | "grf" | "translation" | "custom"
    seed: int = 0
    init_args: dict = field(default_factory=dict, hash=False, compare=False)
    extrap: str = "own"  # Neumann wall values: "own" (boundary node) | "linear" (two-point)
    gscale_log2: int = 0  # FP16 storage: stored g = g * 2^gscale_log2 (0: chosen from rho0)

    @property
    def spacing(self) -> float:
        return self.dx if self.dx is not None else 1.0 / self.ny

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# the benchmark workloads

def tension(nx: int = 32, ny: int = 32, nsteps: int = 2000, ramp: int = 1000, model: str = "nh",
            nu: float = 0.3, peak: float = 0.2, precision: str = "fp64") -> Case:
    """Uniaxial tension: left edge clamped (j* = 0), right edge traction
    (peak*E, 0) ramped linearly over the first ``ramp`` iterations, top and
    bottom traction-free (the paper's Sect. 4.1 problem, linear ramp)."""
    right = Edge("neumann", "linear_ramp", (peak * 1.0, 0.0), 0.0, float(ramp))
    return Case(f"tension_{nx}x{ny}_{model}", nx, ny, nsteps, model=model, nu=nu,
                edges=(CLAMPED, right, FREE, FREE), precision=precision)


def shear(n: int = 256, nsteps: int = 20000, model: str = "svk", nu: float = 0.3, gamma: float = 0.5,
          ramp: int = 20000, precision: str = "fp64") -> Case:
    """Simple shear: bottom clamped, top moved in x so that its displacement
    grows linearly to gamma * height over ``ramp`` iterations, left and right
    traction-free (Sect. 4.2 problem with a displacement ramp)."""
    height = n * (1.0 / n)
    top = Edge("dirichlet", "disp_ramp", (gamma * height, 0.0), 0.0, float(ramp))
    return Case(f"shear_{n}_{model}_nu{nu}", n, n, nsteps, model=model, nu=nu,
                edges=(FREE, FREE, CLAMPED, top), precision=precision)


def cantilever(nx: int = 4096, ny: int = 256, nsteps: int = 100000, width: int = 200,
               amp: float = 0.05, nu: float = 0.3, precision: str = "fp32") -> Case:
    """Bending waves in a clamped beam: left end clamped, a transverse
    half-sine traction pulse on the right end, top and bottom free
    (Sect. 4.3 problem with a half-sine pulse in place of the Ricker wavelet)."""
    right = Edge("neumann", "half_sine", (0.0, amp * 1.0), 0.0, float(width))
    return Case(f"cantilever_{nx}x{ny}", nx, ny, nsteps, model="nh", nu=nu,
                edges=(CLAMPED, right, FREE, FREE), precision=precision)


def roofline(n: int = 16384, nsteps: int = 500, precision: str = "fp32", seed: int = 5,
             corr: float = 64.0, modes: int = 64, strain: float = 0.2, nx: int | None = None) -> Case:
    """Periodic lattice with a smooth Gaussian random initial velocity
    (correlation length ``corr`` cells); the peak speed is ``strain`` times
    the shear wave speed so that plane-wave strains reach about ``strain``."""
    nx = n if nx is None else nx
    return Case(f"roofline_{nx}x{n}", nx, n, nsteps, model="nh", nu=0.3,
                edges=(PERIODIC, PERIODIC, PERIODIC, PERIODIC), precision=precision,
                init="grf", seed=seed, init_args=dict(corr=corr, modes=modes, strain=strain))


def shear_speed(case: Case) -> float:
    """Shear wave speed sqrt(mu/rho0) of the workload's material; used only to
    scale synthetic initial velocities."""
    mu = case.E / (2.0 * (1.0 + case.nu))
    return math.sqrt(mu / case.rho0)


# --------------------------------------------------------------------------
# the paper's own examples (Sect. 4), with times in the paper's time unit

def paper_tension(model: str = "nh", nu: float = 0.3, n: int = 40, precision: str = "fp64") -> Case:
    """Sect. 4.1: 1L x 1L, traction sigma* = alpha sin^2(pi t / 4) for t < 2,
    then alpha, on top (+) and bottom (-); left and right free; alpha = 0.175
    (SVK) or 0.35 (neo-Hooke); dx = 1/n (0.025 for n = 40)."""
    alpha = 0.175 if model == "svk" else 0.35
    top = Edge("neumann", "sin2_ramp", (0.0, alpha), 0.0, 2.0, unit="time")
    bottom = Edge("neumann", "sin2_ramp", (0.0, -alpha), 0.0, 2.0, unit="time")
    return Case(f"paper_tension_{model}_nu{nu}_{n}", n, n, 0, model=model, nu=nu, dx=1.0 / n,
                edges=(FREE, FREE, bottom, top), precision=precision)


def paper_shear(model: str = "nh", nu: float = 0.3, n: int = 40, precision: str = "fp64") -> Case:
    """Sect. 4.2: bottom clamped, top momentum j* = alpha sin(pi t / 2) for
    t < 2, then 0; alpha = 0.03 (SVK) or 0.1 (neo-Hooke)."""
    alpha = 0.03 if model == "svk" else 0.1
    top = Edge("dirichlet", "half_sine", (alpha, 0.0), 0.0, 2.0, unit="time")
    return Case(f"paper_shear_{model}_nu{nu}_{n}", n, n, 0, model=model, nu=nu, dx=1.0 / n,
                edges=(FREE, FREE, CLAMPED, top), precision=precision)


def paper_wave(tau: float = 0.55, n: int = 40, precision: str = "fp64") -> Case:
    """Sect. 4.3: 4L x 1L beam, left end clamped, tangential Ricker traction on
    the right end (alpha = 0.15, s = 0.215, t0 = 1, free for t > 2), neo-Hooke
    nu = 0.2.  The garbled prefactor of Eq. ricker is read as
    2 / (sqrt(3 sigma) pi^(1/4)) with sigma = sqrt(s) and folded into amp."""
    s_ = 0.215
    sigma = math.sqrt(s_)
    amp = 0.15 * 2.0 / (math.sqrt(3.0 * sigma) * math.pi ** 0.25)
    right = Edge("neumann", "ricker", (0.0, amp), 1.0, 2.0, s_, unit="time")
    return Case(f"paper_wave_tau{tau}", 4 * n, n, 0, model="nh", nu=0.2, dx=1.0 / n, tau=tau,
                edges=(CLAMPED, right, FREE, FREE), precision=precision)


# --------------------------------------------------------------------------
# seeded initial fields

def grf_modes(case: Case):
    """Wave vectors, amplitudes and phases of the periodic random field.

    v_c(x, y) = sum_m a[c, m] cos(2 pi (kx_m x / nx + ky_m y / ny) + phi[c, m]).
    Integer wave numbers make the field exactly periodic; they are drawn from a
    Gaussian of width n / (2 pi corr) so that the correlation length is about
    ``corr`` cells.
    """
    a = case.init_args
    rng = np.random.default_rng(case.seed)
    m = int(a.get("modes", 64))
    corr = float(a.get("corr", 64.0))
    kx = np.rint(rng.normal(0.0, case.nx / (2 * math.pi * corr), m)).astype(np.int64)
    ky = np.rint(rng.normal(0.0, case.ny / (2 * math.pi * corr), m)).astype(np.int64)
    both_zero = (kx == 0) & (ky == 0)
    kx[both_zero] = 1
    amp = rng.normal(0.0, 1.0, (2, m))
    phi = rng.uniform(0.0, 2 * math.pi, (2, m))
    return kx, ky, amp, phi


def grf_velocity(case: Case, x0: int = 0, y0: int = 0, wx: int | None = None, wy: int | None = None,
                 device=None):
    """Seeded periodic random velocity, shape [wy, wx, 2], float64.

    Without ``device`` it is the window [x0, x0+wx) x [y0, y0+wy) (coordinates
    taken modulo the lattice), built with numpy.  With ``device`` it is the
    whole lattice, built with torch on that device by the same formula.  The
    peak over the whole lattice (max over nodes and components of |v|) is
    normalised to ``strain * shear_speed``.
    """
    target = float(case.init_args.get("strain", 0.2)) * shear_speed(case)
    if device is not None:
        raw = _grf_raw(case, 0, 0, case.nx, case.ny, device)
        return raw * (target / float(raw.abs().max()))
    wx = case.nx if wx is None else wx
    wy = case.ny if wy is None else wy
    return _grf_raw(case, x0, y0, wx, wy, None) * (target / _grf_peak(case))


def _grf_raw(case, x0, y0, wx, wy, device):
    kx, ky, amp, phi = grf_modes(case)
    xs = (np.arange(x0, x0 + wx) % case.nx).astype(np.float64)
    ys = (np.arange(y0, y0 + wy) % case.ny).astype(np.float64)
    # cos(A + B + phi) = cos(A + phi) cos(B) - sin(A + phi) sin(B): a sum of
    # separable products, evaluated as one matrix product per component
    if device is None:
        ax = 2 * np.pi * np.outer(xs, kx) / case.nx  # [wx, m]
        by = 2 * np.pi * np.outer(ys, ky) / case.ny  # [wy, m]
        out = np.empty((wy, wx, 2))
        for c in range(2):
            A = np.concatenate([np.cos(ax + phi[c]), np.sin(ax + phi[c])], axis=1)  # [wx, 2m]
            B = np.concatenate([amp[c] * np.cos(by), -amp[c] * np.sin(by)], axis=1)  # [wy, 2m]
            out[:, :, c] = B @ A.T
        return out
    import torch
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device)
    ax = 2 * math.pi * torch.outer(t(xs), t(kx.astype(np.float64))) / case.nx
    by = 2 * math.pi * torch.outer(t(ys), t(ky.astype(np.float64))) / case.ny
    out = torch.empty((wy, wx, 2), dtype=torch.float64, device=device)
    for c in range(2):
        A = torch.cat([torch.cos(ax + t(phi[c])), torch.sin(ax + t(phi[c]))], dim=1)
        B = torch.cat([t(amp[c]) * torch.cos(by), -t(amp[c]) * torch.sin(by)], dim=1)
        out[:, :, c] = B @ A.T
    return out


_PEAK_CACHE: dict = {}


def _grf_peak(case: Case) -> float:
    """max |v_raw| over the whole lattice, evaluated in row blocks."""
    key = (case.nx, case.ny, case.seed, tuple(sorted(case.init_args.items())))
    if key not in _PEAK_CACHE:
        peak = 0.0
        block = max(1, min(case.ny, (1 << 22) // max(case.nx, 1)))
        for y0 in range(0, case.ny, block):
            h = min(block, case.ny - y0)
            peak = max(peak, float(np.abs(_grf_raw(case, 0, y0, case.nx, h, None)).max()))
        _PEAK_CACHE[key] = peak
    return _PEAK_CACHE[key]


def initial_fields(case: Case, device=None):
    """(u0, v0) as float64 arrays [ny, nx, 2], or (None, None) for a body at rest."""
    if case.init == "rest":
        return None, None
    if case.init == "grf":
        return None, grf_velocity(case, device=device)
    if case.init == "translation":
        a = case.init_args
        u0 = np.broadcast_to(np.asarray(a.get("u0", (0.0, 0.0)), dtype=np.float64), (case.ny, case.nx, 2)).copy()
        v0 = np.broadcast_to(np.asarray(a.get("v0", (0.0, 0.0)), dtype=np.float64), (case.ny, case.nx, 2)).copy()
        return u0, v0
    if case.init == "custom":
        return case.init_args.get("u0"), case.init_args.get("v0")
    raise ValueError(f"unknown init {case.init!r}")


def random_state(nx: int, ny: int, seed: int, amp_u: float = 1e-3, amp_v: float = 1e-2):
    """Smooth-ish seeded displacement and velocity fields (a few low Fourier
    modes plus small white noise) for parity tests on small lattices."""
    rng = np.random.default_rng(seed)
    xs = np.arange(nx)[None, :] / nx
    ys = np.arange(ny)[:, None] / ny
    u0 = np.zeros((ny, nx, 2))
    v0 = np.zeros((ny, nx, 2))
    for c in range(2):
        for _ in range(3):
            kx, ky = rng.integers(1, 3, 2)
            ph = rng.uniform(0, 2 * np.pi, 2)
            u0[:, :, c] += amp_u * np.sin(2 * np.pi * (kx * xs + ky * ys) + ph[0])
            v0[:, :, c] += amp_v * np.sin(2 * np.pi * (kx * xs - ky * ys) + ph[1])
        u0[:, :, c] += 0.05 * amp_u * rng.standard_normal((ny, nx))
        v0[:, :, c] += 0.05 * amp_v * rng.standard_normal((ny, nx))
    return u0, v0


# --------------------------------------------------------------------------
# the serving trace

def serving_trace(n_requests: int = 512, seed: int = 4, rate: float = 1.0, min_side: int = 32,
                  max_nx: int = 1024, max_ny: int = 512, min_steps: int = 1000, max_steps: int = 50000,
                  precision: str = "fp32"):
    """Poisson arrivals of mixed requests: lattices log-uniform in size,
    SVK or neo-Hooke (1/2 each), Poisson ratio uniform in [0, 0.45], load
    tension / shear / tip pulse (1/3 each), steps log-uniform.

    Returns a list of (arrival_time_seconds, Case).  ``rate`` is in requests
    per second.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        nx = int(round(math.exp(rng.uniform(math.log(min_side), math.log(max_nx)))))
        ny = int(round(math.exp(rng.uniform(math.log(min_side), math.log(max_ny)))))
        model = "svk" if rng.random() < 0.5 else "nh"
        nu = float(rng.uniform(0.0, 0.45))
        steps = int(round(math.exp(rng.uniform(math.log(min_steps), math.log(max_steps)))))
        load = int(rng.integers(0, 3))
        if load == 0:
            c = tension(nx, ny, steps, ramp=max(1, steps // 2), model=model, nu=nu, precision=precision)
        elif load == 1:
            amp = 0.05 if model == "svk" else 0.5
            top = Edge("dirichlet", "disp_ramp", (amp * ny * (1.0 / ny), 0.0), 0.0, float(steps))
            c = Case(f"shear_{nx}x{ny}", nx, ny, steps, model=model, nu=nu,
                     edges=(FREE, FREE, CLAMPED, top), precision=precision)
        else:
            c = cantilever(nx, ny, steps, width=min(200, max(2, steps // 5)), nu=nu, precision=precision)
            c = c.replace(model=model)
        out.append((t, c.replace(name=f"req{i:04d}_{c.name}")))
    return out
