"""Pins of the oracle against values the paper prints (tests/golden/, each
file citing where): the D2Q9 table (Tab. 1) through the equilibrium, the
stability bounds of Sect. 3.2 through the plane-strain parameters, and the
boundary loads of the examples of Sect. 4 through the oracle's load
function.  A reordered velocity table, a plane-stress Lame constant, a
load evaluated in iterations instead of time, or a wrong ramp shape each
fails one of them."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2502_00920_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LEFT, RIGHT, BOTTOM, TOP = 0, 1, 2, 3


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split("#")[0].strip() for l in f if l.split("#")[0].strip()]


def _number(tok):
    named = {"sqrt3": math.sqrt(3.0), "4/pi": 4.0 / math.pi}
    return named[tok] if tok in named else float(Fraction(tok))


def _keys(name):
    out = {}
    for line in _lines(name):
        k, v = (s.strip() for s in line.split("=", 1))
        vals = [_number(t) for t in v.split()]
        out[k] = vals[0] if len(vals) == 1 else vals
    return out


def d2q9():
    rows = [l.split() for l in _lines("d2q9_tab1.txt")]
    q = [int(r[0]) for r in rows]
    assert q == list(range(9))
    return (np.array([int(r[1]) for r in rows]), np.array([int(r[2]) for r in rows]),
            np.array([float(Fraction(r[3])) for r in rows]))


def test_d2q9_table_pins_the_equilibrium(oracle_mod):
    """At rest (r = 1, j = 0, Pi = r cs^2 I) the equilibrium is the weights of
    Tab. 1; a pure momentum j gives w_q c_q . j / cs^2, whose pattern over q is
    the table's velocity order (c = sqrt(3) cs, Sect. 3.2)."""
    cx, cy, w = d2q9()
    cfl = _keys("cfl_bounds.txt")
    cs = 0.73
    c = cfl["c_over_cs"] * cs
    rest = oracle_mod.equilibrium(cs, 1.0, np.zeros(2), np.array([[cs * cs, 0.0], [0.0, cs * cs]]))
    np.testing.assert_allclose(rest, w, rtol=0, atol=1e-15)
    for j in (np.array([0.3, 0.0]), np.array([0.0, -0.2]), np.array([0.1, 0.25])):
        f = oracle_mod.equilibrium(cs, 0.0, j, np.zeros((2, 2)))
        np.testing.assert_allclose(f, w * c * (cx * j[0] + cy * j[1]) / cs ** 2, rtol=0, atol=1e-15)


def test_cfl_bounds_pin_plane_strain_parameters(oracle_mod):
    """c_d = sqrt((lam + 2 mu)/rho0) equals c at nu = 0.25 and 2c at nu = 5/11
    (the bounds Sect. 3.2 prints for first- and second-order stencils), and
    c = sqrt(3) c_s."""
    cfl = _keys("cfl_bounds.txt")
    for nu, ratio in ((cfl["nu_first_order"], cfl["c_d_over_c_first_order"]),
                      (cfl["nu_second_order"], cfl["c_d_over_c_second_order"])):
        case = I.Case("cfl", 8, 8, 0, nu=nu, E=1.7, rho0=1.3, dx=0.05)
        p = oracle_mod.params(case)
        c_d = math.sqrt((p["lam"] + 2 * p["mu"]) / case.rho0)
        assert c_d / p["c"] == pytest.approx(ratio, rel=1e-13)
        assert p["c"] / p["cs"] == pytest.approx(cfl["c_over_cs"], rel=1e-15)
    assert I.Case("d", 8, 8, 0).tau == cfl["tau_adopted"]
    with pytest.raises(Exception):
        oracle_mod.OracleSim(I.Case("t", 8, 8, 0, tau=cfl["tau_min_exclusive"]))


@pytest.mark.parametrize("model", ["svk", "nh"])
def test_tension_load_is_the_printed_ramp(oracle_mod, model):
    """Sect. 4.1: traction alpha sin^2(pi t / 4) for t < 2, alpha after, on the
    top edge (and its mirror on the bottom), in the paper's time unit."""
    g = _keys("paper_examples.txt")
    case = I.paper_tension(model, 0.3)
    assert case.nx * case.ny == g["tension.nodes"] and case.spacing == pytest.approx(g["tension.dx"])
    alpha = g[f"tension.alpha.{model}"]
    dt = oracle_mod.params(case)["dt"]
    for k in (0, 7, 30, 61, int(g["tension.ramp_end"] / dt) + 3, 400):
        t = k * dt
        expect = alpha * (math.sin(math.pi * t / 4) ** 2 if t < g["tension.ramp_end"] else 1.0)
        np.testing.assert_allclose(oracle_mod.load(case, TOP, k), [0.0, expect], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(oracle_mod.load(case, BOTTOM, k), [0.0, -expect], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("model", ["svk", "nh"])
def test_shear_momentum_integrates_to_the_printed_displacement(oracle_mod, model):
    """Sect. 4.2: the top momentum alpha sin(pi t / 2) (t < 2, then 0),
    integrated over time with rho0 = 1, is the printed displacement
    alpha (2/pi)(1 - cos(pi t / 2)), reaching alpha 4/pi at t = 2 and staying."""
    g = _keys("paper_examples.txt")
    alpha = g[f"shear.alpha.{model}"]
    case = I.paper_shear(model, 0.2, n=400)  # a fine time step for the quadrature
    dt = oracle_mod.params(case)["dt"]
    kmax = int(3.0 / dt)
    j = np.array([oracle_mod.load(case, TOP, k)[0] for k in range(kmax + 1)])
    assert np.all(np.array([oracle_mod.load(case, TOP, k)[1] for k in (0, 5, 50)]) == 0.0)
    u = np.concatenate([[0.0], np.cumsum(0.5 * (j[1:] + j[:-1]) * dt)])  # trapezoidal, rho0 = 1
    for T in (0.5, 1.0, 1.5):
        k = int(round(T / dt))
        t = k * dt
        assert u[k] == pytest.approx(alpha * 2 / math.pi * (1 - math.cos(math.pi * t / 2)), rel=1e-5)
    assert u[-1] == pytest.approx(alpha * g["shear.final_displacement_over_alpha"], rel=1e-3)


def test_wave_ricker_load_has_the_printed_shape(oracle_mod):
    """Sect. 4.3: the tangential traction on the right end follows
    (1 - (t - t0)^2 / s) exp(-(t - t0)^2 / (2 s)) with s = 0.215, t0 = 1, and
    the end is free for t > 2; the domain is 4L x 1L at dx = 0.025, nu = 0.2.
    (The printed prefactor is garbled; only the shape is pinned.)"""
    g = _keys("paper_examples.txt")
    for tau in g["wave.taus"]:
        case = I.paper_wave(tau)
        assert (case.nx * case.spacing, case.ny * case.spacing) == pytest.approx(tuple(g["wave.domain"]))
        assert case.spacing == pytest.approx(g["wave.dx"]) and case.nu == g["wave.nu"] and case.tau == tau
    case = I.paper_wave(0.55)
    dt = oracle_mod.params(case)["dt"]
    s, t0 = g["wave.s"], g["wave.t0"]
    k0 = int(round(t0 / dt))
    d0 = k0 * dt - t0
    peak = oracle_mod.load(case, RIGHT, k0)[1] / ((1.0 - d0 * d0 / s) * math.exp(-0.5 * d0 * d0 / s))
    for k in range(0, int(2.5 / dt), 7):
        t = k * dt
        got = oracle_mod.load(case, RIGHT, k)
        shape = (1 - (t - t0) ** 2 / s) * math.exp(-0.5 * (t - t0) ** 2 / s) if t < g["wave.free_after"] else 0.0
        assert got[0] == 0.0
        assert got[1] == pytest.approx(peak * shape, rel=1e-12, abs=1e-15)
