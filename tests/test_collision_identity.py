"""The kernels' collision is written in ghost combinations of the populations
(one even, four odd) instead of moments and an equilibrium.  This pins that
rewrite on the host: for random populations, sources and relaxation times it
equals the oracle's literal BGK collision with forcing, Alg. 1 with Eq. feq and
the forcing term, to double rounding.  The kernels run the same formulas; the
GPU parity tests compare them with the oracle over whole histories."""
import math

import numpy as np
import pytest

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def literal(O, f, S, cs, tau, dt):
    """Alg. 1 collision: moments of f, feq (Eq. feq) with j = sum c f + dt/2 S,
    then g = f - (f - feq)/tau + (1 - 1/(2 tau)) psi dt."""
    c = math.sqrt(3.0) * cs
    r = f.sum()
    j = np.array([c * (EX * f).sum() + 0.5 * dt * S[0], c * (EY * f).sum() + 0.5 * dt * S[1]])
    Pi = np.array([(c * c * EX * EX * f).sum(), (c * c * EX * EY * f).sum(),
                   (c * c * EY * EX * f).sum(), (c * c * EY * EY * f).sum()])
    feq = O.equilibrium(cs, r, j, Pi)
    psi = O.forcing(cs, S)
    return f - (f - feq) / tau + (1.0 - 0.5 / tau) * psi * dt


def ghost(f, S, cs, tau, dt, scaled_odd=True):
    """The kernels' form: g_q = f_q - omega (f - feq)_q + w_q sigma e_q.S, each
    opposite pair as (f + A) +- b with A the relaxation of the even part and b
    that of the odd part plus the forcing."""
    c = math.sqrt(3.0) * cs
    omega, sigma = 1.0 / tau, c * dt / cs ** 2
    s13, s24, s57, s68 = f[1] + f[3], f[2] + f[4], f[5] + f[7], f[6] + f[8]
    d13, d24, d57, d68 = f[1] - f[3], f[2] - f[4], f[5] - f[7], f[6] - f[8]
    Q = f[0] - 2 * (s13 + s24) + 4 * (s57 + s68)
    fx, fy = S[0] * (sigma / 9), S[1] * (sigma / 9)
    f57, f68 = (S[0] + S[1]) * (sigma / 36), (S[1] - S[0]) * (sigma / 36)
    # even relaxation shared by a pair, odd part and forcing with opposite signs
    A1, A5 = Q * (omega / 18), Q * (-omega / 36)
    if scaled_odd:  # (double precision) the odd parts times 6 and 12, the factor -omega/6, -omega/12
        tx, ty = d13 - 2 * (d57 - d68), d24 - 2 * (d57 + d68)
        t57, t68 = 4 * d57 - (d13 + d24), 4 * d68 - (d24 - d13)
        bx, by = tx * (-omega / 6) + fx, ty * (-omega / 6) + fy
        b57, b68 = t57 * (-omega / 12) + f57, t68 * (-omega / 12) + f68
    else:  # (single precision) the odd parts themselves
        ox, oy = d13 / 6 - (d57 - d68) / 3, d24 / 6 - (d57 + d68) / 3
        o57, o68 = d57 / 3 - (d13 + d24) / 12, d68 / 3 - (d24 - d13) / 12
        bx, by = -omega * ox + fx, -omega * oy + fy
        b57, b68 = -omega * o57 + f57, -omega * o68 + f68
    g = np.empty(9)
    g[0] = f[0] - omega * (Q / 9)
    g[1], g[3] = (f[1] + A1) + bx, (f[3] + A1) - bx
    g[2], g[4] = (f[2] + A1) + by, (f[4] + A1) - by
    g[5], g[7] = (f[5] + A5) + b57, (f[7] + A5) - b57
    g[6], g[8] = (f[6] + A5) + b68, (f[8] + A5) - b68
    return g


@pytest.mark.parametrize("scaled_odd", [True, False])
@pytest.mark.parametrize("seed", range(20))
def test_ghost_form_equals_literal_collision(oracle_mod, seed, scaled_odd):
    rng = np.random.default_rng(seed)
    f = rng.normal(0.0, 0.1, 9)
    S = rng.normal(0.0, 1.0, 2)
    cs = rng.uniform(0.3, 1.5)
    tau = rng.uniform(0.51, 1.5)
    dt = rng.uniform(0.01, 0.1)
    ref = literal(oracle_mod, f, S, cs, tau, dt)
    assert np.abs(ghost(f, S, cs, tau, dt, scaled_odd) - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


def test_ghost_form_conserves_r_pi_and_adds_dt_s(oracle_mod):
    """Collision leaves r and Pi unchanged and adds dt S to c sum e f."""
    rng = np.random.default_rng(7)
    f, S, cs, tau, dt = rng.normal(0, 0.1, 9), rng.normal(0, 1, 2), 0.7, 0.55, 0.03
    g = ghost(f, S, cs, tau, dt)
    c = math.sqrt(3.0) * cs
    assert abs(g.sum() - f.sum()) < 1e-15
    for a, b in ((EX, EX), (EX, EY), (EY, EY)):
        assert abs((a * b * (g - f)).sum()) < 1e-15
    assert np.allclose([c * (EX * (g - f)).sum(), c * (EY * (g - f)).sum()], dt * S, atol=1e-15)
