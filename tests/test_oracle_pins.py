"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: moment
identities of the D2Q9 set (Tab. 1), closed-form stresses of homogeneous
deformations (Sect. 4), derivatives of the strain energies, exactness of the
finite-difference stencils (Sect. 3.2), rigid motions, pre-stressed states
that must stay stationary under the boundary rules (Sect. 3.3),
conservation laws of the moment chain (Sect. 3.1) and the elastic wave
speeds of the Navier-Cauchy limit.
"""
import math

import numpy as np
import pytest

from paper_2502_00920_gb300 import inputs as I

# Tab. 1: lattice directions (velocities are c * e_q) and weights, typed here
# from the paper so that the oracle's own tables are checked against them.
EQ = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], float)
WQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

E_, NU = 1.0, 0.3
MU = E_ / (2 * (1 + NU))
LAM = E_ * NU / ((1 + NU) * (1 - 2 * NU))
P4 = (I.PERIODIC,) * 4


def sym(rng):
    a = rng.normal(size=(2, 2))
    return a + a.T


# ---------------------------------------------------------------- Sect. 3.2

def test_equilibrium_reproduces_moments(oracle_mod):
    """f^eq yields exactly r, j and Pi as its moments (Eq. moments)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        cs = rng.uniform(0.3, 2.0)
        c = math.sqrt(3) * cs
        r = rng.normal()
        j = rng.normal(size=2)
        Pi = sym(rng)
        f = oracle_mod.equilibrium(cs, r, j, Pi.ravel())
        cq = c * EQ
        assert abs(f.sum() - r) <= 1e-13 * (1 + abs(r))
        np.testing.assert_allclose(cq.T @ f, j, atol=1e-13 * (1 + np.abs(j).max()))
        np.testing.assert_allclose(np.einsum("qa,qb,q->ab", cq, cq, f), Pi, atol=1e-12 * (1 + np.abs(Pi).max()))


def test_equilibrium_is_weighted_hermite_expansion(oracle_mod):
    """Each f^eq_q is w_q times a polynomial in c_q; at rest with only r the
    populations are w_q r (2 - |c_q|^2 / (2 c_s^2))."""
    cs = 0.7
    f = oracle_mod.equilibrium(cs, 1.0, [0, 0], [cs * cs, 0, 0, cs * cs])
    np.testing.assert_allclose(f, WQ, rtol=1e-14)  # Pi = r cs^2 I leaves only w_q r
    f = oracle_mod.equilibrium(cs, 2.0, [0, 0], [0, 0, 0, 0])
    cq2 = 3 * cs * cs * (EQ ** 2).sum(1)
    np.testing.assert_allclose(f, WQ * 2.0 * (2 - cq2 / (2 * cs * cs)), rtol=1e-14, atol=1e-15)


def test_forcing_moments(oracle_mod):
    """psi carries the source into the first moment only (Eq. forcing)."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        cs = rng.uniform(0.3, 2.0)
        S = rng.normal(size=2)
        psi = oracle_mod.forcing(cs, S)
        cq = math.sqrt(3) * cs * EQ
        assert abs(psi.sum()) < 1e-14
        np.testing.assert_allclose(cq.T @ psi, S, rtol=1e-13)
        np.testing.assert_allclose(np.einsum("qa,qb,q->ab", cq, cq, psi), 0, atol=1e-13)


def test_parameters_plane_strain_and_lattice_speed(oracle_mod):
    """nu = 1/4 gives lam = mu and nu = 5/11 gives lam = 10 mu: the two CFL
    bounds quoted in Sect. 3.2 hold only for plane-strain Lame constants;
    c = sqrt(3) c_s and dt = dX / c."""
    for nu, ratio in [(0.25, 1.0), (5 / 11, 10.0)]:
        p = oracle_mod.params(I.Case("p", 4, 4, 0, nu=nu, E=2.0, rho0=1.5, dx=0.1))
        assert p["lam"] / p["mu"] == pytest.approx(ratio, rel=1e-13)
        # c_d <= c  <=>  lam + 2 mu <= 3 mu ; c_d <= 2c <=> lam + 2 mu <= 12 mu
        assert p["mu"] == pytest.approx(2.0 / (2 * (1 + nu)), rel=1e-15)
        assert p["cs"] == pytest.approx(math.sqrt(p["mu"] / 1.5), rel=1e-15)
        assert p["c"] == pytest.approx(math.sqrt(3) * p["cs"], rel=1e-15)
        assert p["dt"] == pytest.approx(0.1 / p["c"], rel=1e-15)


# ---------------------------------------------------------------- Sect. 4

def F_of(H):
    return np.eye(2) + np.asarray(H).reshape(2, 2)


def W_svk(F, lam, mu):
    E = 0.5 * (F.T @ F - np.eye(2))
    return 0.5 * lam * np.trace(E) ** 2 + mu * np.trace(E @ E)


def W_nh(F, lam, mu):
    J = np.linalg.det(F)
    C = F.T @ F
    return 0.25 * lam * (J * J - 1 - 2 * math.log(J)) + 0.5 * mu * (np.trace(C) - 2 - 2 * math.log(J))


def W_le(F, lam, mu):
    H = F - np.eye(2)
    e = 0.5 * (H + H.T)
    return 0.5 * lam * np.trace(H) ** 2 + mu * np.sum(e * e)


@pytest.mark.parametrize("model,W", [("svk", W_svk), ("nh", W_nh), ("le", W_le)])
def test_stress_is_energy_derivative(oracle_mod, model, W):
    """P = dW/dF for the hyperelastic energies whose second Piola-Kirchhoff
    stresses are the ones printed in Sect. 4 (central differences in F)."""
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(10):
        H = 0.3 * rng.normal(size=(2, 2))
        if np.linalg.det(F_of(H)) < 0.3:
            continue
        P = oracle_mod.first_piola(model, LAM, MU, H.ravel()).reshape(2, 2)
        G = np.zeros((2, 2))
        for a in range(2):
            for b in range(2):
                d = np.zeros((2, 2))
                d[a, b] = h
                G[a, b] = (W(F_of(H + d), LAM, MU) - W(F_of(H - d), LAM, MU)) / (2 * h)
        np.testing.assert_allclose(P, G, atol=2e-8)


def test_simple_shear_closed_forms(oracle_mod):
    """F = [[1, g], [0, 1]]: neo-Hooke gives P = mu [[0, g], [g, 0]];
    St. Venant-Kirchhoff gives the values derived by hand below."""
    for g in (0.1, 0.5, 1.3):
        P = oracle_mod.first_piola("nh", LAM, MU, [0, g, 0, 0])
        np.testing.assert_allclose(P, [0, MU * g, MU * g, 0], atol=1e-14)
    g = 0.5
    P = oracle_mod.first_piola("svk", LAM, MU, [0, g, 0, 0])
    s11 = LAM * g * g / 2
    s12 = MU * g
    s22 = LAM * g * g / 2 + MU * g * g
    np.testing.assert_allclose(P, [s11 + g * s12, s12 + g * s22, s12, s22], rtol=1e-14)
    np.testing.assert_allclose(P, [0.168269, 0.276442, 0.192308, 0.168269], atol=5e-7)


@pytest.mark.parametrize("model", ["nh", "svk"])
def test_uniaxial_closed_form(oracle_mod, model):
    """Homogeneous uniaxial stress P11 = 0.2, P22 = 0 (E = 1, nu = 0.3): the
    principal stretches solve two scalar equations written from S = S(C, J)
    with C = diag(a^2, b^2); the oracle must return exactly that stress."""
    from scipy.optimize import fsolve

    def principal(ab):
        a, b = ab
        if model == "nh":
            J2 = (a * b) ** 2
            s1 = 0.5 * LAM * (J2 - 1) / a ** 2 + MU * (1 - 1 / a ** 2)
            s2 = 0.5 * LAM * (J2 - 1) / b ** 2 + MU * (1 - 1 / b ** 2)
        else:
            e1, e2 = 0.5 * (a * a - 1), 0.5 * (b * b - 1)
            s1 = LAM * (e1 + e2) + 2 * MU * e1
            s2 = LAM * (e1 + e2) + 2 * MU * e2
        return [a * s1 - 0.2, b * s2]

    a, b = fsolve(principal, [1.1, 0.95], xtol=1e-13)
    ref = {"nh": (1.209694, 0.913410), "svk": (1.147677, 0.929555)}[model]
    assert (a, b) == pytest.approx(ref, abs=2e-6)
    P = oracle_mod.first_piola(model, LAM, MU, [a - 1, 0, 0, b - 1])
    np.testing.assert_allclose(P, [0.2, 0, 0, 0], atol=1e-13)


@pytest.mark.parametrize("model", ["nh", "svk"])
def test_rotation_is_stress_free_and_frame_indifferent(oracle_mod, model):
    rng = np.random.default_rng(4)
    for th in (0.3, 1.0, 2.5):
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        P = oracle_mod.first_piola(model, LAM, MU, (R - np.eye(2)).ravel())
        np.testing.assert_allclose(P, 0, atol=1e-14)
        H = 0.2 * rng.normal(size=(2, 2))
        PF = oracle_mod.first_piola(model, LAM, MU, H.ravel()).reshape(2, 2)
        PQF = oracle_mod.first_piola(model, LAM, MU, (R @ F_of(H) - np.eye(2)).ravel()).reshape(2, 2)
        np.testing.assert_allclose(PQF, R @ PF, atol=1e-13)


def test_constitutive_split_leaves_lame_correction(oracle_mod):
    """For the linear material P + Pi(H) = (lam - mu) tr(H) I exactly: the
    moment chain carries mu(H + H^T + tr H I) and the source the rest.  For
    SVK and NH the remainder differs from it at second order in H."""
    rng = np.random.default_rng(5)
    H = rng.normal(size=(2, 2))
    N = oracle_mod.first_piola("le", LAM, MU, H.ravel()) + oracle_mod.pi_of_h(MU, H.ravel())
    np.testing.assert_allclose(N, ((LAM - MU) * np.trace(H) * np.eye(2)).ravel(), atol=1e-14)
    for model in ("svk", "nh"):
        errs = []
        for eps in (1e-2, 5e-3):
            He = eps * H
            N = oracle_mod.first_piola(model, LAM, MU, He.ravel()) + oracle_mod.pi_of_h(MU, He.ravel())
            errs.append(np.abs(N - ((LAM - MU) * np.trace(He) * np.eye(2)).ravel()).max())
        assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)


# ---------------------------------------------------------------- FD stencils

def test_gradient_stencils(oracle_mod):
    """Linear fields are differentiated exactly everywhere; for u = x^2 the
    central stencil is exact inside and the first-order one-sided stencil on
    the walls errs by exactly +dx (left) and -dx (right)."""
    nx, ny, dx = 7, 5, 0.1
    case = I.Case("g", nx, ny, 0, dx=dx, edges=(I.FREE,) * 4)
    X, Y = np.meshgrid(np.arange(nx) * dx, np.arange(ny) * dx)
    A = np.array([[0.3, -1.2], [2.0, 0.7]])
    u = np.stack([A[0, 0] * X + A[0, 1] * Y, A[1, 0] * X + A[1, 1] * Y], -1)
    H = oracle_mod.gradient(case, u)
    np.testing.assert_allclose(H, np.broadcast_to(A.ravel(), H.shape), atol=1e-13)
    u = np.stack([X ** 2, np.zeros_like(X)], -1)
    H = oracle_mod.gradient(case, u)
    exact = 2 * X
    err = H[:, :, 0] - exact
    np.testing.assert_allclose(err[:, 1:-1], 0, atol=1e-13)
    np.testing.assert_allclose(err[:, 0], dx, atol=1e-13)
    np.testing.assert_allclose(err[:, -1], -dx, atol=1e-13)
    np.testing.assert_allclose(H[:, :, 1:], 0, atol=1e-13)


def test_gradient_periodic_wraps(oracle_mod):
    nx, ny = 16, 8
    case = I.Case("g", nx, ny, 0, dx=1.0 / ny, edges=P4)
    x = np.arange(nx) / nx
    u = np.zeros((ny, nx, 2))
    u[:, :, 1] = np.sin(2 * np.pi * x)[None, :]
    H = oracle_mod.gradient(case, u)
    dx = 1.0 / ny
    central = (np.sin(2 * np.pi * (x + 1 / nx)) - np.sin(2 * np.pi * (x - 1 / nx))) / (2 * dx)
    np.testing.assert_allclose(H[:, :, 2], np.broadcast_to(central, (ny, nx)), atol=1e-13)


# ---------------------------------------------------------------- loads

def test_load_shapes(oracle_mod):
    edges = (I.Edge("neumann", "linear_ramp", (2.0, -1.0), 10, 30),
             I.Edge("neumann", "half_sine", (0.0, 1.0), 0, 200),
             I.Edge("neumann", "sin2_ramp", (1.0, 0.0), 0, 100),
             I.Edge("dirichlet", "disp_ramp", (0.5, 0.0), 0, 1000))
    case = I.Case("l", 8, 8, 0, edges=edges, nu=0.25)
    L = lambda e, k: oracle_mod.load(case, e, k)
    np.testing.assert_allclose(L(0, 5), [0, 0])
    np.testing.assert_allclose(L(0, 20), [1.0, -0.5], rtol=1e-15)
    np.testing.assert_allclose(L(0, 99), [2.0, -1.0], rtol=1e-15)
    np.testing.assert_allclose(L(1, 100), [0, 1.0], atol=1e-15)
    np.testing.assert_allclose(L(1, 50), [0, math.sin(math.pi / 4)], rtol=1e-15)
    np.testing.assert_allclose(L(1, 200), [0, 0])
    np.testing.assert_allclose(L(2, 50), [0.5, 0], rtol=1e-14)
    np.testing.assert_allclose(L(2, 150), [1.0, 0], rtol=1e-15)
    dt = oracle_mod.params(case)["dt"]
    np.testing.assert_allclose(L(3, 0), [0.5 / (1000 * dt), 0], rtol=1e-14)
    np.testing.assert_allclose(L(3, 1000), [0, 0])
    ricker = I.Case("r", 8, 8, 0, edges=(I.Edge("neumann", "ricker", (0, 3.0), 40, 80, 25.0),) + (I.FREE,) * 3)
    d = 47 - 40
    np.testing.assert_allclose(oracle_mod.load(ricker, 0, 47), [0, 3.0 * (1 - d * d / 25) * math.exp(-d * d / 50)],
                               rtol=1e-14)
    np.testing.assert_allclose(oracle_mod.load(ricker, 0, 90), [0, 0])


# ---------------------------------------------------------------- whole scheme

def run(oracle_mod, case, u0=None, v0=None, steps=0, order="text"):
    s = oracle_mod.OracleSim(case, u0, v0, order=order)
    s.step(steps)
    return s, s.fields()


def const_field(case, vec):
    return np.broadcast_to(np.asarray(vec, float), (case.ny, case.nx, 2)).copy()


@pytest.mark.parametrize("walls", ["periodic", "dirichlet", "neumann", "mixed"])
def test_uniform_translation_is_exact(oracle_mod, walls):
    """A rigid translation u = u0 + v0 t: H = 0, S = 0, f = f^eq stays put and
    the trapezoidal rule must advance u by exactly dt v0 per step (this pins
    the dt factor of the displacement update).  With walls, Dirichlet edges
    prescribe j* = rho0 v0 and Neumann edges are traction-free."""
    v = np.array([0.013, -0.021])
    mov = I.Edge("dirichlet", "const", tuple(1.0 * v))
    edges = {"periodic": P4, "dirichlet": (mov,) * 4, "neumann": (I.FREE,) * 4,
             "mixed": (mov, mov, I.FREE, I.FREE)}[walls]
    case = I.Case("t", 9, 7, 0, model="nh", edges=edges)
    u0 = const_field(case, [0.1, -0.05])
    s, (u, vv, P) = run(oracle_mod, case, u0, const_field(case, v), 40)
    dt = oracle_mod.params(case)["dt"]
    np.testing.assert_allclose(u, u0 + 40 * dt * v, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vv, const_field(case, v), rtol=0, atol=1e-14)
    np.testing.assert_allclose(P, 0, atol=1e-14)


@pytest.mark.parametrize("model", ["nh", "svk"])
def test_rigid_rotation_stays_put(oracle_mod, model):
    """A finite rotation at rest with traction-free Neumann edges: P = 0
    everywhere and the anti-bounce-back rule must return the equilibrium
    populations unchanged, so u stays (R - I) X and v stays 0."""
    th = 0.6
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    case = I.Case("rot", 8, 6, 0, model=model, edges=(I.FREE,) * 4)
    dx = case.spacing
    X, Y = np.meshgrid(np.arange(case.nx) * dx, np.arange(case.ny) * dx)
    Xv = np.stack([X, Y], -1)
    u0 = Xv @ (R - np.eye(2)).T
    # 15 steps: the state is exactly stationary, but around a large rotation
    # the explicit source term carries O(1) stiffness and rounding noise grows
    # by about 1.2x per step, so longer runs only measure that growth
    s, (u, v, P) = run(oracle_mod, case, u0, None, 15)
    np.testing.assert_allclose(u, u0, atol=1e-13)
    np.testing.assert_allclose(v, 0, atol=1e-13)
    np.testing.assert_allclose(P, 0, atol=1e-13)


def prestressed_case(oracle_mod, model, Fmat, nx=7, ny=6):
    """Homogeneous deformation u = (F - I) X held by tractions T = P N on
    every edge, with P the closed-form stress of F."""
    P = oracle_mod.first_piola(model, LAM, MU, (Fmat - np.eye(2)).ravel()).reshape(2, 2)
    normals = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    edges = tuple(I.Edge("neumann", "const", tuple(P @ np.array(nv, float))) for nv in normals)
    case = I.Case("pre", nx, ny, 0, model=model, nu=NU, edges=edges)
    dx = case.spacing
    X, Y = np.meshgrid(np.arange(nx) * dx, np.arange(ny) * dx)
    u0 = np.stack([X, Y], -1) @ (Fmat - np.eye(2)).T
    return case, u0, P


@pytest.mark.parametrize("model", ["nh", "svk"])
@pytest.mark.parametrize("kind", ["uniaxial", "shear", "general"])
def test_prestressed_homogeneous_state_is_stationary(oracle_mod, model, kind):
    """Under tractions T* = P N of a homogeneous finite deformation the
    quasi-boundary traction -T* + (P + Pi(H)) N equals Pi(H) N, so the
    Neumann rule reflects the equilibrium populations and nothing moves.  A
    wrong traction sign, a transposed H or a wrong P breaks this."""
    Fm = {"uniaxial": np.diag([1.209694, 0.913410]), "shear": np.array([[1.0, 0.4], [0.0, 1.0]]),
          "general": np.array([[1.1, 0.15], [-0.08, 0.93]])}[kind]
    case, u0, P = prestressed_case(oracle_mod, model, Fm)
    s, (u, v, Pf) = run(oracle_mod, case, u0, None, 40)
    np.testing.assert_allclose(u, u0, atol=1e-13)
    np.testing.assert_allclose(v, 0, atol=1e-12)
    np.testing.assert_allclose(Pf, np.broadcast_to(P.ravel(), Pf.shape), atol=1e-12)


def test_prestressed_state_moves_under_wrong_traction(oracle_mod):
    """Control for the stationarity pin: flipping the traction sign on one
    edge must set the body in motion."""
    Fm = np.diag([1.1, 0.95])
    case, u0, P = prestressed_case(oracle_mod, "nh", Fm)
    e = list(case.edges)
    e[1] = I.Edge("neumann", "const", tuple(-np.asarray(e[1].amp)))
    s, (u, v, _) = run(oracle_mod, case.replace(edges=tuple(e)), u0, None, 10)
    assert np.abs(v).max() > 1e-3


def test_momentum_conservation_periodic(oracle_mod):
    """Periodic lattice, no body force: central differences telescope, so the
    total momentum is constant (moment chain, Sect. 3.1); with a body force b
    it grows by exactly rho0 b dt per node and step."""
    case = I.Case("c", 24, 20, 0, model="nh", edges=P4)
    u0, v0 = I.random_state(24, 20, 7, amp_u=2e-2, amp_v=5e-2)
    s = oracle_mod.OracleSim(case, u0, v0)
    p0 = s.fields()[1].sum(axis=(0, 1))
    s.step(300)
    u, v, _ = s.fields()
    assert np.isfinite(u).all()
    np.testing.assert_allclose(v.sum(axis=(0, 1)), p0, atol=1e-12 * np.abs(v).sum())
    b = np.array([0.01, -0.02])
    caseb = case.replace(body=tuple(b))
    s = oracle_mod.OracleSim(caseb, u0, v0)
    s.step(50)
    dt = oracle_mod.params(caseb)["dt"]
    np.testing.assert_allclose(s.fields()[1].sum(axis=(0, 1)), p0 + 50 * dt * b * case.cells, rtol=1e-11)


def wave_frequency(oracle_mod, nx, comp, nu, model="le"):
    """Angular frequency of a standing wave v0 = A sin(2 pi x / L) e_comp on a
    periodic strip, from the time between the first and the fifth sign change
    of u at the crest node (two full periods; the start-up transient's phase
    offset cancels)."""
    case = I.Case("w", nx, 4, 0, model=model, nu=nu, dx=1.0 / nx, edges=P4)
    x = np.arange(nx) / nx
    v0 = np.zeros((4, nx, 2))
    v0[:, :, comp] = 1e-4 * np.sin(2 * np.pi * x)[None, :]
    s = oracle_mod.OracleSim(case, None, v0)
    p = oracle_mod.params(case)
    i = nx // 4
    prev = 0.0
    zeros = []
    for k in range(1, 40 * nx):
        s.step(1)
        cur = s.fields()[0][0, i, comp]
        if k > 2 and (prev > 0 >= cur or prev < 0 <= cur):
            zeros.append(k - 1 + prev / (prev - cur))
            if len(zeros) == 5:
                return 2 * math.pi / ((zeros[4] - zeros[0]) / 2 * p["dt"]), p
        prev = cur
    raise AssertionError("too few zero crossings")


@pytest.mark.parametrize("nu", [0.0, 0.2, 0.3])
def test_wave_speeds_converge_to_navier_cauchy(oracle_mod, nu):
    """Standing shear and pressure waves oscillate at c_s k and c_d k with
    c_d^2 = (lam + 2 mu)/rho0 (Sect. 3.2): the lattice carries c_s, the
    source term corrects the dilatational speed from sqrt(3) c_s to c_d.
    The error shrinks at second order when the lattice is refined."""
    for comp in (0, 1):
        errs = []
        for nx in (32, 64):
            w, p = wave_frequency(oracle_mod, nx, comp, nu)
            speed = p["cs"] if comp == 1 else math.sqrt((p["lam"] + 2 * p["mu"]) / 1.0)
            errs.append(abs(w / (speed * 2 * math.pi) - 1))
        assert errs[1] < 2e-3
        assert 3.5 < errs[0] / errs[1] < 4.5


def test_listing_order_is_unstable_where_text_order_is_not(oracle_mod):
    """Reading of the step order: with the stress block before the
    displacement update (as Algorithm 1 is printed) the collision lags the
    source by one step and a periodic nu = 0.3 lattice blows up; with the
    order the text of Sect. 3.1 requires it stays bounded."""
    case = I.Case("o", 32, 32, 0, model="le", nu=0.3, edges=P4)
    u0, v0 = I.random_state(32, 32, 1)
    amp = {}
    for order in ("text", "listing"):
        s = oracle_mod.OracleSim(case, None, v0, order=order)
        s.step(400)
        amp[order] = np.abs(s.fields()[0]).max()
    assert amp["text"] < 1e-2
    assert not amp["listing"] < 1.0


@pytest.mark.parametrize("extrap", ["own", "linear"])
def test_mirror_symmetry(oracle_mod, extrap):
    """Tension with a clamped left edge and a normal traction on the right is
    symmetric about the horizontal mid-line: u_x even, u_y odd (with either
    reading of the wall extrapolation: a bottom wall taking its inner node
    from the wrong side breaks it)."""
    case = I.tension(10, 9, 0, ramp=50, model="nh").replace(extrap=extrap)
    s, (u, v, P) = run(oracle_mod, case, None, None, 120)
    assert np.abs(u).max() > 1e-3
    np.testing.assert_allclose(u[:, :, 0], u[::-1, :, 0], atol=1e-14)
    np.testing.assert_allclose(u[:, :, 1], -u[::-1, :, 1], atol=1e-14)


@pytest.mark.parametrize("extrap", ["own", "linear"])
def test_mirror_symmetry_left_right(oracle_mod, extrap):
    """Opposite normal tractions on the left and right edges, both free
    elsewhere: the solution is mirror symmetric about the vertical mid-line,
    u_x odd and u_y even, so the left and right walls (and their inner nodes
    under the linear reading) are treated alike."""
    left = I.Edge("neumann", "linear_ramp", (-0.02, 0.0), 0, 40)
    right = I.Edge("neumann", "linear_ramp", (0.02, 0.0), 0, 40)
    case = I.Case("lr", 11, 8, 0, model="nh", nu=0.2, edges=(left, right, I.FREE, I.FREE), extrap=extrap)
    s, (u, v, P) = run(oracle_mod, case, None, None, 90)
    assert np.abs(u).max() > 1e-3
    np.testing.assert_allclose(u[:, :, 0], -u[:, ::-1, 0], atol=1e-14)
    np.testing.assert_allclose(u[:, :, 1], u[:, ::-1, 1], atol=1e-14)


def test_linear_reading_uses_its_own_inner_nodes(oracle_mod):
    """The two readings agree while the fields next to the walls are uniform
    and part once they vary: on a tension case the linear reading changes u
    (its wall values are not the node's own), and by a small amount against
    the size of u (the correction is half a node's difference)."""
    case = I.tension(16, 12, 0, ramp=50, model="nh")
    _, (u0, _, _) = run(oracle_mod, case, None, None, 100)
    _, (u1, _, _) = run(oracle_mod, case.replace(extrap="linear"), None, None, 100)
    d = np.abs(u1 - u0).max() / np.abs(u0).max()
    assert 1e-4 < d < 0.2, d


@pytest.mark.parametrize("extrap", ["own", "linear"])
def test_transpose_symmetry(oracle_mod, extrap):
    """Swapping the roles of x and y (edges, components, lattice) gives the
    transposed solution: no axis is treated differently from the other (with
    either reading of the wall extrapolation)."""
    a = I.tension(9, 7, 0, ramp=40, model="svk").replace(extrap=extrap)
    e = a.edges
    right = e[1]
    top = I.Edge(right.kind, right.shape, (right.amp[1], right.amp[0]), right.t0, right.t1)
    b = a.replace(nx=7, ny=9, dx=a.spacing, edges=(e[2], e[3], e[0], top))
    sa, (ua, _, _) = run(oracle_mod, a.replace(dx=a.spacing), None, None, 80)
    sb, (ub, _, _) = run(oracle_mod, b, None, None, 80)
    np.testing.assert_allclose(ub.transpose(1, 0, 2)[:, :, ::-1], ua, atol=1e-14)


@pytest.mark.parametrize("extrap", ["own", "linear"])
def test_linear_material_scales_linearly(oracle_mod, extrap):
    """With the linear material every step is linear in (state, loads):
    doubling the traction doubles the displacement (both wall readings are
    linear in the node values)."""
    base = I.tension(8, 8, 0, ramp=30, model="le", nu=0.2, peak=1e-3).replace(extrap=extrap)
    dbl = I.tension(8, 8, 0, ramp=30, model="le", nu=0.2, peak=2e-3).replace(extrap=extrap)
    _, (u1, _, _) = run(oracle_mod, base, None, None, 60)
    _, (u2, _, _) = run(oracle_mod, dbl, None, None, 60)
    assert np.abs(u1).max() > 1e-6
    np.testing.assert_allclose(u2, 2 * u1, rtol=0, atol=1e-13 * np.abs(u2).max())


def homogeneous_case(I, O, model, extrap, nx=24, ny=16):
    """A block under a uniform deformation F with every edge loaded by the
    traction P(F) N of its outward normal N (Cauchy's relation): the exact
    solution is static, u = (F - I) X, P = P(F) everywhere."""
    base = I.Case("h", nx, ny, 0, model=model, nu=0.2)
    prm = O.params(base)
    H = np.array([[0.06, 0.02], [-0.01, -0.03]])
    P = O.first_piola(model, prm["lam"], prm["mu"], H).reshape(2, 2)
    T = lambda n: tuple(float(v) for v in P @ np.array(n, float))
    edges = (I.Edge("neumann", "const", T((-1, 0))), I.Edge("neumann", "const", T((1, 0))),
             I.Edge("neumann", "const", T((0, -1))), I.Edge("neumann", "const", T((0, 1))))
    case = base.replace(edges=edges, extrap=extrap)
    dx = case.spacing
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    u0 = np.stack([H[0, 0] * X + H[0, 1] * Y, H[1, 0] * X + H[1, 1] * Y], -1)
    return case, u0, P


@pytest.mark.parametrize("model", ["svk", "nh", "le"])
@pytest.mark.parametrize("extrap", ["own", "linear"])
def test_homogeneous_stress_under_its_traction_is_static(oracle_mod, model, extrap):
    """Pins the Neumann rule (Eq. abbcon with Pi* from -T* + (P + Pi(H)) N),
    the one-sided wall differences, the initial equilibrium with Pi(H0) and
    the zero source of a uniform stress: a wrong sign of T*, a transposed
    normal column or a missing Pi(H) term sets the block in motion.  Both
    readings of the wall extrapolation agree here (uniform fields)."""
    from paper_2502_00920_gb300 import inputs as I
    case, u0, P = homogeneous_case(I, oracle_mod, model, extrap)
    s = oracle_mod.OracleSim(case, u0, None)
    s.step(200)
    u, v, Pf = s.fields()
    assert np.abs(u - u0).max() <= 1e-13
    assert np.abs(v).max() <= 1e-13
    assert np.abs(Pf - P.reshape(4)).max() <= 1e-13


@pytest.mark.parametrize("xwall,ywall", [("left", None), ("right", None), (None, "bottom"), (None, "top"),
                                         ("left", "bottom"), ("right", "bottom"), ("left", "top"),
                                         ("right", "top")])
def test_linear_wall_value_is_the_field_at_the_wall(oracle_mod, xwall, ywall):
    """Pins the coefficient of the two-point reading of "extrapolated to the
    boundary" (Sect. 3.3): the wall lies half a spacing beyond the boundary
    node, so for a field that is linear across it the carried value must be
    the field at the wall position exactly (at a corner, at the corner point
    half a spacing out along both normals).  The expected value is the
    linear field evaluated at that point, not the extrapolation formula; a
    coefficient of 0, 1/4 or 1 (checked below to give another number), or an
    inner node taken from the wrong side, fails it.  The node's own value
    (the default reading) is what the other reading returns."""
    from paper_2502_00920_gb300 import inputs as I
    nx, ny = 7, 5
    alpha, beta, gamma = 3.0, 0.75, -1.25  # binary fractions: every value below is exact
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)  # node centres, spacing 1
    a = alpha + beta * X + gamma * Y
    x = {None: 2, "left": 0, "right": nx - 1}[xwall]
    y = {None: 3, "bottom": 0, "top": ny - 1}[ywall]
    # the wall position along each crossed normal; the node's own coordinate otherwise
    Xw = {None: x + 0.5, "left": 0.0, "right": float(nx)}[xwall]
    Yw = {None: y + 0.5, "bottom": 0.0, "top": float(ny)}[ywall]
    at_wall = alpha + beta * Xw + gamma * Yw
    case = I.Case("w", nx, ny, 0, model="le")
    lin = oracle_mod.wall_value(case.replace(extrap="linear"), a, x, y, xwall, ywall)
    own = oracle_mod.wall_value(case.replace(extrap="own"), a, x, y, xwall, ywall)
    assert lin == at_wall, (lin, at_wall)
    assert own == a[y, x]
    # the pin discriminates: other coefficients on the same inner nodes miss it
    xi = {None: x, "left": x + 1, "right": x - 1}[xwall]
    yi = {None: y, "bottom": y + 1, "top": y - 1}[ywall]
    for coef in (0.0, 0.25, 1.0):
        other = a[y, x] + coef * (a[y, x] - a[y, xi]) + coef * (a[y, x] - a[yi, x])
        assert other != at_wall
    # a node that is not on the named wall is refused
    assert np.isnan(oracle_mod.wall_value(case, a, 2, 2, "left", None))


def test_grid_error_norms_worked_example(oracle_mod):
    """Eq. griderror on two nodes, values checked by hand: u_ref = ((3, 4),
    (0, 0)), du = ((0, 1), (-2, 0)); ||u_ref||_2 = 5, ||du||_2 = sqrt(5),
    ||du||_inf = 2 (the larger |component| over nodes).  E2 = (1/n) sqrt(5)/5
    with n = 2, Einf = 2/5.  A dropped 1/n, the computed field's norm in the
    denominator or a maximum without absolute values each miss these."""
    u_ref = np.array([[3.0, 4.0], [0.0, 0.0]])
    u = u_ref + np.array([[0.0, 1.0], [-2.0, 0.0]])
    e2, einf = oracle_mod.grid_error(u, u_ref)
    assert abs(e2 - np.sqrt(5.0) / 10.0) <= 1e-16
    assert einf == 0.4
    # identical fields: no error; a field equal to twice the reference: du = u_ref
    assert oracle_mod.grid_error(u_ref, u_ref) == (0.0, 0.0)
    e2, einf = oracle_mod.grid_error(2 * u_ref, u_ref)
    assert abs(e2 - 0.5) <= 1e-16 and einf == 4.0 / 5.0
