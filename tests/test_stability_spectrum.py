"""Linear stability of one iteration (CPU, the oracle).

With the linear test material and zero prescribed values, one iteration of
the scheme (Algorithm 1, text order) is a linear map of the state it carries
(distributions, displacement, and the stresses and source computed from it).
These tests build that map's matrix on a 12 x 12 lattice column by column
(one oracle iteration per unit vector) and take its eigenvalues: a spectral
radius above 1 means that any perturbation, rounding included, grows by that
factor per iteration.  They pin what the analysis found:

  - periodic and Dirichlet (bounce-back) edges are neutral (|lambda| <= 1);
  - the Neumann (anti-bounce-back) edge of Sect. 3.3 is stable only where the
    non-linear extension adds nothing to the linear scheme it builds on
    (nu = 1/4, i.e. lambda = mu, so that P + Pi(H) = (lambda - mu) tr H I
    vanishes) and tau is not too close to 1/2;
  - for nu > 1/4 (outside the bound nu <= 1/4 that Sect. 3.2 states for
    first-order boundary stencils) a flat Neumann edge grows by more than 1 %
    per iteration on this lattice, whatever tau;
  - for 0 <= nu < 1/4 it grows more slowly, faster with Neumann-Neumann
    corners.

Run as a script it prints the table the design notes quote.
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2502_00920_gb300 import inputs as I  # noqa: E402

N, P, D = I.FREE, I.PERIODIC, I.CLAMPED
EDGES = {
    "all Neumann": (N, N, N, N),
    "periodic x, Neumann y": (P, P, N, N),
    "Dirichlet left, Neumann else": (D, N, N, N),
    "periodic x, Dirichlet y": (P, P, D, D),
    "all Dirichlet": (D, D, D, D),
    "all periodic": (P, P, P, P),
}


# |lambda| = 1 is a defective eigenvalue of these maps (a rigid translation at
# constant velocity grows linearly), which dense eigensolvers return to about
# the square root of the rounding unit: "neutral" means within 1e-6 of 1
NEUTRAL = 1.0 + 1e-6


def spectral_radius(O, edges, n=12, nu=0.3, tau=0.55, extrap="own", order="text"):
    """Largest |eigenvalue| of the one-iteration map of the linear material
    with zero prescribed values on an n x n lattice."""
    case = I.Case("spectrum", n, n, 0, model="le", nu=nu, tau=tau, edges=edges, extrap=extrap)
    sim = O.OracleSim(case, order=order)
    dim = sim.state().size
    A = np.empty((dim, dim))
    e = np.zeros(dim)
    for i in range(dim):
        e[i] = 1.0
        sim.set_state(e)
        sim.step(1)
        A[:, i] = sim.state()
        e[i] = 0.0
    return float(np.abs(np.linalg.eigvals(A)).max())


def test_the_state_round_trips(oracle_mod):
    """The carried state is all an iteration reads: restoring it into a
    fresh simulation continues the same trajectory bitwise."""
    case = I.Case("rt", 9, 7, 0, model="le", nu=0.2, edges=(D, N, N, N))
    u0, v0 = I.random_state(9, 7, 2)
    a = oracle_mod.OracleSim(case, u0, v0)
    a.step(4)
    b = oracle_mod.OracleSim(case)
    b.set_state(a.state())
    a.step(3)
    b.step(3)
    assert np.array_equal(a.state(), b.state())


@pytest.mark.parametrize("name", ["all Dirichlet", "periodic x, Dirichlet y", "all periodic"])
def test_periodic_and_dirichlet_edges_are_neutral(oracle_mod, name):
    rho = spectral_radius(oracle_mod, EDGES[name], nu=0.3)
    assert rho <= NEUTRAL, rho


def test_neumann_edge_is_stable_where_the_extension_adds_nothing(oracle_mod):
    """nu = 1/4: lambda = mu, P + Pi(H) = 0 for the linear material, and the
    scheme is the linear one with anti-bounce-back walls: neutral for
    tau >= 0.58, still slightly growing at tau = 0.55."""
    assert spectral_radius(oracle_mod, EDGES["periodic x, Neumann y"], nu=0.25, tau=0.7) <= NEUTRAL
    assert spectral_radius(oracle_mod, EDGES["all Neumann"], nu=0.25, tau=0.7) <= NEUTRAL
    assert 1.0005 < spectral_radius(oracle_mod, EDGES["periodic x, Neumann y"], nu=0.25, tau=0.55) < 1.005


@pytest.mark.parametrize("tau", [0.55, 0.7, 1.0])
def test_neumann_edge_beyond_the_cfl_bound_grows(oracle_mod, tau):
    """nu = 0.3 > 1/4: a flat Neumann edge (no corner) grows by 1.35 % per
    iteration on the 12 x 12 lattice, independent of tau."""
    rho = spectral_radius(oracle_mod, EDGES["periodic x, Neumann y"], nu=0.3, tau=tau)
    assert 1.01 < rho < 1.02, rho


def test_neumann_edge_below_the_bound_grows_slowly(oracle_mod):
    """nu = 0.2 at tau = 0.55: the flat edge grows by 0.3 % per iteration;
    Neumann-Neumann corners at nu = 0 by 1.8 %."""
    strip = spectral_radius(oracle_mod, EDGES["periodic x, Neumann y"], nu=0.2)
    assert 1.001 < strip < 1.005, strip
    corners = spectral_radius(oracle_mod, EDGES["all Neumann"], nu=0.0)
    assert 1.01 < corners < 1.03, corners


def test_growth_of_the_static_block_under_the_linear_reading(oracle_mod):
    """The 24 x 16 block with every edge Neumann at nu = 0.2 (the static
    homogeneous-stress test of the GPU path) is close to neutral with the
    node's own wall values and grows by about 1.5 % per iteration with the
    two-point reading: about 19x over 200 iterations (the GPU test widens
    its reduced-precision bar by 20x for that reading only)."""
    import scipy.sparse.linalg as sla
    for extrap, lo, hi in (("own", 1.0, 1.0005), ("linear", 1.012, 1.0151)):
        case = I.Case("h", 24, 16, 0, model="le", nu=0.2, edges=EDGES["all Neumann"], extrap=extrap)
        sim = oracle_mod.OracleSim(case)
        dim = sim.state().size

        def step(x):
            sim.set_state(x)
            sim.step(1)
            return sim.state()

        op = sla.LinearOperator((dim, dim), matvec=step, dtype=np.float64)
        vals = sla.eigs(op, k=6, which="LM", v0=np.random.default_rng(0).standard_normal(dim), maxiter=20000,
                        tol=1e-12, return_eigenvectors=False)
        rho = float(np.abs(vals).max())
        assert lo <= rho <= hi, (extrap, rho)


def table(O):
    rows = []
    for name, edges in EDGES.items():
        for nu in (0.0, 0.2, 0.25, 0.3, 0.45):
            r = [spectral_radius(O, edges, nu=nu, tau=t) for t in (0.55, 0.7)]
            r.append(spectral_radius(O, edges, nu=nu, extrap="linear"))
            r.append(spectral_radius(O, edges, nu=nu, order="listing"))
            rows.append((name, nu, r))
            print(f"| {name} | {nu} | " + " | ".join(f"{x:.5f}" for x in r) + " |", flush=True)
    return rows


if __name__ == "__main__":
    from oracle import oracle as O
    print("| edges | nu | tau 0.55 | tau 0.7 | linear wall reading | listing order |")
    print("|---|---|---|---|---|---|")
    table(O)
