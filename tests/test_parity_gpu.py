"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (relative max norm over nodes and components):
  FP64 storage and arithmetic ....... 1e-12 on u and v (the stated target)
  FP32 storage, u as a float pair ... 1e-5 on u
  FP16 storage (scaled), FP32 math .. 1e-2 on u
Stresses P are compared at 1e-10 (FP64): the oracle evaluates the printed
formulas, whose rounding error is absolute (order 1e-16 times the moduli).
"""
import math

import numpy as np
import pytest

from paper_2502_00920_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16s": 1e-2}


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_00920_gb300 import build
    build.build()
    from paper_2502_00920_gb300 import lbs
    return lbs


ERRORS = {}


@pytest.fixture(scope="module", autouse=True)
def _error_report():
    """With LBS_ERROR_REPORT set to a directory, write every measured error
    to parity_errors.json there (for the record); otherwise write nothing."""
    yield
    import json
    import os
    out = os.environ.get("LBS_ERROR_REPORT")
    if not out:
        return
    try:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "parity_errors.json"), "w") as f:
            json.dump(ERRORS, f, indent=1, sort_keys=True)
    except OSError:
        pass


def record(key, **errs):
    ERRORS[key] = {k: float(v) for k, v in errs.items()}


def rel(a, b):
    d = np.abs(b).max()
    return np.abs(a - b).max() / (d if d > 0 else 1.0)


def run_gpu(L, case, steps, u0=None, v0=None, **kw):
    with L.Simulation(case, **kw) as s:
        if u0 is not None or v0 is not None:
            s.set_initial(u0, v0)
        s.step(steps)
        s.sync()
        return s.fields()


def run_oracle(O, case, steps, u0=None, v0=None):
    o = O.OracleSim(case, u0, v0)
    o.step(steps)
    return o.fields()


def rnd(case, seed=3, amp_u=1e-2, amp_v=2e-2):
    return I.random_state(case.nx, case.ny, seed, amp_u=amp_u, amp_v=amp_v)


def CASES():
    P4 = (I.PERIODIC,) * 4
    mov = I.Edge("dirichlet", "const", (0.01, -0.004))
    trac = I.Edge("neumann", "sin2_ramp", (0.02, 0.01), 0, 60)
    return {
        "tension_32_nh": (I.tension(32, 32, 0, ramp=200, model="nh"), 300, False),
        "tension_32_svk": (I.tension(32, 32, 0, ramp=200, model="svk", nu=0.2), 300, False),
        "periodic_40x24_nh": (I.Case("p", 40, 24, 0, model="nh", edges=P4), 200, True),
        "periodic_130x90_svk": (I.Case("p", 130, 90, 0, model="svk", nu=0.2, edges=P4), 150, True),
        "periodic_71x69_le_body": (I.Case("p", 71, 69, 0, model="le", nu=0.1, edges=P4, body=(0.01, -0.02)), 150, True),
        "shear_64_svk": (I.shear(64, 0, model="svk", nu=0.2, gamma=0.05, ramp=400), 300, False),
        "mixed_37x29": (I.Case("m", 37, 29, 0, model="nh", nu=0.2, edges=(mov, trac, I.FREE, I.CLAMPED)), 200, True),
        "walls_150x100_nh": (I.tension(150, 100, 0, ramp=100, model="nh", nu=0.25, peak=0.05), 200, False),
        "corners_nn_45x33": (I.Case("c", 45, 33, 0, model="nh", nu=0.2,
                                    edges=(trac, I.FREE, I.Edge("neumann", "linear_ramp", (0.0, -0.02), 0, 50), I.FREE)),
                             150, True),
        "cantilever_256x32": (I.cantilever(256, 32, 0, width=100, amp=0.02, nu=0.25, precision="fp64"), 300, False),
        "periodic_x_walls_y_64x40": (I.Case("py", 64, 40, 0, model="svk", nu=0.25,
                                            edges=(I.PERIODIC, I.PERIODIC, I.CLAMPED, trac)), 200, True),
    }


@pytest.mark.parametrize("name", list(CASES()))
def test_fp64_matches_oracle(L, oracle_mod, name):
    case, steps, random_init = CASES()[name]
    case = case.replace(precision="fp64")
    u0, v0 = rnd(case) if random_init else (None, None)
    u, v, P = run_gpu(L, case, steps, u0, v0)
    ur, vr, Pr = run_oracle(oracle_mod, case, steps, u0, v0)
    record(f"fp64/{name}", u=rel(u, ur), v=rel(v, vr), P=rel(P, Pr))
    assert np.isfinite(ur).all() and np.abs(ur).max() > 1e-6
    assert rel(u, ur) <= TOL["fp64"], rel(u, ur)
    assert rel(v, vr) <= TOL["fp64"], rel(v, vr)
    assert rel(P, Pr) <= 1e-10, rel(P, Pr)


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
@pytest.mark.parametrize("name", ["tension_32_nh", "periodic_130x90_svk", "shear_64_svk", "mixed_37x29",
                                  "cantilever_256x32"])
def test_reduced_precision_matches_oracle(L, oracle_mod, name, precision):
    case, steps, random_init = CASES()[name]
    u0, v0 = rnd(case) if random_init else (None, None)
    u, v, P = run_gpu(L, case.replace(precision=precision), steps, u0, v0)
    ur, vr, Pr = run_oracle(oracle_mod, case, steps, u0, v0)
    record(f"{precision}/{name}", u=rel(u, ur), v=rel(v, vr), P=rel(P, Pr))
    assert rel(u, ur) <= TOL[precision], rel(u, ur)


def test_initial_state_round_trip(L, oracle_mod):
    """Iteration 0: the fields reproduce u0, v0 exactly as Alg. 1 initialises."""
    case = I.Case("i", 33, 21, 0, model="nh", edges=(I.FREE, I.CLAMPED, I.FREE, I.FREE))
    u0, v0 = rnd(case)
    u, v, P = run_gpu(L, case, 0, u0, v0)
    ur, vr, Pr = run_oracle(oracle_mod, case, 0, u0, v0)
    assert rel(u, u0) == 0.0
    assert rel(v, v0) <= 1e-14
    assert rel(P, Pr) <= 1e-12


@pytest.mark.parametrize("walls", ["periodic", "dirichlet", "neumann"])
def test_uniform_translation_exact(L, walls):
    """u = u0 + k dt v0 to rounding, the closed form the oracle is pinned to."""
    v = np.array([0.013, -0.021])
    mov = I.Edge("dirichlet", "const", tuple(v))
    edges = {"periodic": (I.PERIODIC,) * 4, "dirichlet": (mov,) * 4, "neumann": (I.FREE,) * 4}[walls]
    case = I.Case("t", 70, 50, 0, model="nh", edges=edges)
    u0 = np.broadcast_to([0.1, -0.05], (50, 70, 2)).copy()
    v0 = np.broadcast_to(v, (50, 70, 2)).copy()
    u, vv, P = run_gpu(L, case, 40, u0, v0)
    dt = L.params(case)["dt"]
    np.testing.assert_allclose(u, u0 + 40 * dt * v, atol=1e-14)
    np.testing.assert_allclose(vv, v0, atol=1e-14)


def test_graph_and_direct_launches_agree_bitwise(L):
    case = I.tension(48, 40, 0, ramp=50, model="nh", precision="fp32")
    a = run_gpu(L, case, 150, graph_chunk=0)
    b = run_gpu(L, case, 150, graph_chunk=16)
    c = run_gpu(L, case, 150, graph_chunk=64)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_tile_variants_agree_bitwise(L, precision):
    """Every tile shape computes each node with the same operations."""
    case = I.Case("v", 150, 70, 0, model="svk", nu=0.2, precision=precision,
                  edges=(I.CLAMPED, I.Edge("neumann", "linear_ramp", (0.01, 0.0), 0, 50), I.FREE, I.FREE))
    outs = [run_gpu(L, case, 60, variant=v) for v in range(len(L.tile_variants(precision)))]
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("steps,chunk", [(61, 0), (64, 16), (131, 64)])
def test_fused_iterations_equal_single_ones_bitwise(L, oracle_mod, steps, chunk):
    """The two-iterations-per-launch variant (periodic lattices) computes
    every node with the single-iteration arithmetic: equal bitwise to the
    default variant over even and odd iteration counts, direct launches and
    graphs, on lattices with ragged tiles and frame tiles; and it matches the
    oracle at the FP64 bar's FP32 counterpart."""
    fused = next(v for v in range(len(L.tile_variants("fp32"))) if L.tile_variant_name("fp32", v) ==
                 "step_fused2_tma_kernel")
    for nx, ny in ((130, 90), (256, 100), (40, 40)):
        case = I.Case("f", nx, ny, 0, model="nh", nu=0.3, precision="fp32", edges=(I.PERIODIC,) * 4)
        u0, v0 = rnd(case)
        a = run_gpu(L, case, steps, u0, v0, graph_chunk=chunk)
        b = run_gpu(L, case, steps, u0, v0, graph_chunk=chunk, variant=fused)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), (nx, ny)
    ur = run_oracle(oracle_mod, case, steps, u0, v0)[0]
    assert rel(b[0], ur) <= TOL["fp32"]


def test_grid_error_norms_match_the_oracle(L, oracle_mod):
    """lbs_grid_error (host and device reference) against the oracle's
    Eq. griderror on the same fields: the norms of the GPU's u against a
    seeded reference."""
    import torch
    case = I.tension(70, 45, 0, ramp=50, model="nh", precision="fp32")
    ref, _ = I.random_state(case.nx, case.ny, 11, amp_u=2e-3)
    with L.Simulation(case) as s:
        s.step(120)
        s.sync()
        u = s.fields(True, False, False)[0]
        host = s.grid_error(ref)
        dev = s.grid_error(torch.as_tensor(ref, device="cuda"))
    want = oracle_mod.grid_error(u, ref)
    for got in (host, dev):
        assert abs(got[0] - want[0]) <= 1e-13 * want[0] and abs(got[1] - want[1]) <= 1e-13 * want[1], (got, want)


def test_monitor_matches_oracle(L, oracle_mod):
    """max|u| and the total momentum (sum of the first moment of the stored
    post-collision populations = rho0 sum v on a periodic lattice without body
    force) against the oracle at the same iteration."""
    case = I.Case("m", 64, 48, 0, model="nh", edges=(I.PERIODIC,) * 4)
    u0, v0 = rnd(case)
    with L.Simulation(case, u0=u0, v0=v0) as s:
        s.step(80)
        m = s.monitor()
    ur, vr, _ = run_oracle(oracle_mod, case, 80, u0, v0)
    assert m["nonfinite"] == 0 and m["iteration"] == 80
    assert m["max_abs_u"] == pytest.approx(np.abs(ur).max(), rel=1e-12)
    np.testing.assert_allclose(m["momentum"], case.rho0 * vr.sum(axis=(0, 1)), rtol=1e-9, atol=1e-12)


def test_probe_matches_oracle(L, oracle_mod):
    case = I.cantilever(128, 16, 0, width=50, amp=0.02, nu=0.25, precision="fp64")
    with L.Simulation(case) as s:
        s.step(100)
        nodes = [8 * 128 + 127, 0, 15 * 128 + 64]
        pr = s.probe(nodes)
    ur, _, _ = run_oracle(oracle_mod, case, 100)
    flat = ur.reshape(-1, 2)
    np.testing.assert_allclose(pr, flat[nodes], rtol=1e-12, atol=1e-16)


def test_instability_reported(L, oracle_mod):
    """A configuration beyond the scheme's stability (nu = 0.45 on a periodic
    lattice) goes non-finite in both codes; the library reports it as
    LBS_EUNSTABLE at the first monitor after the oracle's blow-up."""
    case = I.Case("u", 32, 32, 0, model="le", nu=0.45, edges=(I.PERIODIC,) * 4)
    u0, v0 = rnd(case)
    o = oracle_mod.OracleSim(case, u0, v0)
    k_nan = None
    for k in range(1, 2000):
        o.step(1)
        if not np.isfinite(o.fields()[0]).all():
            k_nan = k
            break
    assert k_nan is not None
    with L.Simulation(case, u0=u0, v0=v0, monitor_interval=10, graph_chunk=0) as s:
        with pytest.raises(L.LbsError) as e:
            for _ in range(0, 2000, 10):
                s.step(10)
                s.sync()
        assert e.value.code == L.EUNSTABLE
        assert k_nan <= s.unstable_iteration <= k_nan + 10


def test_device_fields_and_initial(L, oracle_mod):
    import torch
    case = I.Case("d", 50, 30, 0, model="nh", edges=(I.PERIODIC,) * 4)
    u0, v0 = rnd(case)
    dev = torch.device("cuda")
    tu, tv = torch.tensor(u0, device=dev), torch.tensor(v0, device=dev)
    with L.Simulation(case) as s:
        s.set_initial(tu, tv)
        s.step(50)
        out = [torch.empty((30, 50, w), dtype=torch.float64, device=dev) for w in (2, 2, 4)]
        s.fields_device(*out)
        s.sync()
        hu, hv, hP = s.fields()
    assert np.array_equal(out[0].cpu().numpy(), hu) and np.array_equal(out[2].cpu().numpy(), hP)
    ur, vr, _ = run_oracle(oracle_mod, case, 50, u0, v0)
    assert rel(hu, ur) <= 1e-12


# ---------------------------------------------------------------- full-size workloads

def light_cone_windows(L, oracle_mod, case, steps, starts, w=32, precision="fp64", graph_chunk=None):
    """Run the whole periodic lattice on the GPU; for each window, run the
    oracle on the window plus a margin wider than the distance information
    travels in `steps` iterations (3 nodes per iteration plus the
    initialisation stencil) and compare the window interior."""
    import torch
    margin = 3 * steps + 8
    dev = torch.device("cuda")
    v0 = I.grf_velocity(case, device=dev)
    kw = {} if graph_chunk is None else dict(graph_chunk=graph_chunk)
    with L.Simulation(case.replace(precision=precision), **kw) as s:
        s.set_initial(None, v0)
        s.step(steps)
        s.sync()
        u = torch.empty((case.ny, case.nx, 2), dtype=torch.float64, device=dev)
        v = torch.empty_like(u)
        s.fields_device(u, v, None)
        s.sync()
    errs = []
    for (x0, y0) in starts:
        xs = (np.arange(x0 - margin, x0 + w + margin) % case.nx)
        ys = (np.arange(y0 - margin, y0 + w + margin) % case.ny)
        xi, yi = torch.tensor(xs, device=dev), torch.tensor(ys, device=dev)
        vw = v0.index_select(0, yi).index_select(1, xi).cpu().numpy()
        W = w + 2 * margin
        wcase = case.replace(nx=W, ny=W, dx=case.spacing, edges=(I.FREE,) * 4, precision="fp64")
        ur, vr, _ = run_oracle(oracle_mod, wcase, steps, None, vw)
        ug = u.index_select(0, yi).index_select(1, xi).cpu().numpy()
        vg = v.index_select(0, yi).index_select(1, xi).cpu().numpy()
        sl = (slice(margin, margin + w), slice(margin, margin + w))
        scale = np.abs(ur[sl]).max()
        errs.append((np.abs(ug[sl] - ur[sl]).max() / scale, np.abs(vg[sl] - vr[sl]).max() / np.abs(vr[sl]).max()))
    return errs


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_roofline_lattice_16384_windows(L, oracle_mod, precision):
    """The benchmark workload at full size (16384^2 periodic, neo-Hooke,
    random initial velocity) in the benchmark's launch configuration, checked
    on windows (including ones that wrap around the periodic edges)."""
    case = I.roofline(n=16384, nsteps=6)
    starts = [(0, 0), (16384 - 16, 100), (8000, 16384 - 20), (12345, 6789)]
    errs = light_cone_windows(L, oracle_mod, case, 6, starts, precision=precision, graph_chunk=64)
    record(f"{precision}/roofline_16384_windows", u=max(e[0] for e in errs), v=max(e[1] for e in errs))
    for eu, ev in errs:
        assert eu <= TOL[precision], errs
        if precision == "fp64":
            assert ev <= TOL[precision], errs


def test_shear_256_sweep(L, oracle_mod):
    """Simple-shear workload at full lattice size, all six Poisson ratios."""
    for nu in (0.0, 0.1, 0.2, 0.3, 0.4, 0.45):
        case = I.shear(256, 0, model="svk", nu=nu, gamma=0.5, ramp=20000)
        u, v, P = run_gpu(L, case, 400)
        ur, vr, Pr = run_oracle(oracle_mod, case, 400)
        if not np.isfinite(ur).all():
            continue
        record(f"fp64/shear_256_nu{nu}", u=rel(u, ur), v=rel(v, vr), P=rel(P, Pr))
        assert rel(u, ur) <= 1e-12 and rel(v, vr) <= 1e-12, (nu, rel(u, ur))


def test_cantilever_4096x256(L, oracle_mod):
    """Bending-wave workload at full lattice size (pulse phase)."""
    case = I.cantilever(4096, 256, 0, precision="fp64")
    u, v, P = run_gpu(L, case, 250)
    ur, vr, Pr = run_oracle(oracle_mod, case, 250)
    u32 = run_gpu(L, case.replace(precision="fp32"), 250)[0]
    record("fp64/cantilever_4096x256", u=rel(u, ur), v=rel(v, vr), P=rel(P, Pr))
    record("fp32/cantilever_4096x256", u=rel(u32, ur))
    assert rel(u, ur) <= 1e-12 and rel(v, vr) <= 1e-12
    assert rel(u32, ur) <= 1e-5


def test_tension_32_full_history(L, oracle_mod):
    """Uniaxial-tension workload (32x32, 2000 iterations).  Both codes either
    stay finite and agree, or go non-finite: the library then reports
    LBS_EUNSTABLE at a monitor within one interval of the oracle's blow-up."""
    case = I.tension(32, 32, 2000)
    o = oracle_mod.OracleSim(case)
    k_nan = None
    for k in range(0, 2000, 50):
        o.step(50)
        if not np.isfinite(o.fields()[0]).all():
            k_nan = k + 50
            break
    with L.Simulation(case, monitor_interval=50, graph_chunk=0) as s:
        if k_nan is None:
            s.step(2000)
            s.sync()
            u = s.fields()[0]
            assert rel(u, o.fields()[0]) <= 1e-12
        else:
            with pytest.raises(L.LbsError):
                for _ in range(40):
                    s.step(50)
                    s.sync()
            assert abs(s.unstable_iteration - k_nan) <= 50
            # the agreement holds until the growth sets in
    with L.Simulation(case) as s:
        s.step(1000)
        s.sync()
        u = s.fields()[0]
    ur = run_oracle(oracle_mod, case, 1000)[0]
    assert rel(u, ur) <= 1e-12


def paper_cases():
    """The paper's own examples at its lattice sizes (Sect. 4): 40 x 40
    tension and shear to t = 2.2, the 160 x 40 bending wave to t = 12 at each
    relaxation time of the paper's sweep (0.54, 0.55, 0.57, 0.59)."""
    return {
        "paper_tension_nh_0.3": (I.paper_tension("nh", 0.3), 2.2),
        "paper_tension_svk_0.25": (I.paper_tension("svk", 0.25), 2.2),
        "paper_shear_nh_0.3": (I.paper_shear("nh", 0.3), 2.2),
        "paper_shear_svk_0.2": (I.paper_shear("svk", 0.2), 2.2),
        "paper_wave_tau0.54": (I.paper_wave(0.54), 12.0),
        "paper_wave_tau0.55": (I.paper_wave(0.55), 12.0),
        "paper_wave_tau0.57": (I.paper_wave(0.57), 12.0),
        "paper_wave_tau0.59": (I.paper_wave(0.59), 12.0),
    }


@pytest.mark.parametrize("name", list(paper_cases()))
def test_paper_examples_match_oracle(L, oracle_mod, name):
    """GPU FP64 against the oracle over the paper's whole horizon, with the
    loads given in the paper's time unit."""
    case, T = paper_cases()[name]
    steps = int(round(T / oracle_mod.params(case)["dt"]))
    u, v, P = run_gpu(L, case, steps)
    ur, vr, Pr = run_oracle(oracle_mod, case, steps)
    record(f"fp64/{name}", u=rel(u, ur), v=rel(v, vr), P=rel(P, Pr))
    assert np.isfinite(ur).all() and np.abs(ur).max() > 1e-4
    assert rel(u, ur) <= TOL["fp64"], rel(u, ur)
    assert rel(v, vr) <= TOL["fp64"], rel(v, vr)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6), ("fp16s", 1e-2)])
@pytest.mark.parametrize("model", ["svk", "nh"])
def test_homogeneous_stress_under_its_traction_is_static(L, oracle_mod, model, precision, tol):
    """A block under uniform F with every edge loaded by P(F) N stays at
    u = (F - I) X with P = P(F) (the exact static solution; the oracle is
    pinned to it on the host)."""
    from test_oracle_pins import homogeneous_case
    case, u0, P = homogeneous_case(I, oracle_mod, model, "own")
    u, v, Pf = run_gpu(L, case.replace(precision=precision), 200, u0, None)
    scale = np.abs(u0).max()
    record(f"{precision}/homogeneous_{model}", u=float(np.abs(u - u0).max() / scale),
           P=float(np.abs(Pf - P.reshape(4)).max() / np.abs(P).max()))
    # the stored populations of the static state are not exact in reduced
    # precision: the bar on u is each precision's parity bar
    assert np.abs(u - u0).max() <= tol * scale
    assert np.abs(Pf - P.reshape(4)).max() <= tol * 5 * np.abs(P).max()


def shape_cases():
    """Degenerate and ragged shapes: lattices three nodes wide (every node on
    a wall, or a 3-node periodic ring whose halos wrap more than once),
    lattices smaller than one tile, exact multiples of the tile sizes and one
    node more, and a material with rho0 != 1 and E != 1."""
    trac = I.Edge("neumann", "linear_ramp", (0.01, -0.004), 0, 40)
    mov = I.Edge("dirichlet", "const", (0.002, 0.001))
    P2 = (I.PERIODIC, I.PERIODIC)
    return {
        "3x3_mixed": I.Case("s", 3, 3, 0, model="nh", nu=0.2, edges=(I.CLAMPED, trac, I.FREE, mov)),
        "3x40_walls": I.Case("s", 3, 40, 0, model="svk", nu=0.1, edges=(I.FREE, I.FREE, I.CLAMPED, trac)),
        "40x3_walls": I.Case("s", 40, 3, 0, model="nh", nu=0.1, edges=(I.CLAMPED, trac, I.FREE, I.FREE)),
        "3x7_periodic_x": I.Case("s", 3, 7, 0, model="nh", nu=0.2, edges=P2 + (I.CLAMPED, trac)),
        "5x5_periodic": I.Case("s", 5, 5, 0, model="svk", nu=0.2, edges=P2 + P2),
        "17x9_sub_tile": I.Case("s", 17, 9, 0, model="nh", nu=0.25, edges=(I.CLAMPED, trac, I.FREE, I.FREE)),
        "64x48_tile_multiple": I.Case("s", 64, 48, 0, model="nh", nu=0.2, edges=(I.CLAMPED, trac, I.FREE, I.FREE)),
        "65x49_one_more": I.Case("s", 65, 49, 0, model="nh", nu=0.2, edges=(I.CLAMPED, trac, I.FREE, I.FREE)),
        "rho2.5_E3": I.Case("s", 41, 27, 0, model="nh", nu=0.2, E=3.0, rho0=2.5,
                            edges=(I.CLAMPED, trac, I.FREE, mov)),
    }


@pytest.mark.parametrize("name", list(shape_cases()))
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_degenerate_and_ragged_shapes_match_oracle(L, oracle_mod, name, precision):
    case = shape_cases()[name].replace(precision=precision)
    u0, v0 = rnd(case, amp_u=2e-3, amp_v=4e-3) if case.edges[0].kind == "periodic" else (None, None)
    u, v, P = run_gpu(L, case, 80, u0, v0)
    ur, vr, Pr = run_oracle(oracle_mod, case, 80, u0, v0)
    record(f"{precision}/shape_{name}", u=rel(u, ur), v=rel(v, vr), P=rel(P, Pr))
    assert np.isfinite(ur).all() and np.abs(ur).max() > 1e-7
    assert rel(u, ur) <= TOL[precision], rel(u, ur)
    if precision == "fp64":
        assert rel(v, vr) <= TOL["fp64"], rel(v, vr)


@pytest.mark.parametrize("scale", [0, 6, 12, 16])
def test_fp16_storage_scale(L, oracle_mod, scale):
    """FP16 storage keeps g * 2^gscale_log2: any scale that keeps the
    populations inside half precision's range meets the FP16 bar (0 picks
    2^12 for rho0 = 1)."""
    case, steps, _ = CASES()["tension_32_nh"]
    u, v, P = run_gpu(L, case.replace(precision="fp16s", gscale_log2=scale), steps)
    ur = run_oracle(oracle_mod, case, steps)[0]
    assert rel(u, ur) <= TOL["fp16s"], rel(u, ur)


def test_fp16_scale_that_overflows_is_reported(L):
    """2^30 times populations of order 0.1 overflows half precision: the run
    is reported non-finite (LBS_EUNSTABLE), not returned as a result."""
    case, steps, _ = CASES()["tension_32_nh"]
    with L.Simulation(case.replace(precision="fp16s", gscale_log2=30), monitor_interval=10) as s:
        with pytest.raises(L.LbsError) as e:
            s.step(steps)
            s.sync()
        assert e.value.code == L.EUNSTABLE
