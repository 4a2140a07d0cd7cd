"""The C ABI library without a GPU: it loads, exports every function that
include/*.h declares, and its host utilities agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2502_00920_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2502_00920_gb300 import build
    build.build()
    from paper_2502_00920_gb300 import lbs
    return lbs


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbs_\w+)\s*\(", src))
    return names - {"lbs_alloc_fn", "lbs_free_fn"}


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    so = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_the_header(L):
    assert declared_functions() <= set(L.SIGNATURES) | {"lbs_alloc_fn", "lbs_free_fn"} | set(
        getattr(L, "SERVE_SIGNATURES", {}))


def test_params_match_oracle(L, oracle_mod):
    for nu in (0.0, 0.25, 0.3, 0.45):
        case = I.Case("p", 10, 12, 0, nu=nu, E=2.5, rho0=1.3, dx=0.07)
        a, b = L.params(case), oracle_mod.params(case)
        for k in a:
            assert a[k] == pytest.approx(b[k], rel=1e-15)


@pytest.mark.parametrize("model", ["svk", "nh", "le"])
def test_kernel_constitutive_forms_match_oracle(L, oracle_mod, model):
    """The kernels evaluate N = P + Pi(H) in a rearranged, cancellation-free
    form; on the host (double) it must agree with the oracle's literal
    formulas of Sect. 4, for small and for large strains."""
    p = oracle_mod.params(I.Case("p", 4, 4, 0, nu=0.3))
    rng = np.random.default_rng(11)
    for scale in (1e-6, 1e-3, 0.3):
        for _ in range(25):
            H = scale * rng.normal(size=4)
            if np.linalg.det(np.eye(2) + H.reshape(2, 2)) < 0.2:
                continue
            P, N = L.constitutive(model, p["lam"], p["mu"], H)
            Po = oracle_mod.first_piola(model, p["lam"], p["mu"], H)
            No = Po + oracle_mod.pi_of_h(p["mu"], H)
            # the literal formulas subtract O(1) terms, so both sides carry an
            # absolute rounding error of order 1e-16 (times the moduli)
            np.testing.assert_allclose(P, Po, rtol=1e-12, atol=2e-15)
            np.testing.assert_allclose(N, No, rtol=1e-10, atol=2e-15)


def test_footprint_accounts_for_state(L):
    small = I.Case("f", 64, 32, 0, precision="fp32")
    fp = L.footprint(small)
    per_node = 2 * (9 * 4 + 16)  # A/B copies of g (float) and u (float pair)
    assert per_node * 64 * 32 <= fp < per_node * 64 * 32 + 64 * 1024
    assert L.footprint(small.replace(precision="fp64")) > fp > L.footprint(small.replace(precision="fp16s"))


def test_linear_wall_extrapolation_adds_a_second_side_array_layer(L):
    """LBS_EXTRAP_LINEAR keeps N at the nodes one step inwards from each wall:
    one more layer of 4 edges x max(nx, ny) x 4 entries in each of the two
    state buffers; an unknown mode is rejected before any device work."""
    import ctypes
    small = I.Case("f", 64, 32, 0, precision="fp32")
    assert L.footprint(small.replace(extrap="linear")) - L.footprint(small) == 2 * 4 * 64 * 4 * 4
    assert L.footprint(small.replace(extrap="linear", precision="fp64")) - L.footprint(
        small.replace(precision="fp64")) == 2 * 4 * 64 * 4 * 8
    lat, mat, bcs = L.structs(small)
    lat.wall_extrap = 7
    h = ctypes.c_void_p()
    assert L.lib().lbs_create(ctypes.byref(lat), ctypes.byref(mat), ctypes.byref(bcs), ctypes.byref(h)) == L.EINVAL
    assert L.lib().lbs_footprint(ctypes.byref(lat)) == 0


def test_invalid_configurations_are_rejected(L):
    bad = [I.Case("b", 2, 8, 0), I.Case("b", 8, 8, 0, tau=0.5), I.Case("b", 8, 8, 0, nu=0.5),
           I.Case("b", 8, 8, 0, edges=(I.PERIODIC, I.FREE, I.FREE, I.FREE)),
           I.Case("b", 8, 8, 0, edges=(I.Edge("neumann", "disp_ramp", (1, 0), 0, 10),) + (I.FREE,) * 3),
           I.Case("b", 8, 8, 0, edges=(I.Edge("neumann", "linear_ramp", (1, 0), 5, 5),) + (I.FREE,) * 3),
           I.Case("b", 200000, 200000, 0)]  # more than 2^34 nodes
    for c in bad:
        with pytest.raises(L.LbsError) as e:
            L.Simulation(c)
        assert e.value.code == L.EINVAL


def test_tile_variants_listed(L):
    for prec in ("fp64", "fp32", "fp16s"):
        v = L.tile_variants(prec)
        assert len(v) >= 2 and all(tx % 32 == 0 and ty > 0 for tx, ty in v)


def test_no_gpu_means_an_error_not_a_fallback(L):
    """Without a CUDA device a valid configuration is refused with LBS_ECUDA:
    the library has no CPU path to fall back to, and null handles are
    rejected before any device call."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LbsError) as e:
        L.Simulation(I.tension(32, 32, 10, ramp=5, model="nh", precision="fp32"))
    assert e.value.code == L.ECUDA
    assert L.lib().lbs_step(None, 1) == L.EINVAL
    assert L.lib().lbs_fields(None, None, None, None) == L.EINVAL
