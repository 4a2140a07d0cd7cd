"""Checkpoint / resume on the GPU: the state saved at an iteration, loaded into
the same handle or into a fresh one, continues bitwise as the uninterrupted
run; checkpoints of another configuration are refused."""
import numpy as np
import pytest

from paper_2502_00920_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_00920_gb300 import build
    build.build()
    from paper_2502_00920_gb300 import lbs
    return lbs


def case(precision, extrap="own"):
    trac = I.Edge("neumann", "linear_ramp", (0.01, -0.005), 0, 120)
    return I.Case("ck", 70, 45, 0, model="nh", nu=0.2, edges=(I.CLAMPED, trac, I.FREE, I.FREE),
                  precision=precision, extrap=extrap)


@pytest.mark.parametrize("extrap", ["own", "linear"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_resume_is_bitwise(L, precision, extrap):
    """With the linear wall reading the checkpoint carries both layers of the
    boundary side array."""
    c = case(precision, extrap)
    with L.Simulation(c) as a:
        a.step(130)  # two graph chunks and two direct iterations: buffers swapped
        ck = a.save()
        a.step(170)
        a.sync()
        ref = a.fields()
        assert a.iteration == 300
        a.load(ck)
        assert a.iteration == 130
        a.step(170)
        a.sync()
        again = a.fields()
    with L.Simulation(c) as b:
        b.load(ck)
        b.step(170)
        b.sync()
        fresh = b.fields()
    assert np.isfinite(ref[0]).all() and np.abs(ref[0]).max() > 1e-6
    for x, y, z in zip(ref, again, fresh):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_load_refuses_other_configurations(L):
    with L.Simulation(case("fp32")) as a:
        a.step(10)
        ck = a.save()
    for other in (case("fp32").replace(nx=71), case("fp64"), case("fp32").replace(nu=0.25), case("fp32", "linear")):
        with L.Simulation(other) as b:
            with pytest.raises(L.LbsError) as e:
                b.load(ck)
            assert e.value.code == L.EINVAL
    with L.Simulation(case("fp32")) as b:
        with pytest.raises(L.LbsError):
            b.load(ck[:100])
        bad = ck.copy()
        bad[0] ^= 1
        with pytest.raises(L.LbsError):
            b.load(bad)
