"""The configuration side of the C ABI on the GPU: the autotuner and its
cache file, the allocator hook, caller streams, launch counting, device
bytes and the CFL flag.  Results never depend on these choices: every run
here is compared bitwise with the same lattice run with the defaults."""
import ctypes
import json

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


def case(precision="fp32", nx=96, ny=64, nu=0.2):
    trac = I.Edge("neumann", "linear_ramp", (0.01, -0.004), 0, 60)
    return I.Case("a", nx, ny, 0, model="nh", nu=nu, edges=(I.CLAMPED, trac, I.FREE, I.FREE), precision=precision)


def run(L, c, steps=130, **kw):
    with L.Simulation(c, **kw) as s:
        s.step(steps)
        s.sync()
        return s.fields()


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_autotune_picks_the_fastest_and_caches(L, tmp_path):
    c = case(nx=300, ny=200)
    best, ms = L.autotune(c, steps=5)
    assert len(ms) == len(L.tile_variants("fp32")) and min(ms) > 0
    assert best == int(np.argmin(ms))
    assert L.autotune(c, steps=5) == (best, ms)  # cached: not timed again
    with L.Simulation(c, variant="auto") as s:
        assert s.variant == best
    assert same(run(L, c, variant="auto"), run(L, c))
    path = tmp_path / "tune.jsonl"
    L.autotune_save(str(path))
    rows = [json.loads(line) for line in path.read_text().splitlines()]
    assert any(r["nx"] == 300 and r["ny"] == 200 and r["variant"] == best for r in rows)


def test_autotune_cache_file_with_extra_and_bad_entries(L, tmp_path):
    """A cache line with more timings than this build has variants fills only
    the caller's per-variant array; lines with unknown variants are skipped."""
    nvar = len(L.tile_variants("fp32"))
    path = tmp_path / "tune.jsonl"
    lines = [{"nx": 123, "ny": 45, "precision": 1, "model": 1, "per_x": 0, "per_y": 0, "variant": 2,
              "ms": [float(i + 1) for i in range(40)]},
             {"nx": 124, "ny": 45, "precision": 1, "model": 1, "per_x": 0, "per_y": 0, "variant": 99, "ms": [1.0]}]
    path.write_text("\n".join(json.dumps(r) for r in lines) + "\n")
    L.autotune_load(str(path))
    best, ms = L.autotune(case(nx=123, ny=45), steps=3)
    assert best == 2 and ms == [float(i + 1) for i in range(nvar)]
    best, ms = L.autotune(case(nx=124, ny=45), steps=3)  # the bad line was skipped: timed now
    assert 0 <= best < nvar and best == int(np.argmin(ms))


def test_custom_allocator(L):
    """Handle state from a caller's allocator (here torch's caching
    allocator); misaligned blocks are refused."""
    import torch
    live, calls = {}, {"alloc": 0, "free": 0}
    AF = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FF = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

    def alloc(nbytes, stream, ctx):
        p = torch.cuda.caching_allocator_alloc(nbytes + 512)
        calls["alloc"] += 1
        off = 0 if not ctx else 16  # ctx != 0: hand out a misaligned block
        live[p + off] = p
        return p + off

    def free(ptr, stream, ctx):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(live.pop(ptr))

    fa, ff = AF(alloc), FF(free)
    lib = L.lib()
    try:
        L.check(lib.lbs_set_allocator(ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(ff, ctypes.c_void_p), None))
        got = run(L, case())
        assert calls["alloc"] > 0 and calls["free"] == calls["alloc"] and not live
        L.check(lib.lbs_set_allocator(ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(ff, ctypes.c_void_p),
                                      ctypes.c_void_p(1)))
        with pytest.raises(L.LbsError):
            L.Simulation(case())
        assert not live
    finally:
        L.check(lib.lbs_set_allocator(None, None, None))
    assert same(got, run(L, case()))


def test_caller_stream_and_graph_chunks(L):
    import torch
    ref = run(L, case())
    st = torch.cuda.Stream()
    assert same(run(L, case(), stream=st), ref)
    for chunk in (0, 2, 64, 128):
        assert same(run(L, case(), graph_chunk=chunk), ref)


def test_launch_count_device_bytes_and_cfl_flag(L):
    c = case()
    with L.Simulation(c, graph_chunk=0, monitor_interval=0) as s:
        n0 = s.launch_count
        s.step(10)
        s.sync()
        # direct launches: one frame-tile kernel per iteration, plus one for the
        # interior tiles when the lattice has any (this one does)
        assert s.launch_count - n0 == 20
        assert s.device_bytes == L.footprint(c)
        assert not s.cfl_warning
    with L.Simulation(case(nu=0.3)) as s:
        assert s.cfl_warning  # nu > 1/4: the first-order wall bound c_d <= c is exceeded


def test_bounded_wait_runs_out_and_the_context_stays_usable(L):
    """A wait on a barrier armed for bytes that never arrive ends by its own
    bound and is reported; the same wait with nothing expected completes; the
    GPU context then runs a lattice as before."""
    ref = run(L, case())
    timed_out, sec = L.selftest_bounded_wait(16, 1 << 14)
    assert timed_out and sec < 30.0
    timed_out, _ = L.selftest_bounded_wait(0, 1 << 14)
    assert not timed_out
    assert same(run(L, case()), ref)


@pytest.mark.parametrize("precision", ["fp32", "fp16s", "fp64"])
def test_switching_variant_and_graph_chunk_mid_run(L, precision):
    """Tile variant and graph chunk changed between steps (graphs are
    recaptured, TMA descriptors rebuilt for the current buffers): the result
    is bitwise that of one uninterrupted run with the defaults."""
    c = case(precision)
    ref = run(L, c, steps=200)
    nvar = len(L.tile_variants(precision))
    with L.Simulation(c) as s:
        for v, chunk in [(nvar - 1, 64), (0, 0), (4, 2), (nvar // 2, 128), (1, 64)]:
            s.set_variant(v % nvar)
            s.set_graph_chunk(chunk)
            s.step(40)
        s.sync()
        assert s.iteration == 200
        got = s.fields()
    assert same(got, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_host_transfers_staged_in_the_idle_buffers(L, precision):
    """set_initial and fields stage host data in the g and u buffers of the
    parity the state is not in (several passes, or one allocated buffer, when
    the outputs do not fit at once): host and device entry points give the
    same bits, any subset of outputs works, and reading fields mid-run leaves
    the continuing run unchanged."""
    import torch
    c = case(precision).replace(edges=(I.PERIODIC,) * 4)
    dev = torch.device("cuda")
    rng = np.random.default_rng(5)
    u0 = 1e-3 * rng.normal(size=(c.ny, c.nx, 2))
    v0 = 1e-3 * rng.normal(size=(c.ny, c.nx, 2))
    with L.Simulation(c) as s:
        s.set_initial(torch.tensor(u0, device=dev), torch.tensor(v0, device=dev))
        s.step(70)
        out = [torch.empty((c.ny, c.nx, w), dtype=torch.float64, device=dev) for w in (2, 2, 4)]
        s.fields_device(*out)
        s.sync()
        ref = [o.cpu().numpy() for o in out]
        s.step(60)
        s.sync()
        ref_end = s.fields()
    with L.Simulation(c) as s:
        s.set_initial(u0, v0)
        s.step(70)
        got = s.fields()
        assert all(np.array_equal(a, b) for a, b in zip(got, ref))
        for want in [(True, False, False), (False, True, False), (False, False, True), (False, True, True)]:
            part = s.fields(*want)
            for w, a, b in zip(want, part, ref):
                assert (a is None) if not w else np.array_equal(a, b)
        s.step(60)
        s.sync()
        assert all(np.array_equal(a, b) for a, b in zip(s.fields(), ref_end))


def test_separate_handles_on_separate_threads(L):
    """Handles are independent: four lattices stepped at once from four host
    threads (each handle on its own streams) give the bits they give when run
    one after another."""
    import threading
    cases = [case(p, nx=96 + 17 * i, ny=64 + 9 * i) for i, p in enumerate(["fp32", "fp16s", "fp64", "fp32"])]
    ref = [run(L, c, steps=150) for c in cases]
    out = [None] * len(cases)
    errors = []

    def work(i):
        try:
            out[i] = run(L, cases[i], steps=150)
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(120)
    assert not errors, errors
    for got, want in zip(out, ref):
        assert same(got, want)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_non_finite_initial_state_is_flagged_and_the_handle_stays_usable(L, precision):
    """A NaN in the initial velocity (injected on the host, not on the GPU)
    is reported as LBS_EUNSTABLE by the monitor at the first iteration it
    runs after, the handle still answers lbs_fields, and a fresh handle of the
    same lattice runs normally."""
    c = case(precision)
    v0 = np.zeros((c.ny, c.nx, 2))
    v0[c.ny // 2, c.nx // 3, 0] = np.nan
    with L.Simulation(c, monitor_interval=1) as s:
        s.set_initial(None, v0)
        with pytest.raises(L.LbsError) as e:
            s.step(20)
            s.sync()
        assert e.value.code == L.EUNSTABLE
        assert 0 <= s.unstable_iteration <= 2
        u, v, P = s.fields()
        assert not np.isfinite(v).all()
    assert same(run(L, c, 40), run(L, c, 40))
