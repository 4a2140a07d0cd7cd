"""Continuous-batching server on the GPU: each result equals the same lattice
run alone (and the oracle within the precision's bar), admission respects
the HBM budget, requests arriving while others run are admitted as memory
frees up, and failures are reported per ticket."""
import threading
import time

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


def mix(precision="fp32"):
    trac = I.Edge("neumann", "linear_ramp", (0.01, 0.0), 0, 80)
    return [
        I.tension(32, 32, 150, ramp=100, model="nh", precision=precision),
        I.shear(64, 220, model="svk", nu=0.2, gamma=0.05, ramp=400, precision=precision),
        I.cantilever(200, 24, 90, width=60, amp=0.01, nu=0.25, precision=precision),
        I.Case("m", 130, 70, 300, model="svk", nu=0.2, edges=(I.CLAMPED, trac, I.FREE, I.FREE), precision=precision),
        I.Case("p", 96, 40, 64, model="nh", nu=0.1, edges=(I.FREE, trac, I.CLAMPED, I.FREE), precision=precision),
        I.tension(45, 33, 77, ramp=40, model="svk", nu=0.0, precision=precision),
    ]


def alone(L, case):
    with L.Simulation(case) as s:
        s.step(case.nsteps)
        s.sync()
        return s.fields()


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16s"])
def test_mixed_batch_equals_alone(L, precision):
    cases = mix(precision)
    with L.Server(precision=precision, chunk=32) as srv:
        tickets = [srv.submit(c) for c in cases]
        srv.drain(120)
        results = [srv.result(t) for t in tickets]
    for c, (u, v, P, rc) in zip(cases, results):
        assert rc == L.OK
        ua, va, Pa = alone(L, c)
        assert np.array_equal(u, ua) and np.array_equal(v, va) and np.array_equal(P, Pa), c.name


def test_batch_matches_oracle(L, oracle_mod):
    cases = mix("fp64")[:3]
    with L.Server(precision="fp64", chunk=16) as srv:
        tickets = [srv.submit(c) for c in cases]
        srv.drain(120)
        results = [srv.result(t) for t in tickets]
    for c, (u, v, P, rc) in zip(cases, results):
        o = oracle_mod.OracleSim(c)
        o.step(c.nsteps)
        ur = o.fields()[0]
        assert np.abs(u - ur).max() <= 1e-12 * np.abs(ur).max()


def test_admission_respects_budget(L):
    case = I.tension(256, 128, 400, ramp=100, model="nh")
    fp = L.footprint(case.replace(precision="fp32"))
    budget = int(2.5 * fp)
    peak = 0
    with L.Server(precision="fp32", hbm_budget=budget, chunk=16) as srv:
        tickets = [srv.submit(case) for _ in range(5)]
        while srv.stats()["completed"] + srv.stats()["failed"] < 5:
            st = srv.stats()
            peak = max(peak, st["bytes_in_use"])
            assert st["resident"] <= 2
            time.sleep(0.002)
        infos = [srv.poll(t) for t in tickets]
        for t in tickets:
            srv.result(t)
    assert 0 < peak <= budget
    assert all(i["state"] == "done" for i in infos)
    # at most two at a time: the third is admitted only after one finished
    admits = sorted(i["t_admit"] for i in infos)
    dones = sorted(i["t_done"] for i in infos)
    assert admits[2] >= dones[0] - 1e-6


def test_continuous_admission(L):
    """Requests arriving while others are on the GPU join the running batch,
    their work overlaps on the device with the lattice already resident, and
    every result, the late arrivals' included, equals the same lattice run
    alone, bitwise."""
    # stable over its whole history in the oracle (finite to beyond 7000
    # iterations; the same load at nu = 0.3 and peak 0.2 goes non-finite
    # between 1000 and 2000 iterations)
    long = I.tension(512, 256, 6500, ramp=500, model="nh", nu=0.2, peak=0.05, precision="fp32")
    trac = I.Edge("neumann", "linear_ramp", (0.01, 0.0), 0, 80)
    short = [I.tension(64, 48, 200, ramp=50, model="svk", nu=0.1, precision="fp32"),
             I.shear(96, 260, model="nh", nu=0.2, gamma=0.05, ramp=300, precision="fp32"),
             I.Case("late_m", 130, 70, 300, model="svk", nu=0.2, edges=(I.CLAMPED, trac, I.FREE, I.FREE),
                    precision="fp32"),
             I.cantilever(200, 24, 150, width=60, amp=0.01, nu=0.25, precision="fp32")]
    with L.Server(precision="fp32", chunk=32) as srv:
        t_long = srv.submit(long)
        t_wait = time.time()
        while srv.poll(t_long)["iterations"] == 0 and time.time() - t_wait < 30:
            time.sleep(0.001)  # the long one is on the GPU
        ts = []
        for c in short:
            ts.append(srv.submit(c))
            time.sleep(0.002)
        srv.drain(120)
        il = srv.poll(t_long)
        infos = [srv.poll(t) for t in ts]
        results = [srv.result(t) for t in [t_long] + ts]
    # the short ones were admitted and finished while the long one was running
    assert all(il["t_admit"] < i["t_submit"] for i in infos)
    assert all(i["t_admit"] < il["t_done"] for i in infos)
    assert all(i["t_done"] < il["t_done"] for i in infos)
    for case, (u, v, P, rc) in zip([long] + short, results):
        assert rc == L.OK, case.name
        ua, va, Pa = alone(L, case)
        assert np.array_equal(u, ua) and np.array_equal(v, va) and np.array_equal(P, Pa), case.name


def test_cancel_queued_and_running_requests(L):
    """lbs_cancel: a queued request leaves the queue at once, a running one
    stops at the next scheduling point with its fields as they stood and its
    memory released; both end failed with ECANCELED, and the request beside
    them still equals its lattice run alone."""
    long = I.tension(512, 256, 6500, ramp=500, model="nh", nu=0.2, peak=0.05, precision="fp32")
    other = I.tension(64, 48, 200, ramp=50, model="svk", nu=0.1, precision="fp32")
    fp = L.footprint(long)
    # a budget that holds the long lattice and the small one, not a second long one
    with L.Server(precision="fp32", chunk=32, hbm_budget=int(fp * 1.5)) as srv:
        t_run = srv.submit(long)
        t_wait = time.time()
        while srv.poll(t_run)["iterations"] == 0 and time.time() - t_wait < 30:
            time.sleep(0.001)
        t_queued = srv.submit(long)  # does not fit beside the first: waits in the queue
        t_other = srv.submit(other)
        assert srv.poll(t_queued)["state"] == "queued"
        srv.cancel(t_queued)
        assert srv.poll(t_queued)["state"] == "failed"
        srv.wait(t_other, 60)
        srv.cancel(t_run)
        srv.wait(t_run, 60)
        info = srv.poll(t_run)
        stats = srv.stats()
        u, v, P, rc = srv.result(t_run)
        uq, _, _, rcq = srv.result(t_queued)
        uo, vo, Po, rco = srv.result(t_other)
        with pytest.raises(L.LbsError) as e:
            srv.cancel(t_run)  # collected: unknown now
        assert e.value.code == L.ENOTFOUND
    assert rc == L.ECANCELED and rcq == L.ECANCELED and rco == L.OK
    assert 0 < info["iterations"] < long.nsteps and info["iterations"] % 32 == 0
    assert stats["resident"] == 0 and stats["queued"] == 0
    assert np.isfinite(u).all()
    ua = alone(L, long.replace(nsteps=info["iterations"]))[0]
    assert np.array_equal(u, ua)  # the fields where it stopped
    ra = alone(L, other)
    assert np.array_equal(uo, ra[0]) and np.array_equal(vo, ra[1]) and np.array_equal(Po, ra[2])


def test_failures_reported_per_ticket(L):
    """A request that goes non-finite (linear material, nu = 0.45, loaded:
    beyond the scheme's stability) fails alone with LBS_EUNSTABLE; the
    request beside it completes."""
    bad = I.tension(32, 32, 1500, ramp=50, model="le", nu=0.45)
    good = I.tension(32, 32, 100, ramp=50, model="nh")
    with L.Server(precision="fp64", chunk=32) as srv:
        tb = srv.submit(bad)
        tg = srv.submit(good)
        srv.drain(120)
        assert srv.poll(tg)["state"] == "done"
        info = srv.poll(tb)
        assert info["state"] == "failed" and info["error"] == L.EUNSTABLE
        assert srv.result(tg)[3] == L.OK
        assert srv.result(tb)[3] == L.EUNSTABLE
    with pytest.raises(L.LbsError) as e:
        with L.Server(precision="fp32", hbm_budget=1 << 20) as srv:
            srv.submit(I.tension(1024, 1024, 10))
    assert e.value.code == L.ENOMEM


def test_preemption_lets_a_short_request_pass_a_long_one(L):
    """With a budget that holds one lattice, a short request that arrives
    while a long one runs waits behind it (FIFO) unless preemption is on; with
    it, the long lattice is swapped out to host memory, the short one runs,
    and the long one resumes.  Both results equal the same lattices run alone,
    bitwise.  Clamped edges under a body force keep both bounded."""
    clamped = (I.CLAMPED,) * 4
    long = I.Case("long", 1024, 1024, 30000, model="nh", nu=0.3, body=(0.0, -0.01), edges=clamped,
                  precision="fp32")
    short = I.Case("short", 1024, 1024, 300, model="svk", nu=0.2, body=(0.01, 0.0), edges=clamped,
                   precision="fp32")
    budget = int(1.5 * L.footprint(long))

    def run(preempt):
        with L.Server(precision="fp32", hbm_budget=budget, chunk=32, preempt_after_s=preempt) as srv:
            tl = srv.submit(long)
            time.sleep(0.2)
            ts = srv.submit(short)
            srv.drain(600)
            il, is_, st = srv.poll(tl), srv.poll(ts), srv.stats()
            rl, rs = srv.result(tl), srv.result(ts)
        assert rl[3] == L.OK and rs[3] == L.OK
        assert il["t_admit"] < is_["t_submit"] < il["t_done"]  # the short one arrived while the long one ran
        return il, is_, st, rl[:3], rs[:3]

    il, is_, st, rl, rs = run(0.05)
    assert is_["t_done"] < il["t_done"]
    assert il["swaps"] >= 1 and st["preemptions"] >= 1 and is_["swaps"] == 0
    for got, case in ((rl, long), (rs, short)):
        for x, y in zip(got, alone(L, case)):
            assert np.array_equal(x, y), case.name
    il, is_, st, _, _ = run(0.0)
    assert is_["t_done"] > il["t_done"] and st["preemptions"] == 0


def test_preemption_setting_is_validated(L):
    with pytest.raises(L.LbsError) as e:
        L.Server(precision="fp32", preempt_after_s=-1.0)
    assert e.value.code == L.EINVAL


def test_zero_iteration_requests_and_steps(L):
    """Empty work: a request of zero iterations, alone or beside others,
    returns its initial state, and lbs_step(h, 0) changes nothing."""
    c0 = I.tension(48, 40, 0, ramp=50, model="nh", nu=0.2, precision="fp32")
    other = I.tension(64, 48, 120, ramp=50, model="svk", nu=0.1, precision="fp32")
    with L.Simulation(c0) as s:
        ref = s.fields()
        s.step(0)
        s.sync()
        assert s.iteration == 0
        assert all(np.array_equal(a, b) for a, b in zip(s.fields(), ref))
    for batch in ([c0], [c0, other]):
        with L.Server(precision="fp32", chunk=32) as srv:
            tickets = [srv.submit(c) for c in batch]
            srv.drain(60)
            u, v, P, rc = srv.result(tickets[0])
            assert rc == L.OK and all(srv.result(t)[3] == L.OK for t in tickets[1:])
        assert np.array_equal(u, ref[0]) and np.array_equal(v, ref[1]) and np.array_equal(P, ref[2])


def test_batch_tile_shapes_give_the_same_results_and_are_tuned(L):
    """The server's four batch tile shapes compute every node with the same
    operations: fixing any of them, or letting the server time them and
    switch mid-run, gives bitwise the same results (equal to the lattices run
    alone); an unknown shape is refused."""
    cases = mix("fp32")
    ref = [alone(L, c) for c in cases]
    for shape in (0, 1, 2, 3, None):
        with L.Server(precision="fp32", chunk=16, batch_shape=shape) as srv:
            tickets = [srv.submit(c) for c in cases]
            srv.drain(120)
            st = srv.stats()
            results = [srv.result(t) for t in tickets]
        if shape is None:
            assert st["batch_tunings"] >= 1
        else:
            assert st["batch_shape"] == shape
        for c, (u, v, P, rc), (ua, va, Pa) in zip(cases, results, ref):
            assert rc == L.OK
            assert np.array_equal(u, ua) and np.array_equal(v, va) and np.array_equal(P, Pa), (c.name, shape)
    with pytest.raises(L.LbsError) as e:
        L.Server(precision="fp32", batch_shape=7)
    assert e.value.code == L.EINVAL
