#!/usr/bin/env python
"""Throughput of the fused lattice update (MLUPS) on the roofline workload.

Workload: a 16384 x 16384 periodic neo-Hooke lattice (E = 1, nu = 0.3,
rho0 = 1, tau = 0.55) started from a smooth seeded random velocity field
(correlation length 64 nodes, peak speed 0.2 c_s), FP32 storage and
arithmetic (the displacement as a compensated float pair).  One benchmark
step = one iteration of the method over the whole lattice (one fused kernel
launch pair: interior tiles + frame tiles).

    python bench.py [--gpus N --steps K --warmup W] [--precision fp32|fp64|fp16s]
    python bench.py --impl reference       # the CPU oracle on the host cores

N > 1 (torchrun): every rank steps its own lattice (independent replicas,
no collective on the data path; weak scaling); the time is the maximum over
ranks and the value the aggregate.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic bytes per node update of the fused step: read and write of the
# nine distributions and of the displacement record (the halo comes from L1/L2)
BYTES_PER_NODE = {"fp64": 2 * 9 * 8 + 2 * 16, "fp32": 2 * 9 * 4 + 2 * 16, "fp16s": 2 * 9 * 2 + 2 * 16}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16s": "f16-storage/f32"}
FALLBACK_HBM_GBS = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profile_traffic(precision: str, n: int):
    """DRAM bytes per node update of the step kernels from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        from paper_2502_00920_gb300 import build as B
        if rec.get("source_hash") != B.source_hash():
            return None
        per_node = rec["bytes_per_node"].get(precision)
        return None if per_node is None else per_node * n * n
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            self.out.flush()
            rows = [r.split(",") for r in open(self.out.name).read().strip().splitlines() if r.strip()]
            os.unlink(self.out.name)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_rate(n: int, target_s: float, seed: int = 5):
    """MLUPS of the CPU oracle on a bounded sample of the workload: the same
    recipe (periodic neo-Hooke, seeded random velocity) on an n x n lattice,
    stepped for about target_s seconds on all host cores."""
    from oracle import oracle as O
    from paper_2502_00920_gb300 import inputs as I
    case = I.roofline(n=n, nsteps=0, precision="fp64", seed=seed)
    v0 = I.grf_velocity(case)
    sim = O.OracleSim(case, None, v0)
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter() - t0
    steps = max(1, int(target_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS", "cores": O.OracleSim.threads(), "kind": "oracle",
            "sample": f"{n}x{n} periodic neo-Hooke lattice, same random-velocity recipe, {steps} iterations "
                      f"({dt:.1f} s) after 1 untimed"}, steps, dt


L2_BYTES = 129 * 1024 * 1024  # GB300 L2


def arm_config(n: int, precision: str, world: int) -> dict:
    """The workload both arms report on: the roofline lattice."""
    bpn = BYTES_PER_NODE[precision]
    state = bpn * n * n  # both buffers of g and u
    l2 = (f"state {state / 1e9:.1f} GB per lattice, larger than L2 (no flush needed)" if state > L2_BYTES else
          f"state {state / 1e6:.1f} MB per lattice, fits in L2 (not flushed: a small-lattice run, not a bench value)")
    return {"workload": f"roofline {n}x{n} periodic neo-Hooke, random initial velocity",
            "nx": n, "ny": n, "model": "nh", "E": 1.0, "nu": 0.3, "tau": 0.55,
            "precision": precision, "parallelism": f"replicas x{world}", "l2": l2}


def run_reference(args, rank: int, world: int):
    """The oracle on the host cores, on this arm's workload: each of the K
    timed steps (after W warm-up steps) is a bounded sample, m iterations of
    the same recipe on a ref_n x ref_n lattice, with m chosen so that the K
    steps take about ref_seconds."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2502_00920_gb300 import inputs as I
    n, K, W = args.ref_n, args.steps, args.warmup
    case = I.roofline(n=n, nsteps=0, precision="fp64", seed=5)
    sim = O.OracleSim(case, None, I.grf_velocity(case))
    t0 = time.perf_counter()
    sim.step(1)
    t1 = max(time.perf_counter() - t0, 1e-6)
    m = max(1, int(args.ref_seconds / (K * t1)))
    mw = max(1, min(m, int(args.ref_seconds / (W * t1))))  # warm-up bounded by ref_seconds too
    for _ in range(W):
        sim.step(mw)
    t0 = time.perf_counter()
    for _ in range(K):
        sim.step(m)
    dt = time.perf_counter() - t0
    value = n * n * m * K / dt / 1e6
    cb = {"value": value, "unit": "MLUPS", "cores": O.OracleSim.threads(), "kind": "oracle",
          "sample": f"{n}x{n} lattice of the same recipe; each step {m} iterations ({K} steps, {dt:.1f} s) after "
                    f"{W} warm-up steps of {mw}"}
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * dt / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args.n, args.precision, world),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_alu_roofline(mlups: float):
    """FP64 is bound by the FP64 pipe, not HBM: FLOP per node from the
    committed ncu record (if taken on the current kernel source; DADD + DMUL +
    2 DFMA as ncu counts them) against the FP64 FMA rate of the GPU (2 per
    clock per SM), and the pipe operations per node against the pipe's slots;
    else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "step_fp64_alu.json")) as f:
            rec = json.load(f)
        from paper_2502_00920_gb300 import build as B
        if rec.get("source_hash") != B.source_hash():
            return None
        achieved = rec["flops_per_node"] * mlups * 1e6 / 1e12
        # every DADD, DMUL and DFMA takes one slot of the pipe, which issues
        # half the FMA-counted FLOP rate: the slots, not the FLOP, bound it
        slots = rec["fp64_pipe_ops_per_node"] * mlups * 1e6 / (rec["peak_tflops"] * 1e12 / 2)
        return {"bound": "alu", "achieved": achieved, "peak": rec["peak_tflops"], "unit": "TFLOP/s",
                "frac": achieved / rec["peak_tflops"], "flops_per_node": rec["flops_per_node"],
                "fp64_pipe_ops_per_node": rec["fp64_pipe_ops_per_node"], "pipe_slot_frac": slots,
                "fp64_pipe_active_ncu": rec["fp64_pipe_active"], "peak_source": rec["peak_source"]}
    except Exception:
        return None


def time_precision(L, I, torch, precision, n, steps, warmup, stream, v0dev, uref=None):
    """Time one precision on the roofline lattice; with uref (the FP64 u after
    warmup + steps iterations) also state its error."""
    case = I.roofline(n=n, nsteps=steps, precision=precision)
    sim = L.Simulation(case, stream=stream)
    sim.set_initial(None, v0dev)
    sim.step(warmup)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    u = torch.empty((n, n, 2), dtype=torch.float64, device=v0dev.device)
    sim.fields_device(u, None, None)
    sim.sync()
    sim.close()
    bpn = BYTES_PER_NODE[precision]
    out = {"mlups": n * n / (ms * 1e-3) / 1e6, "ms_per_step": ms, "gbs": bpn * n * n / (ms * 1e-3) / 1e9,
           "bytes_per_node": bpn, "iterations": warmup + steps}
    if uref is not None:
        out["u_rel_err_vs_fp64"] = float((u - uref).abs().max() / uref.abs().max())
    if precision == "fp64":
        out["roofline"] = fp64_alu_roofline(out["mlups"])
    return out, u


def serving(L, I, n_requests: int, steps_scale: float, seed: int = 4, load: float = 1.5):
    """Batched serving vs one-at-a-time FP64 on a seeded trace of mixed
    requests (sizes log-uniform 32..1024 x 32..512, SVK or neo-Hooke, nu in
    [0, 0.45], tension / shear / tip-pulse loads, iterations log-uniform
    1k..50k scaled by steps_scale).

    The one-at-a-time FP64 baseline runs every request alone (create, step in
    chunks of 1000 iterations, fetch fields, destroy) and records its service
    time; its FIFO queue under the arrival times is then exact: done_i =
    max(arrival_i, done_{i-1}) + service_i.  Arrivals are Poisson at `load`
    times that baseline's capacity.  The FP32 server then receives the same
    arrivals in real time (latency p50/p99), and, on a fresh server, the whole
    trace at once (capacity).  Both arms stop a request that went non-finite
    at their next 1000-iteration check and count it as failed (also when its
    final u is not finite); aggregate MLUPS counts the node updates actually
    executed.  Every request finite in both arms states its FP32 error on u
    against its FP64 result; each one above 1e-5 also states how much its FP64
    result moves under perturbations of one double rounding unit."""
    import threading
    trace = I.serving_trace(n_requests, seed=seed, rate=1.0)
    cases = [c.replace(nsteps=max(100, int(round(c.nsteps * steps_scale)))) for _, c in trace]
    work = [c.nx * c.ny * c.nsteps for c in cases]
    # one at a time, FP64
    service, u64, done64 = [], [], 0
    for c in cases:
        t0 = time.perf_counter()
        u = None
        with L.Simulation(c.replace(precision="fp64")) as s:
            try:
                while s.iteration < c.nsteps:
                    s.step(min(1000, c.nsteps - s.iteration))
                    s.sync()  # the chunk's monitor: stops a request that went non-finite
                u, _, _ = s.fields(True, True, True)
            except L.LbsError:
                pass
            done64 += c.nx * c.ny * s.iteration
        service.append(time.perf_counter() - t0)
        u64.append(u if u is not None and np.isfinite(u).all() else None)
    capacity = len(cases) / sum(service)
    rate = load * capacity
    gaps = [a for a, _ in trace]
    arrivals = [t / rate for t in gaps]  # the trace was drawn at rate 1
    done, t = [], 0.0
    for a, sv in zip(arrivals, service):
        t = max(a, t) + sv
        done.append(t)
    seq_ttr = [d - a for d, a in zip(done, arrivals)]
    q = lambda xs, p: sorted(xs)[min(len(xs) - 1, int(round(p * (len(xs) - 1))))] if xs else None

    def collect(srv, tickets):
        infos = [srv.poll(tk) for tk in tickets]
        us = []
        for tk in tickets:
            u, _, _, rc = srv.result(tk)
            us.append(u if rc == L.OK and np.isfinite(u).all() else None)
        return infos, us

    # batched FP32, Poisson arrivals in real time
    with L.Server(precision="fp32", chunk=64) as srv:
        tickets = [None] * len(cases)
        t_start = time.perf_counter()

        def submitter():
            for i, (a, c) in enumerate(zip(arrivals, cases)):
                delay = a - (time.perf_counter() - t_start)
                if delay > 0:
                    time.sleep(delay)
                tickets[i] = srv.submit(c.replace(precision="fp32"))

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        srv.drain(-1)
        stats = srv.stats()
        infos, u32 = collect(srv, tickets)
    ttr = [i["t_done"] - i["t_submit"] for i in infos]
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    # batched FP32, the whole trace at once
    with L.Server(precision="fp32", chunk=64) as srv:
        t0 = time.perf_counter()
        tickets = [srv.submit(c.replace(precision="fp32")) for c in cases]
        srv.drain(-1)
        makespan = time.perf_counter() - t0
        sat_stats = srv.stats()
        sat_infos, sat_u = collect(srv, tickets)
    ok = [u is not None for u in u64]
    errs = [float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
            for a, b in zip(u32, u64) if a is not None and b is not None]
    above = [dict(request=c.name, nx=c.nx, ny=c.ny, model=c.model, nu=round(c.nu, 4), iterations=c.nsteps,
                  err=float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)))
             for c, a, b in zip(cases, u32, u64) if a is not None and b is not None
             and np.abs(a - b).max() > 1e-5 * max(np.abs(b).max(), 1e-300)]
    # Conditioning of each request above the bar: its FP64 result again,
    # once with Young's modulus moved by one double rounding unit and once
    # from an initial displacement of seeded noise at one double rounding unit
    # of its final |u| (this one reaches every mode, the fast-growing ones
    # included).  The larger relative change of u is the problem's own
    # amplification of a perturbation of that size; FP32 rounds 2^29 times
    # more coarsely, so an FP32 error below 2^29 times that change is what the
    # problem itself allows for FP32 arithmetic.
    by_name = {c.name: (i, c, b) for i, (c, b) in enumerate(zip(cases, u64))}

    def fp64_change(c, b, u0=None, **kw):
        with L.Simulation(c.replace(precision="fp64", **kw)) as s:
            try:
                if u0 is not None:
                    s.set_initial(u0, None)
                s.step(c.nsteps)
                s.sync()
                u, _, _ = s.fields(True, False, False)
            except L.LbsError:
                return None
        return float(np.abs(u - b).max() / max(np.abs(b).max(), 1e-300)) if np.isfinite(u).all() else None

    for r in above:
        i, c, b = by_name[r["request"]]
        noise = np.random.default_rng(1000 + i).standard_normal((c.ny, c.nx, 2)) * (2.0 ** -53 * np.abs(b).max())
        r["fp64_change_one_ulp_E"] = fp64_change(c, b, E=float(np.nextafter(c.E, 2.0 * c.E)))
        r["fp64_change_one_ulp_noise_u0"] = fp64_change(c, b, u0=noise)
        changes = [x for x in (r["fp64_change_one_ulp_E"], r["fp64_change_one_ulp_noise_u0"]) if x is not None]
        r["within_conditioning"] = bool(changes) and r["err"] <= 2.0 ** 29 * max(changes)
    return {"requests": len(cases), "steps_scale": steps_scale, "node_updates_requested": sum(work),
            "offered_load_x_fp64_capacity": load, "arrival_rate_per_s": rate,
            "sequential_fp64": {"aggregate_mlups": done64 / sum(service) / 1e6, "node_updates": done64,
                                "p50_s": q(seq_ttr, 0.5), "p99_s": q(seq_ttr, 0.99),
                                "p50_s_completed": q([x for x, o in zip(seq_ttr, ok) if o], 0.5),
                                "p99_s_completed": q([x for x, o in zip(seq_ttr, ok) if o], 0.99),
                                "failed": sum(u is None for u in u64), "service_s": sum(service)},
            "batched_fp32_poisson": {"aggregate_mlups": stats["node_updates"] / span / 1e6,
                                     "node_updates": stats["node_updates"], "p50_s": q(ttr, 0.5),
                                     "p99_s": q(ttr, 0.99),
                                     "p50_s_completed": q([x for x, u in zip(ttr, u32) if u is not None], 0.5),
                                     "p99_s_completed": q([x for x, u in zip(ttr, u32) if u is not None], 0.99),
                                     "failed": sum(u is None for u in u32),
                                     "launches": stats["launches"], "busy_s": stats["busy_seconds"]},
            "batched_fp32_saturated": {"aggregate_mlups": sat_stats["node_updates"] / makespan / 1e6,
                                       "node_updates": sat_stats["node_updates"], "makespan_s": makespan,
                                       "failed": sum(u is None for u in sat_u),
                                       "batch_tile": [sat_stats["batch_tx"], sat_stats["batch_ty"]],
                                       "batch_tunings": sat_stats["batch_tunings"],
                                       "equal_to_poisson_run": all(
                                           (a is None and b is None) or (a is not None and b is not None
                                                                          and np.array_equal(a, b))
                                           for a, b in zip(u32, sat_u))},
            "failed_fp32_only": sum(a is None and b is not None for a, b in zip(u32, u64)),
            "failed_fp64_only": sum(a is not None and b is None for a, b in zip(u32, u64)),
            "u_err_fp32_vs_fp64": {"compared": len(errs), "max": max(errs) if errs else None,
                                   "median": float(np.median(errs)) if errs else None,
                                   "above_1e-5": sum(e > 1e-5 for e in errs),
                                   "above_1e-5_beyond_conditioning": sum(not r["within_conditioning"] for r in above),
                                   "above_1e-5_requests": above}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16s"])
    ap.add_argument("--variant", type=int, default=None, help="tile variant of the timed lattice (default: the "
                    "precision's default variant)")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--ref-n", type=int, default=1024)
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=128)
    ap.add_argument("--serving-steps-scale", type=float, default=0.25)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    from paper_2502_00920_gb300 import replicas as RP
    rank, world, local = RP.ranks()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_2502_00920_gb300 import build as B
    B.build()
    from paper_2502_00920_gb300 import inputs as I
    from paper_2502_00920_gb300 import lbs as L

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    RP.init(world)

    def barrier():
        RP.barrier(world)

    n, K, W = args.n, args.steps, args.warmup
    case = I.roofline(n=n, nsteps=args.e2e_steps, precision=args.precision, seed=5 + rank)
    stream = torch.cuda.Stream(device=dev)
    v0 = I.grf_velocity(case, device=dev)
    sim = L.Simulation(case, stream=stream, variant=args.variant)
    sim.set_initial(None, v0)
    sim.step(W)
    sim.sync()
    launches0 = sim.launch_count

    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = sim.launch_count - launches0
    sim.sync()  # raises if a monitor saw a non-finite value
    variant = sim.variant
    ms_max = RP.max_over_ranks(ms, world)
    cells = n * n
    value = RP.aggregate_rate(cells * K, ms_max * 1e-3, world) / 1e6

    # roofline of the step kernels: algorithmic bytes per launch pair / its
    # average duration in the timed region (events on the launching stream)
    peak, peak_kind = peaks()
    bpn = BYTES_PER_NODE[args.precision]
    if L.tile_variant_name(args.precision, variant) == "step_fused2_tma_kernel":
        bpn = bpn / 2  # two iterations per pass over the state (periodic lattice)
    achieved = bpn * cells / (ms / K * 1e-3) / 1e9
    traffic = profile_traffic(args.precision, n)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": f"{L.tile_variant_name(args.precision, variant)} + step_edge_kernel (one iteration, "
                          f"tile variant {variant})",
                "bytes_per_node": bpn, "peak_source": f"{peak_kind} hbm_gbs"}
    clocks = clk.summary()
    sim.close()

    # end to end through the C ABI: pinned host initial velocity -> device,
    # e2e_steps iterations, device -> pinned host u and v
    E = args.e2e_steps
    e2e = None
    if args.no_e2e:
        E = 0
    if E > 0:
        vh = torch.empty((n, n, 2), dtype=torch.float64, pin_memory=True)
        vh.copy_(v0)
        del v0
        torch.cuda.empty_cache()
        uo = torch.empty((n, n, 2), dtype=torch.float64, pin_memory=True)
        vo = torch.empty((n, n, 2), dtype=torch.float64, pin_memory=True)
        sim = L.Simulation(case, stream=stream, variant=args.variant)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_initial(None, vh.numpy())
        sim.step(E)
        sim.fields(uo.numpy(), vo.numpy(), False)
        te = time.perf_counter() - t0
        sim.close()
        te_max = RP.max_over_ranks(te, world)
        e2e = {"value": RP.aggregate_rate(cells * E, te_max, world) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": vh.numel() * 8 / E, "d2h_bytes_per_step": (uo.numel() + vo.numel()) * 8 / E,
               "job": f"set_initial(host v0) + {E} iterations + fields(host u, v)", "seconds": te_max}
        del vh, uo, vo
    else:
        del v0

    variants = None
    if not args.no_variants:
        variants = {}
        v0 = I.grf_velocity(case, device=dev)
        ks = max(10, K // 10)
        variants["fp64"], uref = time_precision(L, I, torch, "fp64", n, ks, W, stream, v0)
        for p in ("fp32", "fp16s"):
            variants[p], _ = time_precision(L, I, torch, p, n, ks, W, stream, v0, uref)
        del v0, uref
        torch.cuda.empty_cache()

    serve = None
    if not args.no_serving and rank == 0:
        serve = serving(L, I, args.serving_requests, args.serving_steps_scale)

    barrier()
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(args.ref_n, args.ref_seconds)[0]
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": arm_config(n, args.precision, world),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "precisions": variants, "serving": serve}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
