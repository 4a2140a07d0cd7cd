"""Every benchmark configuration in every precision, against the oracle
(test infrastructure: GPU and CPU oracle).

For each workload of the benchmark table (32^2 tension, 256^2 shear sweep,
4096 x 256 cantilever, the paper's own examples and refinement ladder, the
serving trace, the 16384^2 roofline lattice) it prints one JSON line per
result: MLUPS of the GPU path and of the oracle, the error on u (and P)
against the oracle where the oracle can run the whole history, else against
the GPU's FP64 (itself checked against the oracle on a prefix), the first
non-finite iteration of both codes where a history goes non-finite, and for
the refinement ladder the paper's grid error norms evaluated on the GPU.

    python tests/suite_all_workloads.py [--parts tension,shear,...]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from bench import oracle_rate, serving, time_precision  # noqa: E402


def oracle_config_rate(O, case, steps: int) -> dict:
    """The oracle timed on one workload configuration (all host cores):
    `steps` iterations from the configuration's initial state."""
    sim = O.OracleSim(case.replace(precision="fp64"))
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    return {"oracle_mlups": case.nx * case.ny * steps / dt / 1e6, "oracle_cores": O.OracleSim.threads(),
            "oracle_sample": f"{steps} iterations from the initial state ({dt:.1f} s)"}


def suite(args):
    """Every benchmark configuration in every precision: MLUPS, and the error
    on u (and P) against the oracle where it can run the whole history, else
    against the GPU's own FP64 (itself checked against the oracle on a prefix
    and on windows).  Prints one JSON line per result."""
    import torch
    from oracle import oracle as O
    from paper_2502_00920_gb300 import inputs as I
    from paper_2502_00920_gb300 import lbs as L

    dev = torch.device("cuda")
    rel = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    def emit(**kw):
        print(json.dumps(kw), flush=True)

    def gpu_run(case, steps, monitor=0, probe=None, every=100):
        sim = L.Simulation(case, monitor_interval=monitor)
        hist = []
        t0 = time.perf_counter()
        k, unstable = 0, None
        try:
            while k < steps:
                n = min(every if probe is not None else steps, steps - k)
                sim.step(n)
                k += n
                if probe is not None:
                    hist.append(sim.probe([probe])[0].copy())
            sim.sync()
        except L.LbsError as e:
            unstable = sim.unstable_iteration if e.code == L.EUNSTABLE else str(e)
        dt = time.perf_counter() - t0
        out = sim.fields()
        sim.close()
        return out, dt, unstable, np.array(hist)

    def first_nonfinite_gpu(case, steps):
        """First iteration whose state holds a non-finite value (GPU FP64, a
        monitor after every iteration), or None."""
        sim = L.Simulation(case.replace(precision="fp64"), monitor_interval=1, graph_chunk=0)
        try:
            sim.step(steps)
            sim.sync()
        except L.LbsError:
            pass
        k = sim.unstable_iteration
        sim.close()
        return None if k < 0 else k

    def first_nonfinite_oracle(case, steps, coarse=50):
        """(first iteration whose u, v or P is non-finite or None, fields after
        `steps` iterations if they stayed finite)."""
        finite = lambda f: all(np.isfinite(a).all() for a in f)
        o = O.OracleSim(case)
        k = 0
        while k < steps:
            n = min(coarse, steps - k)
            o.step(n)
            k += n
            if not finite(o.fields()):
                o = O.OracleSim(case)
                o.step(k - n)
                for kk in range(k - n + 1, k + 1):
                    o.step(1)
                    if not finite(o.fields()):
                        return kk, None
        return None, o.fields()

    want = lambda part: args.suite_parts == "all" or part in args.suite_parts.split(",")
    # tension 32x32, neo-Hooke, 2000 iterations
    if want("tension"):
        suite_tension(args, L, I, O, emit, gpu_run, rel, first_nonfinite_gpu, first_nonfinite_oracle)
    if want("shear"):
        suite_shear(args, L, I, O, emit, gpu_run, rel, first_nonfinite_gpu, first_nonfinite_oracle)
    if want("cantilever"):
        suite_cantilever(args, L, I, O, emit, gpu_run, rel)
    if want("paper"):
        suite_paper(args, L, I, O, emit, gpu_run, rel)
    if want("serving"):
        emit(config="serving", **serving(L, I, args.serving_requests_suite, args.suite_serving_steps_scale))
    if want("roofline"):
        suite_roofline(args, L, I, torch, dev, emit)


def suite_tension(args, L, I, O, emit, gpu_run, rel, first_nonfinite_gpu, first_nonfinite_oracle):
    case = I.tension()
    emit(config="tension_32x32_nh", first_nonfinite_oracle=first_nonfinite_oracle(case, 2000)[0],
         first_nonfinite_gpu_fp64=first_nonfinite_gpu(case, 2000), **oracle_config_rate(O, case, 1000))
    ora = O.OracleSim(case)
    ora_hist, k_nan = {}, None
    for k in range(0, 2000, 50):
        ora.step(50)
        if k + 50 in (1000, 2000):
            ora_hist[k + 50] = ora.fields()
        if k_nan is None and not np.isfinite(ora.fields()[0]).all():
            k_nan = k + 50
    for prec in ("fp64", "fp32", "fp16s"):
        for steps in (1000, 2000):
            (u, v, P), dt, unstable, _ = gpu_run(case.replace(precision=prec), steps, monitor=50)
            ur, vr, Pr = ora_hist[steps]
            fin = bool(np.isfinite(ur).all())
            emit(config="tension_32x32_nh", precision=prec, iterations=steps, mlups=32 * 32 * steps / dt / 1e6,
                 unstable_gpu=unstable, unstable_oracle=k_nan,
                 u_err=rel(u, ur) if fin and np.isfinite(u).all() else None,
                 v_err=rel(v, vr) if fin and np.isfinite(v).all() else None,
                 P_err=rel(P, Pr) if fin and np.isfinite(P).all() else None,
                 P11_interior=float(P[8:24, 8:24, 0].mean()) if np.isfinite(P).all() else None)


def suite_shear(args, L, I, O, emit, gpu_run, rel, first_nonfinite_gpu, first_nonfinite_oracle):
    # simple shear 256^2, SVK, six Poisson ratios, 20k iterations
    nsh = args.suite_shear_steps
    for nu in (0.0, 0.1, 0.2, 0.3, 0.4, 0.45):
        case = I.shear(256, nsh, model="svk", nu=nu)
        k_o, fo = first_nonfinite_oracle(case, nsh)
        extra = oracle_config_rate(O, case, 500) if nu == 0.2 else {}
        emit(config="shear_256_svk", nu=nu, first_nonfinite_oracle=k_o,
             first_nonfinite_gpu_fp64=first_nonfinite_gpu(case, nsh), **extra)
        for prec in ("fp64", "fp32", "fp16s"):
            (u, v, P), dt, unstable, _ = gpu_run(case.replace(precision=prec), nsh, monitor=1000)
            fin = fo is not None and np.isfinite(u).all()
            emit(config="shear_256_svk", nu=nu, precision=prec, iterations=nsh, mlups=256 * 256 * nsh / dt / 1e6,
                 unstable_gpu=unstable, oracle_finite=fo is not None,
                 u_err=rel(u, fo[0]) if fin else None, P_err=rel(P, fo[2]) if fin else None)


def suite_cantilever(args, L, I, O, emit, gpu_run, rel):
    # cantilever 4096x256, 100k iterations, tip history every 100 iterations
    nc = args.suite_cantilever_steps
    case = I.cantilever(4096, 256, nc)
    tip = (256 // 2) * 4096 + 4095
    ref = {}
    for prec in ("fp64", "fp32", "fp16s"):
        (u, v, P), dt, unstable, hist = gpu_run(case.replace(precision=prec), nc, monitor=1000, probe=tip,
                                                every=100)
        ref[prec] = (u, hist)
        # the tip history up to its first non-finite sample
        fin = np.isfinite(hist).all(axis=-1) if len(hist) else np.zeros(0, bool)
        nfin = int(np.argmin(fin)) if len(fin) and not fin.all() else len(fin)
        row = dict(config="cantilever_4096x256", precision=prec, iterations=nc, mlups=4096 * 256 * 100 * len(hist) / dt / 1e6,
                   unstable_gpu=unstable, finite_iterations=100 * nfin,
                   tip_max=float(np.abs(hist[:nfin]).max()) if nfin else None)
        if prec != "fp64":
            h64 = ref["fp64"][1]
            m = min(nfin, len(h64))
            while m and not np.isfinite(h64[:m]).all():
                m -= 1
            if m:
                row["tip_history_err_vs_fp64"] = float(np.abs(hist[:m] - h64[:m]).max() / np.abs(h64[:m]).max())
                row["compared_iterations"] = 100 * m
            if np.isfinite(u).all() and np.isfinite(ref["fp64"][0]).all():
                row["u_err_vs_fp64"] = rel(u, ref["fp64"][0])
        emit(**row)
    o = O.OracleSim(case.replace(precision="fp64"))
    t0 = time.perf_counter()
    o.step(args.suite_cantilever_prefix)
    t_ora = time.perf_counter() - t0
    with L.Simulation(case.replace(precision="fp64")) as s:
        s.step(args.suite_cantilever_prefix)
        s.sync()
        ug = s.fields()[0]
    emit(config="cantilever_4096x256", precision="fp64", iterations=args.suite_cantilever_prefix,
         u_err_vs_oracle=rel(ug, o.fields()[0]),
         oracle_mlups=4096 * 256 * args.suite_cantilever_prefix / t_ora / 1e6, oracle_cores=O.OracleSim.threads(),
         oracle_sample=f"{args.suite_cantilever_prefix} iterations from the initial state ({t_ora:.1f} s)")


def suite_paper(args, L, I, O, emit, gpu_run, rel):
    # the paper's examples at its own sizes against the oracle over their
    # horizons, and a refinement ladder (self-convergence on the GPU, FP64)
    # the bending wave at each relaxation time of the paper's sweep; besides
    # parity, how far each tau moves u from tau = 0.55 (the paper compares
    # each against FE data, which is not available here)
    u_wave = {}
    for name, case, T in (("paper_tension_nh_0.3", I.paper_tension("nh", 0.3), 2.2),
                          ("paper_shear_svk_0.2", I.paper_shear("svk", 0.2), 2.2),
                          ("paper_wave_tau0.54", I.paper_wave(0.54), 12.0),
                          ("paper_wave_tau0.55", I.paper_wave(0.55), 12.0),
                          ("paper_wave_tau0.57", I.paper_wave(0.57), 12.0),
                          ("paper_wave_tau0.59", I.paper_wave(0.59), 12.0)):
        steps = int(round(T / O.params(case)["dt"]))
        (u, v, P), dt, unstable, _ = gpu_run(case, steps)
        o = O.OracleSim(case)
        t0 = time.perf_counter()
        o.step(steps)
        t_ora = time.perf_counter() - t0
        ur, vr, Pr = o.fields()
        row = dict(config=name, precision="fp64", nx=case.nx, ny=case.ny, iterations=steps, unstable_gpu=unstable,
                   u_err=rel(u, ur), v_err=rel(v, vr), P_err=rel(P, Pr), max_abs_u=float(np.abs(ur).max()),
                   gpu_mlups=case.nx * case.ny * steps / dt / 1e6,
                   oracle_mlups=case.nx * case.ny * steps / t_ora / 1e6, oracle_cores=O.OracleSim.threads())
        if name.startswith("paper_wave"):
            u_wave[case.tau] = u
        emit(**row)
    if 0.55 in u_wave:
        emit(config="paper_wave_tau_sweep", precision="fp64", t=12.0,
             u_change_vs_tau055={str(t): rel(u, u_wave[0.55]) for t, u in u_wave.items() if t != 0.55})
    for name, mk in (("tension_nh_0.3", lambda n: I.paper_tension("nh", 0.3, n=n)),
                     ("shear_svk_0.2", lambda n: I.paper_shear("svk", 0.2, n=n))):
        c20 = mk(20)
        K = int(round(2.2 / O.params(c20)["dt"]))  # iterations at n = 20; n = 20 * 2^m runs K * 2^m
        us = []
        for m in range(5):
            n = 20 * 2 ** m
            (u, _, _), dt, unstable, _ = gpu_run(mk(n), K * 2 ** m)
            us.append(u)
        diffs = []
        restrict = lambda f: 0.25 * (f[0::2, 0::2] + f[1::2, 0::2] + f[0::2, 1::2] + f[1::2, 1::2])
        for m in range(4):
            diffs.append(float(np.abs(restrict(us[m + 1]) - us[m]).max()))
        orders = [math.log2(diffs[m] / diffs[m + 1]) for m in range(3)]
        # the paper's grid error norms (Eq. griderror) of each coarser lattice
        # against the finest one restricted to it, evaluated on the GPU
        # (lbs_grid_error on the coarse lattice's handle)
        refs, f = [], us[4]
        for m in range(3, -1, -1):
            f = restrict(f)
            refs.insert(0, f)
        norms = []
        for m in range(4):
            with L.Simulation(mk(20 * 2 ** m)) as sim:
                sim.step(K * 2 ** m)
                sim.sync()
                norms.append(sim.grid_error(refs[m]))
        emit(config=f"paper_refinement_{name}", precision="fp64", n=[20 * 2 ** m for m in range(5)],
             t=K * O.params(c20)["dt"], diff_to_next=diffs, observed_order=orders,
             E2_vs_finest=[e[0] for e in norms], Einf_vs_finest=[e[1] for e in norms],
             E2_order=[math.log2(norms[m][0] / norms[m + 1][0]) for m in range(3)],
             Einf_order=[math.log2(norms[m][1] / norms[m + 1][1]) for m in range(3)])


def suite_roofline(args, L, I, torch, dev, emit):
    # roofline 16384^2, 500 iterations
    case = I.roofline(n=16384, nsteps=500)
    v0 = I.grf_velocity(case, device=dev)
    st = torch.cuda.Stream()
    uref = None
    for prec in ("fp64", "fp32", "fp16s"):
        r, u = time_precision(L, I, torch, prec, 16384, 495, 5, st, v0, uref)
        if prec == "fp64":
            uref = u
        emit(config="roofline_16384", precision=prec, **r)
        del u
        torch.cuda.empty_cache()
    cpu = oracle_rate(1024, 10.0)[0]
    emit(config="roofline_16384", oracle_mlups=cpu["value"], oracle_cores=cpu["cores"], oracle_sample=cpu["sample"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--suite-shear-steps", type=int, default=20000)
    ap.add_argument("--suite-cantilever-steps", type=int, default=100000)
    ap.add_argument("--suite-cantilever-prefix", type=int, default=1000)
    ap.add_argument("--serving-requests-suite", type=int, default=512)
    ap.add_argument("--suite-serving-steps-scale", type=float, default=1.0)
    ap.add_argument("--suite-parts", default="all",
                    help="comma list of tension,shear,cantilever,paper,serving,roofline")
    args = ap.parse_args()
    from paper_2502_00920_gb300 import build as B
    B.build()
    suite(args)


if __name__ == "__main__":
    main()
