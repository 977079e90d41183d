#!/usr/bin/env python
"""Benchmark of the BDIM incompressible-flow time step on B300.

One step = one Heun predictor-corrector step of the solver (two convection-
diffusion + BDIM stages, two projections each converged to a 1e-6 relative
Poisson residual, CFL update) through the C ABI of libwl.so.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload msphere]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Multi-GPU: the time step does not shard without a halo exchange, so N > 1 runs
N independent replicas (one per rank, weak scaling) and reports the aggregate.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s at 1e-6 Poisson residual (learned-guess vs plain MG); HBM GB/s"
UNIT = "cell-steps/s"


def workload(name):
    import synth
    table = {
        "tgv256": lambda: synth.config2_tgv(256),
        "tgv128": lambda: synth.config2_tgv(128),
        "tgv64": lambda: synth.config2_tgv(64),
        "sphere": lambda: synth.config3_sphere(),
        "msphere": lambda: synth.config5_moving_sphere(),
        # the same flow at 3/4 scale (384 x 192 x 192): the size ncu captures use
        "msphere384": lambda: synth.scaled(synth.config5_moving_sphere(), 0.75),
        "circle": lambda: synth.config1_circle(),
        "ellipse": lambda: synth.config4_ellipse(),
        "cylinder64": lambda: synth.cylinder_benchmark(64),
        "tgv_octant512": lambda: synth.tgv_octant(512),
        # 512^3 cells (134.22 M): the grid of the paper's largest TGV benchmark
        "tgv_octant1024": lambda: synth.tgv_octant(1024),
    }
    return table[name]()


def describe(case, prec):
    return {"workload": f"{case.name} {'x'.join(str(v) for v in case.n[:case.ndim])}",
            "cells": case.ncell, "nu": case.nu, "body": case.body.kind,
            "bc": ("periodic" if all(case.periodic[:case.ndim]) else
                   "inflow/slip/convective-exit" if case.exit_hi_x else
                   "slip walls" + (" (periodic " + "".join("xyz"[a] for a in range(case.ndim) if case.periodic[a]) + ")"
                                   if any(case.periodic[:case.ndim]) else "")),
            "precision": prec, "poisson_tol": 1e-6, "smoother": "PCG x4 per level, V(0,4)",
            "guess": "warm start (previous pressure); learned guess in learned_guess",
            "l2": "inputs larger than L2 (velocity alone > 126 MB)" if case.ncell * 12 > 126e6 else "small"}


# Bytes per cell of each kernel's algorithmic traffic (T = element size, nd =
# ndim): the arrays the method must read and write once per launch. Away from
# the body the Poisson coefficients are uniform and formed from the position,
# so the multigrid kernels move no coefficient arrays there (body tiles, a
# small fraction, also read them: not counted, so the figure is a lower bound).
def algo_bytes(name, T, nd, has_body=False, const_diag=False):
    """const_diag: a body-free grid with every axis periodic, where every cell
    has the same Jacobi diagonal and the kernels do not read 1/D."""
    m1 = nd * nd
    d = 0 if const_diag else 1
    return {
        "flux_pred": 2 * nd * T, "flux_pred_f": 2 * nd * T, "flux_pred_m": 2 * nd * T,
        "flux_corr": 3 * nd * T, "flux_corr_f": 3 * nd * T, "flux_corr_m": 3 * nd * T,
        "blend": (nd + nd + m1 + nd + nd) * T,
        "div": (nd + 2) * T,                          # u -> b (pair)
        "resid": (4 + 1 + 1 / 2 ** nd) * T,           # ph, pl, b, bl -> r, coarse r
        "restrict": (2 ** nd + 1) * T,                # per coarse cell
        "pcg_init": (1 / 2 ** nd + 1 + d + 2) * T,    # xc, r, (1/D) -> x, s
        "pcg_dq1": 3 * T,                             # s -> d, q (first iteration)
        "pcg_dq": 4 * T,                              # s, d_old -> d, q
        "pcg_u": (6 + d) * T,                         # x, d, s, q, (1/D) -> x, s
        "pcg_u_last": 3 * T,                          # x, d -> x
        "pcg_u_last_fine": 6 * T,                     # x, d, ph, pl -> ph, pl
        "grad": (2 + 2 * nd) * T,                     # ph, pl, u -> u
        "cfl": nd * T,
        "measure": ((nd + m1 + nd) if has_body else nd) * T,
        "measure_sampled": (nd + m1 + nd + 3 * nd) * T,   # d, n -> c, mu1 n (in place)
    }.get(name)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel, case):
    """DRAM bytes per launch of `kernel` on `case` from the committed ncu
    summary (profiles/traffic.json), if it was taken on the kernel's current
    source files and on the same flow: either the same grid, or the same flow
    on a smaller grid whose traffic is scaled by the cells a launch processes
    (the entry then says "scaled_from"). Else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get(f"{kernel}@{case.name}")
    if not e or e.get("source_hash") != source_hash(e.get("source_files", [])):
        return None
    return int(round(e["dram_bytes_per_cell"] * case.ncell))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        # wait (at most 10 s) for the first sample, so that the timed region
        # that follows is covered
        t0 = time.time()
        while self.p is not None and time.time() - t0 < 10.0:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[3:7]):
                if v.strip().lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(name):
    """The bounded workload the FP64 oracle is timed on for a bench workload:
    the same flow at its oracle size (the moving sphere at 128x64x64, the
    fixed sphere at 128x64x64, the Taylor-Green vortex at 96^3, ...); the
    oracle's cost per cell-step does not depend on the size."""
    import synth
    case = workload(name)
    if case.ncell <= 600_000:
        return case
    if name.startswith("tgv") and "octant" not in name:
        return synth.config2_tgv(96)
    f = (524288 / case.ncell) ** (1.0 / case.ndim)
    f = 2.0 ** round(np.log2(f)) if case.ndim == 3 else 0.25
    return synth.scaled(case, f)


def time_oracle(case, steps, threads):
    """Oracle steps of `case` from its start (one untimed step first) with
    `threads` OpenMP threads: (cell-steps/s, seconds)."""
    import oracle
    oracle.set_threads(threads)
    s = oracle.Sim(case, tol=1e-6)
    s.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        s.step()
    dt = time.perf_counter() - t0
    return case.ncell * steps / dt, dt


def cpu_baseline(name, steps=4):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload
    (oracle_sample), on all host cores; a single-thread step alongside."""
    import oracle
    case = oracle_sample(name)
    cores = oracle.host_cores()
    v, dt = time_oracle(case, steps, cores)
    v1, dt1 = time_oracle(case, 1, 1)
    oracle.set_threads(cores)
    dims = "x".join(str(v) for v in case.n[:case.ndim])
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{case.name} {dims} ({case.ncell} cells), {steps} timed steps after 1 untimed, "
                      f"FP64 C oracle, OpenMP over all {cores} host cores, MG to 1e-6; {dt:.1f} s",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "single_thread": {"value": v1, "cores": 1, "sample": f"1 timed step, {dt1:.1f} s"}}


def max_over_ranks(x, dist, device):
    """The largest value of one host number over all ranks (x itself on one
    rank): the job takes as long as its slowest replica."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ncell, steps, world, seconds):
    """Whole-job throughput of `world` replicas: the cell-steps all ranks made
    over the slowest rank's time."""
    return ncell * steps * world / seconds


def run_reference(args, rank, world):
    """The oracle on the host cores: each step one oracle step of the bench
    workload's bounded sample (oracle_sample); rank 0 only."""
    if rank != 0:
        return 0
    import oracle
    case = oracle_sample(args.workload)
    cores = oracle.host_cores()
    oracle.set_threads(cores)
    s = oracle.Sim(case, tol=1e-6)
    for _ in range(args.warmup):
        s.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step()
    dt = time.perf_counter() - t0
    v = case.ncell * args.steps / dt
    prec = args.precision or ("f64" if args.workload == "circle" else "f32")
    dims = "x".join(str(x) for x in case.n[:case.ndim])
    sample = f"each step: one FP64 oracle step of {case.name} {dims}, OpenMP over all {cores} host cores"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (analytic fields, seeded noise)",
           "config": describe(workload(args.workload), prec) | {"reference_sample": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                            "cpu_model": cpu_model()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def tgv256_rate(steps, warmup):
    """The body-free Taylor-Green vortex 256^3 (FP32, plain multigrid to 1e-6):
    cell-steps/s over `steps` steps by CUDA events, for comparison with the
    moving-sphere headline."""
    import torch
    import synth
    from paper_2407_16032_b300 import sim_from_case
    case = synth.config2_tgv(256)
    sim = sim_from_case(case, "f32", tol=1e-6, itmax=32)
    u, ue = synth.initial_velocity(case)
    sim.set_velocity(torch.tensor(u, dtype=torch.float32, device="cuda"))
    for _ in range(max(warmup, 3)):
        sim.mom_step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(sim.stream)
    for _ in range(steps):
        sim.mom_step()
    b.record(sim.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    sim.close()
    return {"workload": "tgv256 256x256x256", "value": case.ncell * steps / (ms / 1000.0), "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="msphere")
    ap.add_argument("--no-tgv", action="store_true")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    # coarsest multigrid levels of up to this many cells are solved by the
    # dense FP64 operator (the library's default is 256)
    ap.add_argument("--coarse-dense-max", type=int, default=1024)
    ap.add_argument("--adjoint-spinup", type=int, default=2000)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world:
        # --gpus N is run as N processes (torchrun); a single process is one GPU
        print(f"bench.py: --gpus {args.gpus} but {world} process(es) (WORLD_SIZE); launch one process per GPU "
              f"with torch.distributed.run --nproc-per-node {args.gpus}", file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import synth
    from paper_2407_16032_b300 import build, sim_from_case
    if rank == 0 and world == 1:
        build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    case = workload(args.workload)
    prec = args.precision or ("f64" if args.workload == "circle" else "f32")
    sim = sim_from_case(case, prec, tol=1e-6, itmax=32)
    sim.set_coarse_dense_max(args.coarse_dense_max)
    u, ue = synth.initial_velocity(case)
    tdt = torch.float32 if prec == "f32" else torch.float64
    u_dev = torch.tensor(u, dtype=tdt, device="cuda")
    ue_dev = torch.tensor(ue, dtype=tdt, device="cuda")
    sim.set_velocity(u_dev, ue_dev)
    stream = torch.cuda.current_stream()

    clk = Clocks(local)   # sampling starts before the warm-up (its start-up stays out of the timed region)
    for _ in range(max(args.warmup, 3)):
        sim.mom_step()
    _, l0 = sim.info()
    vcyc = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st, rc = sim.mom_step()
        vcyc.append(st.proj[0].vcycles + st.proj[1].vcycles)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    _, l1 = sim.info()
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_rate(case.ncell, args.steps, world, ms / 1000.0)

    # ---- roofline of the dominant kernel: per-kernel CUDA-event timing pass
    roof, kernels = None, []
    if not args.no_profile:
        sim.profile(True)
        for _ in range(2):
            sim.mom_step()
        rows = sim.profile_report()
        sim.profile(False)
        cdiag = case.body.kind == "none" and all(case.periodic[:case.ndim])
        tot = sum(r[3] for r in rows)
        by = {}
        for nm, lv, n, tms, cells in rows:
            by.setdefault(nm, [0.0, 0, 0.0])
            by[nm][0] += tms
            b = algo_bytes(nm, 4 if prec == "f32" else 8, case.ndim, case.body.kind != "none", cdiag)
            if b is not None:
                by[nm][2] += b * cells * n
            by[nm][1] += n
        peak, src = load_peaks()
        for nm, (tms, n, byt) in sorted(by.items(), key=lambda kv: -kv[1][0]):
            kernels.append({"kernel": nm, "share": round(tms / tot, 4), "launches": n,
                            "avg_us": round(1000 * tms / n, 2),
                            "GBps": round(byt / (tms / 1000) / 1e9, 1) if byt else None})
        fine = [(nm, lv, n, tms, cells) for nm, lv, n, tms, cells in rows if lv == 0 and
                algo_bytes(nm, 4, case.ndim) is not None]
        top = max(fine, key=lambda r: r[3])
        nm, lv, n, tms, cells = top
        bpl = algo_bytes(nm, 4 if prec == "f32" else 8, case.ndim, case.body.kind != "none", cdiag) * cells
        ach = bpl / (tms / n / 1000) / 1e9
        roof = {"bound": "hbm", "kernel": f"{nm} (fine level)", "achieved": round(ach, 1), "peak": peak,
                "unit": "GB/s", "frac": round(ach / peak, 4), "peak_source": src,
                "algorithmic_bytes_per_launch": int(bpl), "traffic": traffic_for(nm, case)}

    # ---- learned Poisson guess vs plain multigrid on the same workload. Both
    # learned parts are fitted on the solver's own converged projections: the
    # temporal guess (a 1x1x1 convolution over each stage's pressure history,
    # least squares in the residual norm) and the coarse-level CNN (Adam on
    # the GPU). Arms from the same state, each timed over the same steps after
    # three untimed steps (the temporal guess needs two steps of history).
    learned = None
    if not args.no_learned:
        sim.tguess_mode(collect=True, use=False)
        sim.guess_setup(level=2, capacity=64)
        sim.guess_mode(collect=True)
        for _ in range(16):
            sim.mom_step()
        sim.guess_mode(collect=False)
        sim.tguess_mode(collect=False, use=False)
        tw, tratio = sim.tguess_fit()
        t0 = time.perf_counter()
        loss0, loss1 = sim.guess_train(iters=300, lr=2e-3, batch=4, seed=0)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        su, sue = sim.get_velocity()
        sp = sim.get_pressure()
        tt, dtt = sim.get_time()
        arms = {"plain": (False, False), "temporal": (True, False), "temporal+cnn": (True, True)}
        res = {}
        for name, (tgu, cnn) in arms.items():
            sim.set_velocity(su, sue)
            sim.set_pressure(sp)
            sim.set_time(tt, dtt)
            sim.tguess_mode(collect=False, use=tgu)
            sim.guess_mode(use=cnn)
            for _ in range(3):
                sim.mom_step()
            torch.cuda.synchronize()
            a, bq = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            vc, r0 = [], []
            a.record(stream)
            for _ in range(args.steps):
                st, rc = sim.mom_step()
                vc.append(st.proj[0].vcycles + st.proj[1].vcycles)
                r0.append(0.5 * (st.proj[0].rel_initial + st.proj[1].rel_initial))
            bq.record(stream)
            torch.cuda.synchronize()
            res[name] = {"value": case.ncell * args.steps / (a.elapsed_time(bq) / 1000.0),
                         "vcycles_per_step": statistics.mean(vc), "initial_rel_residual": statistics.mean(r0)}
        sim.guess_mode(use=False)
        sim.tguess_mode(collect=False, use=False)
        learned = {"value": res["temporal"]["value"], "plain_mg_value": res["plain"]["value"], "unit": UNIT,
                   "speedup": res["temporal"]["value"] / res["plain"]["value"], "arms": res,
                   "temporal": {"net": "1x1x1 conv over (H1, H1 - H2, Ho - H1) per projection stage",
                                "weights": {"predictor": tw[0].tolist(), "corrector": tw[1].tolist()},
                                "fit_residual_ratio": tratio.tolist(), "projections_fitted": 30},
                   "cnn": {"net": "bias-free ReLU 3D CNN 1-16-16-1, 3^3 kernels, BF16 tcgen05 convolutions (weight gradient on mma.sync), on MG level 2",
                           "train": {"samples": 32, "adam_steps": 300, "batch": 4, "loss_first": loss0,
                                     "loss_last": loss1, "seconds": t_train}}}

    # ---- adjoint of the flapping-foil window: heaving + pitching ellipse,
    # 1024 x 512 FP32, spun up from rest, then the mean thrust over a 200-step
    # window and its gradient with respect to the heave and pitch amplitudes
    # (checkpoints every 20 steps; backward = recomputation + adjoint sweep).
    # 200 steps: on this grid the adjoint agrees with central differences up to
    # about 360 steps and departs from them (and differs between FP32 and FP64)
    # beyond; the central differences at step 1e-3 are printed beside it.
    adjoint = None
    if not args.no_adjoint:
        c4 = synth.config4_ellipse()
        s4 = sim_from_case(c4, "f32", tol=1e-6, itmax=32)
        u4, ue4 = synth.initial_velocity(c4)
        s4.set_velocity(torch.tensor(u4, dtype=torch.float32, device="cuda"),
                        torch.tensor(ue4, dtype=torch.float32, device="cuda"))
        for _ in range(args.adjoint_spinup):
            s4.mom_step(allow_unconverged=True)
        U4, UE4 = s4.get_velocity()
        P4 = s4.get_pressure()
        T4, DT4 = s4.get_time()
        nwin, ck = 200, 20
        wv = (-1.0 / nwin, 0.0, 0.0)
        a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        a0.record(s4.stream)
        J, dts = s4.window_forward(nwin, ck, None, wv)
        a1.record(s4.stream)
        _, _, dp = s4.window_backward(1.0, tol=1e-6)
        a2.record(s4.stream)
        torch.cuda.synchronize()
        tf, tb = a0.elapsed_time(a1) / 1000.0, a1.elapsed_time(a2) / 1000.0
        wstats = s4.window_stats()
        fd = {}
        for name in ("heave_amp", "pitch_amp"):
            Js = []
            for sg in (1.0, -1.0):
                s4.set_body(dataclasses.replace(c4.body, **{name: getattr(c4.body, name) + sg * 1e-3}))
                s4.set_velocity(U4, UE4)
                s4.set_pressure(P4)
                s4.set_time(T4, DT4)
                Js.append(s4.window_forward(nwin, ck, dts, wv)[0])
            fd[name] = (Js[0] - Js[1]) / 2e-3
        adjoint = {"workload": f"ellipse2d {c4.n[0]}x{c4.n[1]} FP32, {args.adjoint_spinup}-step spin-up, "
                               f"{nwin}-step window, checkpoints every {ck}",
                   "objective": "mean thrust -(1/N) sum F_x", "J": J,
                   "dJ_dheave_amp": float(dp[0]), "dJ_dpitch_amp": float(dp[1]),
                   "central_difference_1e-3": {"dJ_dheave_amp": fd["heave_amp"], "dJ_dpitch_amp": fd["pitch_amp"]},
                   "adjoint_solves": wstats,
                   "forward_cell_steps_per_s": c4.ncell * nwin / tf,
                   "backward_cell_steps_per_s": c4.ncell * nwin / tb,
                   "backward_over_forward": tb / tf, "forward_s": tf, "backward_s": tb}
        s4.close()

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        hu = torch.empty_like(u_dev, device="cpu").pin_memory()
        hue = torch.empty_like(ue_dev, device="cpu").pin_memory()
        sim.get_velocity(hu, hue)
        n_e2e = max(3, args.steps // 2)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            sim.set_velocity(hu, hue)       # H2D of the step's input field
            st, rc = sim.mom_step()
            sim.get_velocity(hu, hue)       # D2H of the step's result field
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        el = max_over_ranks(el, dist, "cuda")
        nb = hu.numel() * hu.element_size() + (hue.numel() * hue.element_size() if case.exit_hi_x else 0)
        e2e = {"value": job_rate(case.ncell, n_e2e, world, el), "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb + 96}

    if rank == 0:
        cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(args.workload)
        tgv = None if (args.no_tgv or args.workload == "tgv256") else tgv256_rate(args.steps, args.warmup)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic (analytic fields, seeded noise)",
               "config": describe(case, prec) | {"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                                 "vcycles_per_step_mean": statistics.mean(vcyc),
                                                 "coarse_dense_max": args.coarse_dense_max},
               "hbm_GBps_dominant_kernel": roof["achieved"] if roof else None,
               "roofline": roof, "kernels": kernels[:16], "learned_guess": learned, "adjoint": adjoint,
               "cpu_baseline": cpu, "e2e": e2e, "tgv256": tgv,
               "gpu_launches": l1 - l0, "clocks": clocks,
               "paper_context": {"ns_per_cell_step": 1.57, "cell_steps_per_s": 6.4e8,
                                 "hw": "NVIDIA H100, FP32, TGV 134M cells (Sec. 4.1)"}}
        print(json.dumps(out))
    sim.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
