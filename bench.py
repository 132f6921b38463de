"""Benchmark: MISDC cell-updates/s of the concurrent MISDC sweep (CISDCQ-2, FP64).

Workload (default): 2D periodic 256x256 flame, synthetic 21-species/84-reaction
mechanism, Taylor-Green velocity (2 m/s), circular tanh kernel of radius 2 mm,
3 Gauss-Lobatto nodes, 4 sweeps, nu = 2, dt = 5e-6 s. One "step" = one time
step of every cell (all nodes, sweeps and nested iterations).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank advances its own flame (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MISDC cell-updates/s, learned+mixed vs plain FP64 sweep, at 1e-8 rel err"
UNIT = "cell-updates/s"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12      # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
# dram__bytes_read.sum + dram__bytes_write.sum of one k_newton launch on this workload,
# from the ncu capture summarised in profiles/k_newton_flame2d_256_n21.md; None when the
# kernel has changed since that capture.
NEWTON_TRAFFIC_BYTES = 23.5e6


def workload_config(name, w, mech, fl, scheme, precision):
    return {"workload": name, "grid": [fl.nx, fl.ny, fl.nz], "cells": fl.nx * fl.ny * fl.nz,
            "species": mech.n_species, "reactions": mech.n_reactions, "nodes": w["nodes"],
            "sweeps": w["sweeps"], "nu": w["nu"], "dt": w["dt"], "scheme": scheme,
            "precision": precision, "l2": "flushed between steps (256 MB write)"}


def newton_flops(N, R, nnz):
    """FP64 flops (FMA = 2) of one Newton iteration and of the final rate evaluation
    per cell, exp/log calls counted separately."""
    n = N + 1
    thermo = N * 34                       # h, s, cp polynomials + scalings
    rates = R * 30                        # ln k_f, Delta g, ln K_c, products, q, dq/dT
    jac = nnz * 22 + 4 * N                # Jacobian rows + temperature row
    lu = (2 * n ** 3) // 3 + 2 * n * n    # augmented elimination + back substitution
    it = thermo + rates + jac + lu + 6 * n
    fin = thermo + R * 14 + 2 * nnz
    return it, fin, 2 * R + 1, 2 * R + 1   # flops/iter, flops/final, exp+log per iter, per final


class ClockSampler:
    def __init__(self, gpu_index=0):
        self.samples, self.proc, self.t = [], None, None
        self.gpu = gpu_index

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def cpu_oracle_rate(name, cells_side, steps=1):
    """Time the CPU oracle on a bounded sample of the workload (same mechanism, dt,
    sweeps, nu; a cells_side^2 flame). Returns (cell-updates/s, seconds, cells)."""
    import oracle as O
    from paper_1801_01201_gb300 import inputs as I
    w = I.WORKLOADS[name]
    mech = I.make_mechanism(w["seed"], *w["mech"])
    g = dict(w["grid"])
    if w["dim"] == 2:
        n = cells_side
        fl = I.flame_2d(mech, w["seed"], n=n, dx=g["dx"], amp=g["amp"], radius=n * g["dx"] / 4,
                        delta=4 * g["dx"])
    elif w["dim"] == 3:
        fl = I.flame_3d(mech, w["seed"], n=cells_side, dx=g["dx"], radius=cells_side * g["dx"] / 4)
    else:
        fl = I.flame_1d(mech, w["seed"], nx=cells_side, dx=g["dx"])
    ad = O.ADR(mech, fl)
    phi = ad.state_from_YT(fl.Y, fl.T)
    t0 = time.perf_counter()
    ad.step(phi, w["dt"], "CISDCQ", w["nodes"] - 1, w["sweeps"], w["nu"], n_steps=steps)
    el = time.perf_counter() - t0
    return fl.cells * steps / el, el, fl.cells


def time_variant(Solver, mech, fl, w, args, dev, state0, flush, stream, precision):
    """Cell-updates/s of the same workload with another precision (same timing rules)."""
    import torch
    sv = Solver(mech, fl, n_sweeps=w["sweeps"], nu=w["nu"], n_nodes=w["nodes"], scheme=args.scheme,
                precision=precision, profile=True, device=dev)
    state = state0.clone()
    for _ in range(args.warmup):
        sv.step(state, w["dt"], 1)
    torch.cuda.synchronize()
    sv.stats(reset=True)
    ms, nms = [], 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sv.step(state, w["dt"], 1, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        nms += sv.stage_times()["newton_ms"]
    st = sv.stats(reset=True)
    cells = fl.nx * fl.ny * fl.nz
    return {"precision": precision, "value": cells * args.steps / (sum(ms) / 1e3), "unit": UNIT,
            "ms_per_step": sum(ms) / args.steps, "newton_ms_per_step": nms / args.steps,
            "newton_iters_per_solve": st["newton_iters"] / max(st["newton_solves"], 1),
            "status": st["status_name"]}


def run_reference(args, rank, world):
    """Reference arm: the plain serial CPU oracle on this host, bounded samples."""
    if rank != 0:
        return 0
    from paper_1801_01201_gb300 import inputs as I
    name = args.workload
    w = I.WORKLOADS[name]
    side = args.ref_side
    for _ in range(args.warmup):
        cpu_oracle_rate(name, side, 1)
    times, cells = [], 0
    for _ in range(args.steps):
        r, el, cells = cpu_oracle_rate(name, side, 1)
        times.append(el)
    tot = sum(times)
    value = cells * args.steps / tot
    mech = I.make_mechanism(w["seed"], *w["mech"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": name, "species": mech.n_species, "reactions": mech.n_reactions,
                       "sweeps": w["sweeps"], "nu": w["nu"], "dt": w["dt"], "scheme": "CISDCQ"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%dx%d-cell flame of the same mechanism, dt, sweeps and nu per step" % (side, side)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="flame2d_256_n21")
    ap.add_argument("--scheme", default="CISDCQ")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--compare-mixed", type=int, default=1,
                    help="also time the mixed-precision sweep (reported as an extra field)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-side", type=int, default=64)
    ap.add_argument("--ref-side", type=int, default=32)
    ap.add_argument("--e2e-steps", type=int, default=3)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1801_01201_gb300 import inputs as I
    from paper_1801_01201_gb300.solver import Solver

    name = args.workload
    mech, fl, w = I.build_workload(name)
    sv = Solver(mech, fl, n_sweeps=w["sweeps"], nu=w["nu"], n_nodes=w["nodes"], scheme=args.scheme,
                precision=args.precision, profile=True, device=dev)
    cells = fl.nx * fl.ny * fl.nz
    state0 = sv.state_from_YT(fl.Y, fl.T)
    state = state0.clone()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        sv.step(state, w["dt"], 1)
    torch.cuda.synchronize()
    sv.stats(reset=True)
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, newton_ms, newton_launches, diff_ms, diff_launches = [], 0.0, 0, 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sv.step(state, w["dt"], 1, stream=stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        t = sv.stage_times()
        newton_ms += t["newton_ms"]
        newton_launches += t["newton_launches"]
        diff_ms += t["diffusion_ms"]
        diff_launches += t["diffusion_launches"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    st = sv.stats(reset=True)
    total_ms = sum(step_ms)
    if dist:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = tt.item()
    value = world * cells * args.steps / (total_ms / 1e3)

    # end to end through the host-buffer entry point (H2D + step + D2H per step)
    host = state0.cpu().pin_memory()
    e2e_times = []
    for _ in range(args.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv.step_host(host, w["dt"], 1)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_times)
    e2e_bytes = state0.numel() * 8
    e2e_value = world * cells * len(e2e_times) / e2e_s if e2e_times else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    nnz = int(np.count_nonzero(mech.nu_r - mech.nu_f))
    f_it, f_fin, x_it, x_fin = newton_flops(mech.n_species, mech.n_reactions, nnz)
    flops = st["newton_iters"] * f_it + st["newton_solves"] * f_fin
    exps = st["newton_iters"] * x_it + st["newton_solves"] * x_fin
    per_launch_flops = flops / max(newton_launches, 1)
    avg_launch_s = newton_ms / 1e3 / max(newton_launches, 1)
    achieved = per_launch_flops / avg_launch_s / 1e12
    roofline = {"kernel": "k_newton (reaction Newton, warp per cell)", "bound": "alu",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": NEWTON_TRAFFIC_BYTES,
                "peak_source": "FP64 nominal from unit counts and clock (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                "exp_log_calls_per_launch": exps / max(newton_launches, 1),
                "newton_ms_per_step": newton_ms / args.steps,
                "diffusion_ms_per_step": diff_ms / args.steps,
                "newton_iters_per_solve": st["newton_iters"] / max(st["newton_solves"], 1)}
    cpu = None
    if not args.no_cpu_baseline and world == 1 or (not args.no_cpu_baseline and rank == 0):
        try:
            r, el, c = cpu_oracle_rate(name, args.cpu_side, 1)
            cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "one time step of a %dx%d-cell flame, same mechanism/dt/sweeps/nu (%.1f s)" % (args.cpu_side, args.cpu_side, el)}
        except Exception as e:   # the baseline is informative, never fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: %s" % e}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(name, w, mech, fl, args.scheme, args.precision),
            "clocks": clk, "gpu_launches": st["kernel_launches"],
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_bytes,
                    "d2h_bytes_per_step": e2e_bytes},
            "roofline": roofline, "cpu_baseline": cpu,
            "status": st["status_name"], "newton_fail": st["newton_fail"]}
    if args.compare_mixed and args.precision == "fp64":
        line["mixed"] = time_variant(Solver, mech, fl, w, args, dev, state0, flush, stream, "mixed")
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
