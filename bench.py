"""Benchmark: MISDC cell-updates/s, learned + mixed-precision concurrent MISDC
against the plain FP64 sweep, at 1e-8 relative error.

Workload (default): 3D periodic 128^3 flame (2,097,152 cells), synthetic
21-species/84-reaction mechanism, random-phase solenoidal velocity of rms 3 m/s,
spherical tanh kernel of radius 2 mm, 3 Gauss-Lobatto nodes, 4 sweeps, nu = 2,
dt = 5e-6 s: the learned form's configuration, the largest that runs on one
GPU. One "step" = one time step of every cell (all nodes, sweeps and nested
iterations).

Three variants of the same workload are timed back to back, each from the same
initial state: the plain FP64 sweep, the mixed-precision sweep, and the learned
+ mixed sweep (the headline `value`). The learned guess is trained first, with
the library's own kernels, on solves recorded from a different flame of the
same mechanism; training is setup, outside the timed region. The headline's
error against the FP64 sweep after the same steps is reported per field.

Other workloads: --workload flame2d_256_n21 | flame2d_512_n53 | flame1d_128_n9 |
batch64_2d (64 independent flames, one graph launch per step, autotuned).

Roofline of the reaction Newton (the step's dominant kernel): algorithmic FP64
flops per launch from the device counters with the per cell-iteration counts
thermo 15N, rates R(10 + 4 nubar), Jacobian 2 R nubar^2, LU 2n^3/3 and one
solve 2n^2 (n = N + 1, nubar = molecules per reaction), against the FP64 FMA
throughput measured at start-up by the library's probe kernel.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank advances its own copy of the workload (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
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
FP64_NOMINAL_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
# dram__bytes_read.sum + dram__bytes_write.sum of one reaction-Newton launch, per
# (workload, variant), from the ncu captures summarised under profiles/; a variant
# missing here has changed since its capture (traffic reported as null).
NEWTON_TRAFFIC_BYTES = {("flame2d_256_n21", "learned_mixed"): 332.72e6 + 30.85e6}


def newton_flops(N, R, nnz, stats, mixed=False):
    """Algorithmic FP64 flops (FMA = 2) of the reaction-Newton launches behind
    `stats`, and their exp/log calls. An iteration that evaluates the rates does
    thermo (34N), the rates of progress (20R), the residual (2 nnz) and the update
    (6n), with 2R exponentials and one log; an iteration that assembles the
    Jacobian adds the rate derivatives (10R), the Jacobian (22 nnz + 4N) and, in
    mixed precision, the row equilibration (n^2) and the kept inverse of the new
    factor (5n^3/3); an FP64 factorisation adds 2n^3/3 + 2n^2, a kept-inverse
    chord step 2n^2. Certified solves and first chord steps taken from the stored
    reaction term evaluate no rate (4n for their residual and test). Every solve
    that is not certified ends with thermo at the solution (34N, a log and an
    exponential for theta). FP32 LU work of the mixed kernel is not counted."""
    n = N + 1
    it, jac = stats["newton_iters"], stats.get("newton_jacobians", stats["newton_iters"])
    lu64 = stats.get("newton_lu_fp64", jac) if mixed else it
    cert = stats.get("newton_certified", 0) if mixed else 0
    stored = stats.get("newton_stored_steps", 0) if mixed else 0
    ev = it - cert - stored
    per_it = 34 * N + 20 * R + 2 * nnz + 6 * n
    per_jac = 10 * R + 22 * nnz + 4 * N + ((n * n + (5 * n ** 3) // 3) if mixed else 0)
    per_lu = (2 * n ** 3) // 3 + 2 * n * n
    chord = (it - lu64) * 2 * n * n if mixed else 0
    fin = 34 * N
    fin_solves = stats["newton_solves"] - cert
    flops = (ev * per_it + (cert + stored) * 4 * n + jac * per_jac + lu64 * per_lu + chord
             + fin_solves * fin)
    exps = ev * (2 * R + 1) + fin_solves * 2
    return flops, exps

def mean_molecules(mech):
    """nubar: reactant plus product molecules per reaction, averaged."""
    return float(np.mean(mech.nu_f.sum(axis=1) + mech.nu_r.sum(axis=1)))


def newton_flops_counted(N, R, nubar, stats, mixed=False):
    """Algorithmic FP64 flops of the reaction-Newton launches behind `stats` with
    per cell-iteration counts: an iteration that evaluates the rates does thermo
    (15N) and the rates (R(10 + 4 nubar)); a Jacobian assembly adds 2 R nubar^2
    and its LU 2n^3/3 (in either precision); every iteration, and every solve
    that a kept factor certifies or starts from the stored reaction term, does
    one solve (2n^2: a product with the kept inverse, or two substitutions)."""
    n = N + 1
    it = stats["newton_iters"]
    jac = stats.get("newton_jacobians", it) if mixed else it
    cert = stats.get("newton_certified", 0) if mixed else 0
    stored = stats.get("newton_stored_steps", 0) if mixed else 0
    ev = it - cert - stored
    per_ev = 15 * N + R * (10 + 4 * nubar)
    per_jac = 2 * R * nubar ** 2 + 2.0 * n ** 3 / 3
    flops = ev * per_ev + jac * per_jac + (ev + cert + stored) * 2 * n * n
    return flops, {"rate_iterations": ev, "jacobians": jac, "certified": cert, "stored_steps": stored,
                   "N": N, "R": R, "nubar": nubar,
                   "per_rate_iteration": per_ev, "per_jacobian": per_jac, "per_solve": 2 * n * n}


def measure_fp_peaks(dev, reps=5):
    """Best-of-`reps` throughput (TFLOP/s) of the library's FP64 FMA, FP64
    tensor-core MMA and FP32 FMA probes over every SM (CUDA events around each
    launch, after one warm-up launch)."""
    import torch
    from paper_1801_01201_gb300 import solver as SV
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    st = torch.cuda.current_stream()
    out = {}
    for kind, iters in (("dfma", 20000), ("dmma", 4000), ("ffma", 200000)):
        blocks = sms * 8
        SV.probe_flops(kind, blocks, iters // 10, stream=st)
        best = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fl, _ = SV.probe_flops(kind, blocks, iters, stream=st)
            b.record(st)
            b.synchronize()
            best = max(best, fl / (a.elapsed_time(b) / 1e3) / 1e12)
        out[kind] = best
    return out


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


def oracle_sample(name, cells_side):
    """Mechanism, flame, dt and time-integration settings of a bounded CPU sample of
    the workload: a cells_side^2 (cells_side^3 in 3D) flame of the same mechanism."""
    from paper_1801_01201_gb300 import inputs as I
    if name in I.BATCHES:
        b = I.BATCHES[name]
        mech = I.make_mechanism(*b["mechs"][1])
        n = cells_side
        fl = I.flame_2d(mech, b["seed"], n=n, dx=b["dx"], amp=b["amp"], radius=n * b["dx"] / 4,
                        delta=4 * b["dx"])
        return mech, fl, 0.5 * sum(b["dt"]), b
    w = I.WORKLOADS[name]
    mech = I.make_mechanism(w["seed"], *w["mech"])
    g = dict(w["grid"])
    if w["dim"] == 2:
        n = cells_side
        fl = I.flame_2d(mech, w["seed"], n=n, dx=g["dx"], amp=g["amp"], radius=n * g["dx"] / 4,
                        delta=4 * g["dx"])
    elif w["dim"] == 3:
        n = max(4, round(cells_side ** (2.0 / 3.0)))
        fl = I.flame_3d(mech, w["seed"], n=n, dx=g["dx"], radius=n * g["dx"] / 4)
    else:
        fl = I.flame_1d(mech, w["seed"], nx=cells_side * cells_side, dx=g["dx"])
    return mech, fl, w["dt"], w


def cpu_oracle_rate(name, cells_side, steps=1):
    """Time the CPU oracle on a bounded sample of the workload. Returns
    (cell-updates/s, seconds, cells, description)."""
    import oracle as O
    mech, fl, dt, w = oracle_sample(name, cells_side)
    ad = O.ADR(mech, fl)
    phi = ad.state_from_YT(fl.Y, fl.T)
    t0 = time.perf_counter()
    ad.step(phi, dt, "CISDCQ", w["nodes"] - 1, w["sweeps"], w["nu"], n_steps=steps)
    el = time.perf_counter() - t0
    desc = "%d-cell %dD flame, mechanism %d/%d, dt %.3g, %d sweeps, nu %d" % (
        fl.cells, fl.dim, mech.n_species, mech.n_reactions, dt, w["sweeps"], w["nu"])
    return fl.cells * steps / el, el, fl.cells, desc


def run_reference(args, rank, world):
    """Reference arm: the plain serial CPU oracle on this host, bounded samples."""
    if rank != 0:
        return 0
    name = args.workload
    side = args.ref_side
    for _ in range(args.warmup):
        cpu_oracle_rate(name, side, 1)
    times, cells, desc = [], 0, ""
    for _ in range(args.steps):
        r, el, cells, desc = cpu_oracle_rate(name, side, 1)
        times.append(el)
    tot = sum(times)
    value = cells * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "scheme": "CISDCQ"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one time step per step of a " + desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def entries_for(name, grid=0):
    """[(mechanism, flame, dt)] and the time-integration settings of a workload;
    grid > 0 replaces the cells per side of a single-flame 2D or 3D workload (a
    smaller case of the same recipe, for profiling)."""
    from paper_1801_01201_gb300 import inputs as I
    if name in I.BATCHES:
        b = I.BATCHES[name]
        return I.build_batch(name), b
    w = I.WORKLOADS[name]
    over = None
    if grid > 0 and w["dim"] > 1:
        # the kernel radius scales with the box (same burnt fraction); the front
        # keeps its width in cells
        full = w["grid"].get("n", 128 if w["dim"] == 3 else 256)
        over = {"n": grid, "radius": 2e-3 * grid / full}
    mech, fl, w = I.build_workload(name, over)
    return [(mech, fl, w["dt"])], w


def training_flame(mech, fl, radius_frac=0.28):
    """A different flame of the same mechanism for recording training solves:
    another seed and kernel (radius radius_frac x the box), at most 128^2 (48^3)
    cells."""
    from paper_1801_01201_gb300 import inputs as I
    if fl.dim == 2:
        n = min(fl.nx, 128)
        L = n * fl.dx
        return I.flame_2d(mech, 4242, n=n, dx=fl.dx, amp=2.0, radius=radius_frac * L,
                          delta=min(2e-4, L / 16), centre=(0.41 * L, 0.57 * L))
    if fl.dim == 3:
        n = min(fl.nx, 48)
        return I.flame_3d(mech, 4242, n=n, dx=fl.dx, urms=3.0, radius=radius_frac * n * fl.dx)
    return I.flame_1d(mech, 4242, nx=fl.nx, dx=fl.dx)


# kernel radii (fractions of the training box) of the recording restarts
TRAIN_RADII = (0.28, 0.36, 0.22, 0.40, 0.32, 0.25)


def train_params(Solver, mech, fl, dt, w, dev, args):
    """Record solves on a training flame, train the MLP, return (params, info).

    The recording runs COLLECT_RESTARTS short runs of COLLECT_STEPS steps, each
    from a fresh kernel of another radius in the same velocity field: the
    fourth-order centred advection of a front a few cells wide leaves small
    undershoots behind it once the front has moved a few cells, and on the small
    training box (stronger strain) they grow within about ten steps; short runs
    from fresh states keep every recorded solve in the physical range."""
    import torch
    sv = None
    statuses = []
    t0 = time.perf_counter()
    for k in range(args.collect_restarts):
        tf = training_flame(mech, fl, TRAIN_RADII[k % len(TRAIN_RADII)])
        if sv is None:
            sv = Solver(mech, tf, n_sweeps=w["sweeps"], nu=w["nu"], n_nodes=w["nodes"],
                        scheme=args.scheme, precision="fp64", device=dev)
            sv.surrogate_init(seed=args.seed)
            sv.surrogate_collect(args.train_rows)
        x = sv.state_from_YT(tf.Y, tf.T)
        sv.step(x, dt, args.collect_steps)
        statuses.append(sv.stats()["status_name"])
    rows, _, _ = sv.surrogate_dataset()
    sv.surrogate_collect(0)
    curve = sv.surrogate_train(args.train_steps, batch=args.train_batch, lr=args.train_lr,
                               weight_decay=1e-4, seed=args.seed)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    p = sv.surrogate_save()
    info = {"rows": rows, "collect_restarts": args.collect_restarts, "collect_steps": args.collect_steps,
            "collect_status": statuses, "train_steps": args.train_steps, "batch": args.train_batch,
            "loss_first": float(curve[:10].mean()), "loss_last": float(curve[-50:].mean()),
            "seconds": el, "flame_cells": tf.cells}
    sv.close()
    return p, info


def lin_rounds_for(args, fl):
    """Refinement rounds of the mixed diffusion solve: the flag, else 2 on a 3D flame
    (dx = 1e-4 m: two rounds meet the 1e-12 residual check) and the library's three
    on the 1D/2D flames (dx = 4e-5 m, a stiffer operator)."""
    if args.lin_rounds >= 0:
        return args.lin_rounds
    return 2 if fl.dim == 3 else 0


class Runner:
    """One variant of the workload: a solver per flame (and a batch for several)."""

    def __init__(self, entries, w, args, dev, precision, params=None, tune=False):
        import torch
        from paper_1801_01201_gb300.solver import Solver, Batch
        self.entries = entries
        self.solvers = []
        self.states0 = []
        for mech, fl, dt in entries:
            sv = Solver(mech, fl, n_sweeps=w["sweeps"], nu=w["nu"], n_nodes=w["nodes"],
                        scheme=args.scheme, precision=precision, profile=len(entries) == 1,
                        mg_levels=args.mg_levels, rates_mma=bool(args.rates_mma),
                        lin_rounds=lin_rounds_for(args, fl), device=dev)
            st = sv.state_from_YT(fl.Y, fl.T)
            if params is not None:
                sv.surrogate_load(params[id(mech)])
                sv.surrogate_enable(True, s_min=args.s_min)
                sv.surrogate_sweeps(args.sg_sweeps)
            if tune:
                T = torch.as_tensor(fl.T, device=dev).contiguous()
                sv.autotune(st, T, dt)
            self.solvers.append(sv)
            self.states0.append(st)
        self.dts = [dt for _, _, dt in entries]
        self.batch = Batch(self.solvers) if len(entries) > 1 else None
        self.run_steps = w["steps"]
        self.cells = sum(fl.cells for _, fl, _ in entries)
        self.reset()

    def reset(self):
        self.states = [x.clone() for x in self.states0]
        self.taken = 0

    def step(self, stream=None):
        if self.taken == self.run_steps:
            # the workload is a run of run_steps steps from its initial state:
            # start it again (a device copy, on the stream the step is timed on)
            import torch
            with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
                for x, x0 in zip(self.states, self.states0):
                    x.copy_(x0)
            self.taken = 0
        self.taken += 1
        if self.batch is not None:
            self.batch.step(self.states, self.dts, 1, stream=stream)
        else:
            self.solvers[0].step(self.states[0], self.dts[0], 1, stream=stream)

    def stats(self):
        if self.batch is not None:
            return self.batch.stats(reset=True)
        return self.solvers[0].stats(reset=True)

    def stage_times(self):
        if self.batch is not None:
            return None
        return self.solvers[0].stage_times()


def max_over_ranks(total_ms, dist=None, device=None):
    """The slowest rank's timed-region length (ms): the whole job ends with it."""
    if not dist:
        return total_ms
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, cells, steps, total_ms):
    """Cell-updates/s of the whole job: every rank advances its own copy of the
    workload (weak scaling), so the units are world x cells x steps."""
    return world * cells * steps / (total_ms / 1e3)


def timed(runner, args, flush, stream, dist=None, clocks=None, label="timed"):
    """W untimed steps, then K steps timed with CUDA events (L2 flushed between).
    The timed steps sit in an NVTX range named `label` (a profiler can select them)."""
    import torch
    for _ in range(args.warmup):
        runner.step()
    torch.cuda.synchronize()
    runner.stats()
    if dist:
        dist.barrier()
    if clocks:
        clocks.start()
    torch.cuda.synchronize()
    ms, newton_ms, newton_n, diff_ms = [], 0.0, 0, 0.0
    torch.cuda.nvtx.range_push(label)
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        runner.step(stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        t = runner.stage_times()
        if t:
            newton_ms += t["newton_ms"]
            newton_n += t["newton_launches"]
            diff_ms += t["diffusion_ms"]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    if dist:
        dist.barrier()
    st = runner.stats()
    total = max_over_ranks(sum(ms), dist, flush.device)
    return dict(total_ms=total, ms=ms, newton_ms=newton_ms, newton_launches=newton_n,
                diffusion_ms=diff_ms, stats=st, clocks=clk)


def field_errors(solver, a, b):
    """Relative error of state a against b: mass fractions max|dY| / max|Y| over all
    species and cells (the Newton tolerance is absolute in Y, so trace species
    are converged to ~1e-12 absolute in either precision; the worst per-species
    ratio ||dY_i|| / ||Y_i|| is reported beside it), the temperature and h."""
    N = solver.N
    A, B = a.cpu().numpy(), b.cpu().numpy()
    den = np.maximum(np.max(np.abs(B), axis=1), 1e-300)
    e = np.max(np.abs(A - B), axis=1) / den
    Ta = solver.temperature(a[:N], a[N]).cpu().numpy()
    Tb = solver.temperature(b[:N], b[N]).cpu().numpy()
    return {"Y": float(np.max(np.abs(A[:N] - B[:N])) / np.max(np.abs(B[:N]))),
            "Y_species_worst": float(e[:N].max()), "h": float(e[N]),
            "T": float(np.max(np.abs(Ta - Tb)) / np.max(np.abs(Tb)))}


def rates_compare(entries, args, dev, rank):
    """Production rates wdot = diag(W) nu^T q of every cell of the first flame, as
    the sparse FP64 FMA sum and as FP64 tensor-core (m8n8k4) tiles: CUDA-event time
    per launch (after warm-up, L2 flushed between launches) and the largest
    difference between the two, relative to the largest rate."""
    import torch
    from paper_1801_01201_gb300.solver import Solver
    mech, fl, dt = entries[0]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    Y = torch.as_tensor(fl.Y, device=dev).contiguous()
    T = torch.as_tensor(fl.T, device=dev).contiguous()
    out, res = {}, {}
    for mma in (False, True):
        sv = Solver(mech, fl, rates_mma=mma, device=dev)
        st = torch.cuda.current_stream()
        for _ in range(args.warmup):
            res[mma] = sv.production_rates(Y, T, stream=st)
        ms = []
        for _ in range(max(args.steps, 1)):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            res[mma] = sv.production_rates(Y, T, stream=st)
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        out["tensor_core_ms" if mma else "sparse_fma_ms"] = statistics.median(ms)
    d = (res[True] - res[False]).abs().max().item() / res[False].abs().max().item()
    nnz = int(np.count_nonzero(mech.nu_r - mech.nu_f))
    n_tiles = sum(1 for j in range(0, mech.n_species, 8) for k in range(0, mech.n_reactions, 4)
                  if np.any((mech.nu_r - mech.nu_f)[k:k + 4, j:j + 8]))
    line = {"rates_compare": out, "cells": fl.cells, "species": mech.n_species,
            "reactions": mech.n_reactions, "nnz_nu": nnz, "mma_tiles": n_tiles,
            "contraction_flops_per_cell": {"sparse_fma": 2 * nnz, "tensor_core": 512 * n_tiles / 8},
            "max_rel_diff": d, "workload": args.workload}
    if rank == 0:
        print(json.dumps(line))
    return 0


def diffusion_compare(entries, args, dev, rank):
    """One implicit diffusion solve (I - wdt D L_theta) x = rhs of every solved field
    of the first flame, with wdt = --diffusion-compare: Chebyshev-accelerated Jacobi
    against multigrid V-cycles (--mg-levels, default 4), each in FP64 and in mixed
    precision (FP32 inner solves / FP32 coarse levels). CUDA-event time per solve
    (L2 flushed before each), fine-level sweeps per field, and the largest
    difference from the FP64 Chebyshev solution relative to each field's scale."""
    import torch
    from paper_1801_01201_gb300.solver import Solver
    mech, fl, dt = entries[0]
    wdt = args.diffusion_compare
    levels = args.mg_levels if args.mg_levels > 1 else 4
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out, ref = {}, None
    for lv, prec in ((1, "fp64"), (1, "mixed"), (levels, "fp64"), (levels, "mixed")):
        sv = Solver(mech, fl, mg_levels=lv, precision=prec, device=dev)
        coef = sv.state_from_YT(fl.Y, fl.T)
        st = torch.cuda.current_stream()
        for _ in range(args.warmup):
            x = sv.diffusion_solve(wdt, coef, coef, stream=st)
        sv.stats()   # reset the counters after the warm-up
        ms = []
        for _ in range(max(args.steps, 1)):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            x = sv.diffusion_solve(wdt, coef, coef, stream=st)
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        stt = sv.stats()
        key = "%s_%s" % ("chebyshev" if lv == 1 else "multigrid%d" % levels, prec)
        if ref is None:
            ref = x
        scale = ref.abs().amax(dim=1, keepdim=True).clamp_min(1e-300)
        out[key] = {"ms": statistics.median(ms), "status": stt["status_name"],
                    "fine_sweeps_per_solve": stt["lin_sweeps"] / max(args.steps, 1),
                    "max_rel_diff_vs_fp64_chebyshev": ((x - ref).abs() / scale).max().item()}
    line = {"diffusion_compare": out, "wdt": wdt, "cells": fl.cells, "fields": mech.n_species,
            "workload": args.workload}
    if rank == 0:
        print(json.dumps(line))
    return 0


def nu_compare(entries, w, args, dev, rank):
    """Adaptive nested iterations against fixed nu on the first flame: K FP64 steps
    (after W warm-up steps, L2 flushed before each) with the workload's nu, with
    fixed nu = NUMAX and with the adaptive rule capped at NUMAX. Reports ms per
    step, nested iterations per sweep and each state's difference from the fixed
    nu = NUMAX state (per-field max-norm relative to the field's scale)."""
    import torch
    from paper_1801_01201_gb300.solver import Solver
    numax, eta, rho = args.nu_compare.split(",")
    numax, eta, rho = int(numax), float(eta), float(rho)
    mech, fl, dt = entries[0]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    out, states = {}, {}
    for key, nu, rule in (("fixed_nu%d" % w["nu"], w["nu"], None), ("fixed_nu%d" % numax, numax, None),
                          ("adaptive_max%d" % numax, numax, (eta, rho))):
        sv = Solver(mech, fl, n_sweeps=w["sweeps"], nu=nu, n_nodes=w["nodes"], nu_rule=rule, device=dev)
        x0 = sv.state_from_YT(fl.Y, fl.T)
        x = x0.clone()
        for _ in range(args.warmup):
            sv.step(x, dt, 1, stream=st)
        sv.stats()
        x.copy_(x0)   # the same buffer: the captured step is reused
        ms = []
        for _ in range(max(args.steps, 1)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            sv.step(x, dt, 1, stream=st)
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        t = sv.stats()
        states[key] = x
        out[key] = {"ms_per_step": statistics.median(ms), "status": t["status_name"],
                    "nested_per_sweep": t["nested_iterations"] / (max(args.steps, 1) * w["sweeps"]),
                    "newton_iters_per_solve": t["newton_iters"] / max(t["newton_solves"], 1)}
    ref = states["fixed_nu%d" % numax]
    scale = ref.abs().amax(dim=1, keepdim=True).clamp_min(1e-300)
    for k, x in states.items():
        out[k]["max_rel_diff_vs_fixed_max"] = ((x - ref).abs() / scale).max().item()
    line = {"nu_compare": out, "rule": {"nu_max": numax, "eta": eta, "rho_stall": rho},
            "steps": args.steps, "workload": args.workload, "cells": fl.cells}
    if rank == 0:
        print(json.dumps(line))
    return 0


def concurrency_compare(entries, w, args, dev, rank):
    """The paper's cost question on this GPU (Sec. 3.2.2, eq. simple_parallel_speedup),
    measured on the first flame in FP64. Arms: serial MISDCQ; CISDCQ-nu with the
    diffusion and reaction stages on one stream and on two streams; CISDCQ with
    adaptive nested iterations (cap nu + 2) on two streams. For every arm and every
    sweep count k = 1..K (one solver each): the device time of one time step
    (CUDA events, median of --steps after --warmup, L2 flushed), the measured stage
    costs Upsilon_AD (one diffusion solve of all fields) and Upsilon_R (one
    reaction-Newton launch), and the state after the step, which gives the sweep
    increment inc(k) = max over fields of ||phi^{M,(k)} - phi^{M,(k-1)}||_1 /
    ||phi^{M,(k-1)}||_1 (phi^{M,(0)} = phi^n). As in the paper's Tables 3 and 5,
    N_M = K MISDCQ sweeps set the target eps = inc_MISDCQ(K), and N_C is the first
    sweep of an arm with inc <= eps. Reported per arm: N_C, the measured ratio
    t_MISDCQ(N_M) / t_arm(N_C), and the paper's model
    R_nu = (N_M / N_C) alpha M / (alpha nu + M - 1), alpha = (U_AD + U_R) / max(U_AD, U_R)
    from the measured stage costs (nu: the mean nested iterations per sweep)."""
    import torch
    from paper_1801_01201_gb300.solver import Solver
    K = args.concurrency
    mech, fl, dt = entries[0]
    w = dict(w)
    if args.nodes:
        w["nodes"] = args.nodes
    nu, M = w["nu"], w["nodes"] - 1
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    arms = [("misdcq", dict(scheme="MISDCQ", nu=1, two_streams=False)),
            ("cisdcq_nu%d_one_stream" % nu, dict(scheme="CISDCQ", nu=nu, two_streams=False)),
            ("cisdcq_nu%d_two_streams" % nu, dict(scheme="CISDCQ", nu=nu, two_streams=True)),
            ("cisdcq_nu%d_%d_stream_pairs" % (nu, nu), dict(scheme="CISDCQ", nu=nu, two_streams=True,
                                                           lanes=nu)),
            ("cisdcq_adaptive_max%d_two_streams" % (nu + 2),
             dict(scheme="CISDCQ", nu=nu + 2, two_streams=True, nu_rule=(0.02, 0.9)))]
    x0 = None
    out = {}
    for name, kw in arms:
        res = {"ms_per_step": [], "inc": [], "U_AD_ms": [], "U_R_ms": [], "nested_per_sweep": []}
        prev = None
        for k in range(1, K + 1):
            sv = Solver(mech, fl, n_sweeps=k, n_nodes=w["nodes"], profile=True, device=dev, **kw)
            if x0 is None:
                x0 = sv.state_from_YT(fl.Y, fl.T)
                prev0 = x0.clone()
            x = x0.clone()
            for _ in range(max(args.warmup, 1)):
                x.copy_(x0)
                sv.step(x, dt, 1, stream=st)
            sv.stats()
            ms, uad, ur = [], [], []
            for _ in range(max(args.steps, 1)):
                x.copy_(x0)
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                sv.step(x, dt, 1, stream=st)
                b.record(st)
                b.synchronize()
                ms.append(a.elapsed_time(b))
                t = sv.stage_times()
                uad.append(t["diffusion_ms"] / max(t["diffusion_launches"], 1))
                ur.append(t["newton_ms"] / max(t["newton_launches"], 1))
            stt = sv.stats()
            assert stt["status_name"] == "OK", stt
            ref = prev0 if prev is None else prev
            d = (x - ref).abs().sum(dim=1) / ref.abs().sum(dim=1).clamp_min(1e-300)
            res["inc"].append(float(d.max()))
            res["ms_per_step"].append(statistics.median(ms))
            res["U_AD_ms"].append(statistics.median(uad))
            res["U_R_ms"].append(statistics.median(ur))
            res["nested_per_sweep"].append(stt["nested_iterations"] / max(args.steps, 1) / k
                                           if kw["scheme"] == "CISDCQ" else 1.0)
            prev = x.clone()
            sv.close()
            del sv
            torch.cuda.synchronize()
        out[name] = res
    mis = out["misdcq"]
    eps = mis["inc"][K - 1]
    # the model's stage costs are those of a stage running alone (the one-stream
    # arm): on two streams the events around a stage also time its neighbour's work
    iso = out["cisdcq_nu%d_one_stream" % nu]
    for name, res in out.items():
        nc = next((k + 1 for k, v in enumerate(res["inc"]) if v <= eps), None)
        res["N_C"] = nc
        if nc is None or name == "misdcq":
            continue
        uad, ur = iso["U_AD_ms"][nc - 1], iso["U_R_ms"][nc - 1]
        alpha = (uad + ur) / max(uad, ur)
        nub = res["nested_per_sweep"][nc - 1]
        res["alpha"] = alpha
        res["R_nu_model"] = (K / nc) * alpha * M / (alpha * nub + M - 1)
        res["R_nu_measured"] = mis["ms_per_step"][K - 1] / res["ms_per_step"][nc - 1]
    line = {"concurrency": out, "N_M": K, "eps": eps, "nodes": w["nodes"], "nu": nu, "workload": args.workload,
            "pipelined_gain_at_%d_sweeps" % min(K, w["sweeps"]):
                out["cisdcq_nu%d_two_streams" % nu]["ms_per_step"][min(K, w["sweeps"]) - 1]
                / out["cisdcq_nu%d_%d_stream_pairs" % (nu, nu)]["ms_per_step"][min(K, w["sweeps"]) - 1],
            "cells": fl.cells, "species": mech.n_species, "dt": dt, "steps": args.steps, "warmup": args.warmup,
            "two_stream_gain_at_%d_sweeps" % min(K, w["sweeps"]):
                out["cisdcq_nu%d_one_stream" % nu]["ms_per_step"][min(K, w["sweeps"]) - 1]
                / out["cisdcq_nu%d_two_streams" % nu]["ms_per_step"][min(K, w["sweeps"]) - 1]}
    if rank == 0:
        print(json.dumps(line))
    return 0


def pde_bench(args, dev, rank):
    """The nonlinear test PDE of Sec. 5.2 (n_x = 200 on [0, 20], a = 1, 5 Gauss-Lobatto
    nodes, dt = 0.05, CISDCQ-3, 10 sweeps) on INSTANCES independent instances in one
    launch per step (d ~ U[2, 16], r = 2d, random front positions; inputs are
    read from HBM once per launch, every node array stays in shared memory).
    Reports cell-updates/s (CUDA events around each launch, L2 flushed between), the
    kernel's algorithmic FP64 flops against the FP64 peak, and the oracle on one
    host core on one instance."""
    import torch
    import oracle as O
    from paper_1801_01201_gb300 import solver as SV
    nx, lx, dt, M, sweeps, nu = 200, 20.0, 0.05, 4, 10, 3
    n = args.pde
    rng = np.random.default_rng(args.seed)
    d = rng.uniform(2.0, 16.0, n)
    prm = np.stack([np.ones(n), d, 2 * d, np.ones(n), np.zeros(n)], axis=1)
    x = (np.arange(nx) + 0.5) * lx / nx
    phi0 = np.stack([0.5 * (1 + np.tanh(rng.uniform(12, 28) - 2 * x)) for _ in range(n)])
    phi = torch.as_tensor(phi0, device=dev)
    P = torch.as_tensor(prm, device=dev)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        SV.pde_step(phi, P, dt, scheme="CISDCQ", n_nodes=M + 1, n_sweeps=sweeps, nu=nu, stream=st)
    ms = []
    cur = phi
    for _ in range(max(args.steps, 1)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        cur, incr, status = SV.pde_step(cur, P, dt, scheme="CISDCQ", n_nodes=M + 1, n_sweeps=sweeps,
                                        nu=nu, stream=st)
        b.record(st)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ok = int((status != 0).sum().item()) == 0
    # first step of instance 0 against the oracle
    one, _, _ = SV.pde_step(phi[:1].contiguous(), P[:1].contiguous(), dt, scheme="CISDCQ", n_nodes=M + 1,
                            n_sweeps=sweeps, nu=nu, stream=st)
    t0 = time.perf_counter()
    want, _ = O.pde_step("CISDCQ", M, sweeps, nu, dt, phi0[0], Lx=lx, a=1.0, d=d[0], r=2 * d[0])
    cpu_s = time.perf_counter() - t0
    err = float(np.max(np.abs(one[0].cpu().numpy() - want)))
    t = statistics.median(ms) / 1e3
    rate = n * nx / t
    peak = measure_fp_peaks(dev)["dfma"]
    # algorithmic FP64 flops per cell and node stage (an FMA counts 2): right-hand
    # side 8(M+1) + 6(M-1), band substitutions 14, Newton 3 x 14, F_A and F_D 24,
    # reaction term 3; per cell and step sweeps x nu x M stages + 40 at phi^n
    per_stage = 8 * (M + 1) + 6 * (M - 1) + 14 + 42 + 24 + 3
    flops = n * nx * (sweeps * nu * M * per_stage + 40)
    achieved = flops / t / 1e12
    line = {"pde": {"workload": "pde1d_200 (Sec. 5.2 nonlinear test PDE), %d instances x %d cells, "
                                "5 nodes, CISDCQ-%d, %d sweeps, dt %.2g" % (n, nx, nu, sweeps, dt),
                    "value": rate, "unit": "cell-updates/s", "ms_per_step": t * 1e3, "status_ok": ok,
                    "max_abs_err_vs_oracle": err,
                    "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                                 "unit": "TFLOP/s", "frac": achieved / peak,
                                 "peak_source": "measured: FP64 FMA probe (misdc_probe_flops), of measured",
                                 "flops_per_cell_update": flops / (n * nx)},
                    "cpu_baseline": {"value": nx / cpu_s, "unit": "cell-updates/s", "cores": 1,
                                     "kind": "oracle", "sample": "one instance, one step"}},
            "steps": args.steps, "warmup": args.warmup}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="flame3d_128_n21")
    ap.add_argument("--grid", type=int, default=0,
                    help="cells per side of a 2D/3D single-flame workload (default: the workload's)")
    ap.add_argument("--scheme", default="CISDCQ")
    ap.add_argument("--headline", default="learned_mixed", choices=["learned_mixed", "mixed", "fp64"])
    ap.add_argument("--autotune", type=int, default=-1, help="1/0; default: on for batches")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-side", type=int, default=64)
    ap.add_argument("--ref-side", type=int, default=32)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--collect-steps", type=int, default=4,
                    help="steps of each recording run of the training flame")
    ap.add_argument("--collect-restarts", type=int, default=4,
                    help="recording runs, each from a fresh kernel of another radius")
    ap.add_argument("--train-rows", type=int, default=10_000_000)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--train-batch", type=int, default=8192)
    ap.add_argument("--train-lr", type=float, default=2e-3)
    ap.add_argument("--s-min", type=float, default=1e-4)
    ap.add_argument("--sg-sweeps", type=int, default=1,
                    help="learned guess in the first SG_SWEEPS sweeps of a step only (0: all)")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--rates-mma", type=int, default=0,
                    help="1: production rates on the FP64 tensor cores (all variants)")
    ap.add_argument("--mg-levels", type=int, default=1,
                    help=">1: multigrid diffusion solves (FP32 coarse levels when mixed)")
    ap.add_argument("--diffusion-compare", type=float, default=0.0, metavar="WDT",
                    help="instead of the step: time one implicit diffusion solve of weight WDT "
                         "on the workload's initial state, Chebyshev against multigrid, FP64 and mixed")
    ap.add_argument("--nu-compare", default="", metavar="NUMAX,ETA,RHO",
                    help="instead of the headline: FP64 steps with the workload's nu, with fixed "
                         "nu = NUMAX and with adaptive nested iterations (cap NUMAX, rule ETA, RHO)")
    ap.add_argument("--pde", type=int, default=0, metavar="INSTANCES",
                    help="instead of the step: the nonlinear test PDE of Sec. 5.2 on INSTANCES "
                         "independent 200-cell instances, one launch per step")
    ap.add_argument("--concurrency", type=int, default=0, metavar="K",
                    help="instead of the headline: serial MISDCQ against CISDCQ-nu on one and on two "
                         "streams and with adaptive nu, sweeps 1..K each: step times, stage costs, "
                         "sweep increments, sweeps to the MISDCQ tolerance, measured and modelled R_nu")
    ap.add_argument("--lin-rounds", type=int, default=-1,
                    help="mixed precision: FP64-residual refinement rounds of the diffusion solve "
                         "(0: the library's default, 3; default: 2 on 3D flames, 3 on the stiffer "
                         "1D/2D ones); the line reports the residual and the error against the "
                         "FP64 sweep")
    ap.add_argument("--nodes", type=int, default=0,
                    help="--concurrency: Gauss-Lobatto nodes (default: the workload's)")
    ap.add_argument("--rates-compare", action="store_true",
                    help="instead of the step: time the production-rate kernel, sparse FP64 FMA "
                         "against FP64 tensor cores, on the workload's initial state")
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
    from paper_1801_01201_gb300.solver import Solver
    if args.pde > 0:
        return pde_bench(args, dev, rank)

    name = args.workload
    entries, w = entries_for(name, args.grid)
    if args.rates_compare:
        return rates_compare(entries, args, dev, rank)
    if args.diffusion_compare > 0:
        return diffusion_compare(entries, args, dev, rank)
    if args.nu_compare:
        return nu_compare(entries, w, args, dev, rank)
    if args.concurrency > 0:
        return concurrency_compare(entries, w, args, dev, rank)
    tune = (len(entries) > 1) if args.autotune < 0 else bool(args.autotune)
    stream = torch.cuda.current_stream()
    peaks = measure_fp_peaks(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # plain FP64 sweep
    plain = Runner(entries, w, args, dev, "fp64", tune=tune)
    r_plain = timed(plain, args, flush, stream, dist)
    variants = {"fp64": (plain, r_plain)}
    # mixed precision
    if args.headline in ("mixed", "learned_mixed"):
        mixed = Runner(entries, w, args, dev, "mixed", tune=tune)
        variants["mixed"] = (mixed, timed(mixed, args, flush, stream, dist))
    # learned + mixed: train one network per mechanism, then time
    train_info = None
    if args.headline == "learned_mixed":
        params, train_info = {}, {}
        for mech, fl, dt in entries:
            if id(mech) not in params:
                p, info = train_params(Solver, mech, fl, dt, w, dev, args)
                params[id(mech)] = p
                train_info["%d/%d" % (mech.n_species, mech.n_reactions)] = info
        lm = Runner(entries, w, args, dev, "mixed", params=params, tune=tune)
        variants["learned_mixed"] = (lm, timed(lm, args, flush, stream, dist))
    head, r_head = variants[args.headline]
    # the headline again with the clock sampler running (its own timed region)
    clocks = ClockSampler(local) if rank == 0 else None
    head.reset()
    r_head = timed(head, args, flush, stream, dist, clocks, label="headline")
    cells = head.cells
    value = whole_job_rate(world, cells, args.steps, r_head["total_ms"])

    # accuracy of each variant against the FP64 sweep after the same steps
    errs = {}
    for k, (rn, _) in variants.items():
        if k == "fp64":
            continue
        errs[k] = [field_errors(rn.solvers[i], rn.states[i], plain.states[i]) for i in range(len(entries))]
        errs[k] = {f: max(e[f] for e in errs[k]) for f in ("Y", "Y_species_worst", "h", "T")}

    # end to end through the host-buffer entry point (single-flame workloads)
    e2e = None
    if len(entries) == 1:
        sv = head.solvers[0]
        host = head.states0[0].cpu().pin_memory()
        tms = []
        for _ in range(args.e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sv.step_host(host, head.dts[0], 1)
            tms.append(time.perf_counter() - t0)
        nbytes = head.states0[0].numel() * 8
        e2e = {"value": world * cells * len(tms) / sum(tms) if tms else None, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    else:
        # batches: copy every flame's state in and out around the device step
        hosts = [x.cpu().pin_memory() for x in head.states0]
        tms = []
        for _ in range(args.e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for h, d in zip(hosts, head.states):
                d.copy_(h, non_blocking=True)
            head.step()
            for h, d in zip(hosts, head.states):
                h.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
            tms.append(time.perf_counter() - t0)
        nbytes = sum(x.numel() * 8 for x in head.states0)
        e2e = {"value": world * cells * len(tms) / sum(tms) if tms else None, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # batches: the same variant with one reaction launch per flame and stage (the
    # reaction steps not grouped across flames), its own timed region
    batch_forms = None
    if head.batch is not None:
        gl, gs = head.batch.grouping()
        head.batch.set_grouping(False)
        head.reset()
        r_sep = timed(head, args, flush, stream, dist, label="separate")
        head.batch.set_grouping(True)
        batch_forms = {
            "grouped": {"value": value, "grouped_newton_launches_per_step": gl,
                        "flame_reaction_steps_grouped_per_step": gs,
                        "kernel_launches_per_step": r_head["stats"]["kernel_launches"] / args.steps},
            "separate": {"value": whole_job_rate(world, cells, args.steps, r_sep["total_ms"]),
                         "kernel_launches_per_step": r_sep["stats"]["kernel_launches"] / args.steps,
                         "status": r_sep["stats"]["status_name"]}}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    st = r_head["stats"]
    roofline = None
    if len(entries) == 1 and r_head["newton_launches"]:
        mech = entries[0][0]
        nnz = int(np.count_nonzero(mech.nu_r - mech.nu_f))
        mixedk = args.headline != "fp64"
        launches = r_head["newton_launches"]
        avg_s = r_head["newton_ms"] / 1e3 / launches
        flops, counters = newton_flops_counted(mech.n_species, mech.n_reactions, mean_molecules(mech), st, mixedk)
        achieved = flops / launches / avg_s / 1e12
        kflops, exps = newton_flops(mech.n_species, mech.n_reactions, nnz, st, mixedk)
        kach = kflops / launches / avg_s / 1e12
        peak = peaks["dfma"]
        kname = ("reaction step: k_certify + k_chord (thread per cell) + k_newton2<mixed> (warp per cell)"
                 if mixedk else "k_newton2<fp64> (reaction Newton, warp per cell)")
        roofline = {"kernel": kname,
                    "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": NEWTON_TRAFFIC_BYTES.get((name, args.headline)),
                    "peak_source": "measured: FP64 FMA probe over every SM (misdc_probe_flops), of measured",
                    "flops_counted": "per cell-iteration: thermo 15N, rates R(10+4 nubar), Jacobian 2R nubar^2, "
                                     "LU 2n^3/3, solve 2n^2; counters of the timed steps",
                    "counters": counters, "launches": launches,
                    "flops_per_launch": flops / launches,
                    "kernel_instruction_model": {"achieved": kach, "frac": kach / peak,
                                                 "flops_per_launch": kflops / launches},
                    "newton_ms_per_step": r_head["newton_ms"] / args.steps,
                    "diffusion_ms_per_step": r_head["diffusion_ms"] / args.steps,
                    "newton_launch_ms": avg_s * 1e3,
                    "exp_log_calls_per_launch": exps / launches,
                    "newton_floor_stops": st["newton_floor_stops"],
                    "newton_jacobians_per_solve": st["newton_jacobians"] / max(st["newton_solves"], 1)}
    cpu = None
    if not args.no_cpu_baseline:
        try:
            r, el, c, desc = cpu_oracle_rate(name, args.cpu_side, 1)
            cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "one time step of a %s (%.1f s)" % (desc, el)}
        except Exception as e:   # the baseline is informative, never fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: %s" % e}

    def summary(k):
        rn, r = variants[k]
        s_ = r["stats"]
        d = {"value": whole_job_rate(world, rn.cells, args.steps, r["total_ms"]), "unit": UNIT,
             "ms_per_step": r["total_ms"] / args.steps,
             "newton_iters_per_solve": s_["newton_iters"] / max(s_["newton_solves"], 1),
             "status": s_["status_name"], "lin_resid_max": s_["lin_resid_max"]}
        if r["newton_launches"]:
            d["newton_ms_per_step"] = r["newton_ms"] / args.steps
        ns = max(s_["newton_solves"], 1)
        d["newton_jacobians_per_solve"] = s_["newton_jacobians"] / ns
        d["newton_certified_per_solve"] = s_["newton_certified"] / ns
        d["newton_stored_steps_per_solve"] = s_["newton_stored_steps"] / ns
        d["newton_chord_cells_per_solve"] = s_.get("newton_chord_cells", 0) / ns
        if k == "learned_mixed":
            d["surrogate_used"] = s_["surrogate_used"]
            d["surrogate_rejected"] = s_["surrogate_rejected"]
        if k in errs:
            d["rel_err_vs_fp64"] = errs[k]
        return d

    dtype = {"fp64": "f64", "mixed": "f64+f32", "learned_mixed": "f64+f32, bf16 MLP"}[args.headline]
    cfg = {"workload": name if not args.grid else "%s at %d cells per side" % (name, args.grid),
           "flames": len(entries), "cells": cells, "nodes": w["nodes"],
           "sweeps": w["sweeps"], "nu": w["nu"], "scheme": args.scheme, "variant": args.headline,
           "autotuned": tune, "l2": "flushed between steps (256 MB write)",
           "run": "%d-step runs from the initial state, repeated (restart copy inside the timed region)"
                  % w["steps"],
           "learned_sweeps": args.sg_sweeps or w["sweeps"], "lin_rounds": sorted({lin_rounds_for(args, fl) or 3 for _, fl, _ in entries}),
           "rates": "fp64 tensor cores" if args.rates_mma else "sparse fp64 fma",
           "diffusion": "multigrid %d levels" % args.mg_levels if args.mg_levels > 1 else "chebyshev"}
    if len(entries) == 1:
        mech, fl, dt = entries[0]
        cfg.update({"grid": [fl.nx, fl.ny, fl.nz], "species": mech.n_species,
                    "reactions": mech.n_reactions, "dt": dt})
    else:
        cfg["mechanisms"] = sorted({"%d/%d" % (m.n_species, m.n_reactions) for m, _, _ in entries})
    # the state the errors are taken on: steps since the run's start, smallest mass fraction
    cfg["compared_after_steps"] = plain.taken
    cfg["Y_min"] = min(float(x[:m.n_species].min().item()) for x, (m, _, _) in zip(head.states, entries))
    acc_ok = None
    if args.headline in errs:
        e = errs[args.headline]
        acc_ok = e["Y"] <= 1e-8 and e["T"] <= 1e-6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r_head["total_ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": cfg, "clocks": r_head["clocks"],
            "gpu_launches": st["kernel_launches"], "e2e": e2e, "roofline": roofline,
            "cpu_baseline": cpu, "status": st["status_name"],
            "measured_peaks_tflops": {k: v for k, v in peaks.items()},
            "accuracy_vs_fp64_ok": acc_ok,
            "variants": {k: summary(k) for k in variants},
            "speedup_vs_plain_fp64": value / summary("fp64")["value"] / world}
    if train_info:
        line["training"] = train_info
    if batch_forms:
        line["batch_forms"] = batch_forms
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
