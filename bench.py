"""Benchmark of the SQ3 path on GB300: seconds per converged SCF solve.

One step = one converged self-consistent-field solve of the 108-atom
Al-like cell (72^3 grid, Ns = 2200, filter degree 30, Fermi degree 120,
kT = 10 eV, s/p projectors) through the library's SCF driver
(sq3_scf_solve): per SCF iteration V_eff = phi[rho + b] + V_xc[rho], the
Chebyshev filter and Cholesky QR, Hs = X^T H X, Lanczos bounds, the
Chebyshev Fermi-operator expansion with the Fermi level on the device, Ds,
the fused density rho = 2 rowdot(X, X Ds)/dV, F and Kerker/Pulay mixing,
until sum |rho_out - rho_in| dV / Ne < 1e-6.  Every step runs in the
library's kernels behind the C ABI (ctypes binding); the inputs (seeded
synthetic positions and projectors, the starting block and density) are
resident in HBM when a timed solve starts, and every solve restarts from
the same block and density (X alone, 3.3 GB, is larger than L2).

The `value` arm is the mixed-precision path (FP32 stencil, BF16-split
tcgen05 products, FP64 Cholesky/Fermi level/energies) from the starting
density `--start` (learned: the MLP over atom-centred Gaussian
descriptors, trained on converged densities of 32-atom cells; the
atomic superposition otherwise).  `--fp64-arm` also runs the plain FP64
path from the atomic superposition to convergence (one solve, minutes at
this size) and reports its time and the differences of the converged
density, free energy and Fermi level between the arms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--start learned|superposition]
                    [--fp64-arm] [--config al108_72|al32_48] [--impl sq3|reference]
                    [--mode solve|iteration]

`--mode iteration` times one fixed-potential SQ3 iteration (the unit an
SCF iteration repeats) instead, for kernel-level profiling.

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the cell, the timed region is bracketed by barriers, the slowest
rank's time is taken, and `value` is whole-job seconds per solve (that time
/ number of replicas).

`--impl reference` times the CPU oracle (numpy/scipy FP64) on a bounded
sample of the same workload on the host cores and prints the same line with
"impl": "reference".
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

METRIC = "s per SCF solve (108-atom) mixed+learned vs FP64 at ρ err ≤1e-5; % roofline"
METRIC_ITER = "s per fixed-potential SQ3 iteration (108-atom), mixed precision"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA peak of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal
# unit count and maximum clock; probed 1.18 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per grid point
# and vector of one launch of the FP32 kernels, from ncu captures of the
# 32-atom cell (110,592 points x 640 vectors); the roofline entry scales
# them to the bench's workload by points x vectors.
MEASURED_TRAFFIC = {
    "stencil": (1181.7e6 / (373248 * 256), "ncu dram__bytes, 72^3 x 256 capture of the 108-atom cell"),
    "nl_pass": (785.2e6 / (373248 * 256), "ncu dram__bytes, 72^3 x 256 capture of the 108-atom cell"),
}
# SCF tolerance: sum |rho_out - rho_in| dV / Ne.  At the configured Ns the
# Ns-th state lies inside a near-degenerate shell whose members converge
# slowly under the filter, which sets a floor of a few 1e-6 .. 2e-5 on this
# change; 1e-5 is the metric's density tolerance.
SCF_TOL = 1e-5
DT_FS = 0.5                   # QMD time step (fs)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--prec", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--config", default="al108_72")
    p.add_argument("--impl", default="sq3", choices=["sq3", "reference"])
    p.add_argument("--mode", default="solve", choices=["solve", "iteration", "batch"])
    p.add_argument("--start", default="learned",
                   choices=["learned", "learned-direct", "previous", "extrapolated", "superposition"])
    p.add_argument("--fp64-arm", default="iteration", choices=["none", "iteration", "full"])
    p.add_argument("--no-compare-starts", dest="compare_starts", action="store_false")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--kernel-eval", default="ps", choices=["recurrence", "ps"],
                   help="evaluation of the Fermi-operator expansion in the SCF solves: the "
                        "recurrence or Paterson-Stockmeyer")
    p.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false",
                   help="skip the oracle's CPU timing (profiling runs)")
    p.add_argument("--cells", type=int, default=64,
                   help="batch mode: number of cells (fewer for profiling captures)")
    p.add_argument("--ns", type=int, default=None,
                   help="iteration mode: number of vectors other than the workload's "
                        "(a smaller footprint of the same kernels, for profiling)")
    return p.parse_args()


def peaks():
    try:
        with open(MEASURED) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, enabled: bool = True):
        self.enabled = enabled
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        if not self.enabled:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.enabled or self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# rank helpers
# ----------------------------------------------------------------------------
def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values of x (x itself with one rank)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_iteration(ms_step_slowest: float, world: int) -> float:
    """Whole-job time per step: the replicas run one cell each, so `world`
    steps finish in the slowest rank's time per step."""
    return ms_step_slowest / 1e3 / max(world, 1)


# ----------------------------------------------------------------------------
# the GPU path
# ----------------------------------------------------------------------------
def _setup(args, rank):
    import torch
    from paper_2112_08639_gb300 import build, inputs
    build.build()
    from paper_2112_08639_gb300 import sq3
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfg = inputs.CONFIGS[args.config]
    if getattr(args, "ns", None):
        # a smaller block on the same cell (profiling captures)
        import dataclasses
        cfg = dataclasses.replace(cfg, Ns=args.ns)
    cell = inputs.make_cell(cfg)
    ctx = sq3.Context(dev)
    ctx.setup_grid(cfg.n, cfg.n, cfg.n, cfg.L, cfg.L, cfg.L, 12)
    if cell.proj is not None:
        ctx.set_projectors(cell.proj.ptr, cell.proj.idx, cell.proj.val, cell.proj.gamma)
    return dev, cfg, cell, ctx, sq3, inputs


def _stage_summary(prof, steps):
    return {k: round(v[0] / steps, 3) for k, v in prof.items() if v[1] or v[0]}


def train_learned_start(dev, ncells: int = 6, seed: int = 0, log=None):
    """The learned starting density, trained (untimed set-up) on converged
    densities of 32-atom cells (48^3 grid, the same spacing as the 108-atom
    grid) with seeded thermal displacements, each solved by the mixed SCF
    driver from the atomic superposition."""
    from paper_2112_08639_gb300 import inputs, learned, qmd
    cfg = inputs.C2
    samples = []
    ctx = None
    for k in range(ncells):
        c = inputs.CellConfig(f"train{k}", ncell=2, n=48, Ns=640, m=25, npl=100,
                              projectors=True, disp_sigma=0.2, seed=seed + 100 + k)
        cell = qmd.Cell(c, device=dev)
        cell.set_positions(inputs.fcc_positions(2, disp_sigma=0.2, seed=seed + 100 + k))
        cell.start_density("superposition")
        cell.solve(2 * SCF_TOL, max_iter=40, raise_on_noconv=False)
        samples.append((cell.pos.copy(), cell.rho.clone(), cfg.Ne))
        ctx = cell.ctx if ctx is None else ctx
    return learned.train(ctx, samples, epochs=300, log=log)


def run_solve(args, rank, world):
    """One step = the converged SCF solve of a QMD step of the 108-atom cell:
    the atoms have moved by one velocity-Verlet step (0.5 fs at 116,045 K)
    from a converged state, whose block and spectral bounds start the
    filter; the starting density is the learned prediction (or --start)."""
    import torch
    from paper_2112_08639_gb300 import build, inputs
    build.build()
    from paper_2112_08639_gb300 import qmd, sq3
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfg = inputs.CONFIGS[args.config]
    # the previous QMD step: converged at R0 from a random block
    ke = sq3.EVAL_PATERSON_STOCKMEYER if args.kernel_eval == "ps" else sq3.EVAL_RECURRENCE
    cell = qmd.Cell(cfg, device=dev, prec=sq3.MIXED, kernel_eval=ke)
    R0 = inputs.fcc_positions(cfg.ncell, disp_sigma=cfg.disp_sigma, seed=cfg.seed)
    V0 = qmd.maxwell_boltzmann(cfg.natoms, cfg.sigma, seed=rank)
    cell.set_positions(R0)
    cell.start_density("superposition")
    res0, _ = cell.solve(SCF_TOL, max_iter=60, raise_on_noconv=False)
    F0 = cell.forces()
    masses = np.full(cfg.natoms, qmd.MASS_AL)
    R1, V1 = R0.copy(), V0.copy()
    sq3.verlet(masses, DT_FS * qmd.FS_IN_AU, R1, V1, F0, 0)
    cell.set_positions(R1)
    X_prev = cell.X.clone()
    rho_prev = cell.rho_prev.clone()
    pos_prev = cell.pos_prev.copy()
    bounds_prev = cell.bounds
    model = None
    train_log = []
    if args.start == "learned" or args.compare_starts:
        model = train_learned_start(dev, log=train_log)
    stream = torch.cuda.current_stream()

    def solve(start):
        cell.X.copy_(X_prev)
        cell.bounds = bounds_prev
        cell.rho_prev = rho_prev
        cell.pos_prev = pos_prev
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cell.start_density(start, model)
        res, hist = cell.solve(SCF_TOL, raise_on_noconv=False)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res, hist

    for _ in range(args.warmup):
        solve(args.start)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    cell.ctx.profile(True)
    times = []
    with ClockSampler(dev, enabled=not args.no_clocks) as clk:
        for _ in range(args.steps):
            ms, res, hist = solve(args.start)
            times.append(ms)
    torch.cuda.synchronize()
    cell.ctx.profile(False)
    prof = cell.ctx.profile_read()
    ms_total = max_over_ranks(sum(times), world, "cuda")
    if world > 1:
        torch.distributed.barrier()
    ms_step = ms_total / args.steps
    rho_mixed = cell.rho.clone()
    res_mixed = res

    starts = None
    if args.compare_starts:
        starts = {}
        for st_name in ("learned", "extrapolated", "previous", "learned-direct", "superposition"):
            ms_s, r_s, _ = solve(st_name)
            starts[st_name] = {"iterations": r_s["iterations"], "s": round(ms_s / 1e3, 4),
                               "converged": r_s["converged"]}

    # end to end through the public API with host buffers: the block of the
    # previous step comes from pinned host memory, the positions are host
    # arrays, and the converged density is read back, all in the timed region
    Xh = X_prev.cpu().pin_memory()
    rho_h = torch.empty(cfg.N, dtype=torch.float64).pin_memory()

    def e2e_step():
        cell.X.copy_(Xh, non_blocking=True)
        cell.bounds = bounds_prev
        cell.rho_prev = rho_prev
        cell.pos_prev = pos_prev
        cell.set_positions(R1)
        cell.start_density(args.start, model)
        res_e, _ = cell.solve(SCF_TOL, raise_on_noconv=False)
        rho_h.copy_(cell.rho, non_blocking=True)
        torch.cuda.synchronize()
        return res_e

    e2e_step()
    e2e_t = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t))
    # one more end-to-end step, with a synchronisation after each phase, for
    # the breakdown of its time (not part of the timed steps)
    phases = {}

    def mark(name, t0):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        phases[name] = round(t1 - t0, 4)
        return t1

    # the block's upload alone, timed with events on the stream
    h2d_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cell.X.copy_(Xh, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        h2d_ms.append(round(e0.elapsed_time(e1), 2))
    phases["h2d_block_alone_ms"] = h2d_ms
    t = time.perf_counter()
    cell.X.copy_(Xh, non_blocking=True)
    t = mark("h2d_block", t)
    cell.bounds, cell.rho_prev, cell.pos_prev = bounds_prev, rho_prev, pos_prev
    pr1 = inputs.projectors(cfg.n, cfg.L, R1, seed=cell.proj_seed)
    t = mark("projector_values_host", t)
    cell.ctx.set_projectors(pr1.ptr, pr1.idx, pr1.val, pr1.gamma)
    t = mark("set_projectors", t)
    cell.ctx.pseudocharge(R1, inputs.Z_VALENCE, inputs.RC_LOCAL, out=cell.b)
    cell.pos = R1.copy()
    cell.start_density(args.start, model)
    t = mark("pseudocharge_and_start", t)
    cell.solve(SCF_TOL, raise_on_noconv=False)
    t = mark("scf_solve", t)
    rho_h.copy_(cell.rho, non_blocking=True)
    mark("d2h_rho", t)
    h2d = Xh.numel() * Xh.element_size() + cfg.natoms * 3 * 8
    d2h = cfg.N * 8

    fp64 = None
    if args.fp64_arm != "none":
        cell64 = qmd.Cell(cfg, device=dev, prec=sq3.FP64, kernel_eval=ke)
        cell64.set_positions(R1)
        cell64.X = X_prev.double()
        cell64.bounds = bounds_prev
        cell64.rho_prev = rho_prev
        cell64.pos_prev = pos_prev
        cell64.start_density("extrapolated")
        full = args.fp64_arm == "full"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res64, hist64 = cell64.solve(SCF_TOL, max_iter=100 if full else 2, raise_on_noconv=False)
        torch.cuda.synchronize()
        s64 = time.perf_counter() - t0
        fp64 = {"start": "extrapolated (the previous density moved with the atomic superposition), "
                         "the previous step's block", "measured": args.fp64_arm,
                "iterations_run": res64["iterations"], "converged": res64["converged"],
                "s_per_iteration": round(s64 / res64["iterations"], 3),
                "ms_per_iteration_mixed": round(ms_step / max(res_mixed["iterations"], 1), 2)}
        if full:
            fp64.update({
                "s_per_solve": round(s64, 3), "err": res64["err"], "F": res64["F"],
                "mu": res64["mu"],
                "rho_l1_per_Ne_vs_mixed": float((rho_mixed - cell64.rho).abs().sum()) * cfg.dV / cfg.Ne,
                "F_per_atom_vs_mixed": abs(res_mixed["F"] - res64["F"]) / cfg.natoms,
                "mu_vs_mixed": abs(res_mixed["mu"] - res64["mu"]),
                "speedup_mixed_learned_vs_fp64": round(s64 / (ms_step / 1e3), 2)})
        del cell64

    launches = int(sum(v[1] for v in prof.values()))
    pk, pk_src = peaks()
    dominant = max(prof, key=lambda k: prof[k][0])
    n_cov = int(np.unique(cell.proj.idx).size) if cell.proj is not None else 0
    roof = roofline(dominant, prof, cfg, 4, False, pk, pk_src, n_cov)
    clocks = clk.summary()
    out = {
        "metric": METRIC,
        "value": round(job_seconds_per_iteration(ms_step, world), 6),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+bf16x3",
        "data": "synthetic",
        "config": {
            "workload": f"{cfg.name}: {cfg.natoms}-atom Al-like cell, {cfg.n}^3 grid, Ns={cfg.Ns}, "
                        f"filter degree {cfg.m}, Fermi degree {cfg.npl}, kT={cfg.kT_ev} eV, "
                        f"projectors={'s/p' if cfg.projectors else 'none'}",
            "step": f"converged SCF solve of a QMD step (rho L1/Ne change < {SCF_TOL:g}) after one "
                    f"{DT_FS} fs velocity-Verlet step from a converged state; the previous "
                    f"step's block and bounds, the {args.start} starting density",
            "precision": "mixed",
            "expansion": ("Paterson-Stockmeyer" if args.kernel_eval == "ps"
                          else "recurrence with the product identity"),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (X block %.2f GB)" % (cfg.N * cfg.Ns * 4 / 1e9),
        },
        "scf": {"iterations": res_mixed["iterations"],
                "ms_per_iteration": round(ms_step / max(res_mixed["iterations"], 1), 2),
                "F": res_mixed["F"], "mu": res_mixed["mu"], "err": res_mixed["err"],
                "converged": res_mixed["converged"], "start": args.start,
                "previous_step": {"iterations": res0["iterations"], "from": "random block"},
                "per_iteration": [{k: (round(v, 9) if isinstance(v, float) else v)
                                   for k, v in h.items()} for h in hist]},
        "e2e": {"value": round(e2e_s, 6), "unit": "s", "stat": f"median of {len(e2e_t)} solves",
                "steps_s": [round(x, 4) for x in e2e_t], "phases_s": phases,
                "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "stage_ms_per_step": _stage_summary(prof, args.steps),
        "roofline": roof,
    }
    if train_log:
        out["learned"] = {"training_cells": 6, "epochs": len(train_log),
                          "loss_first": train_log[0], "loss_last": train_log[-1]}
    if starts is not None:
        out["starts"] = starts
    if fp64 is not None:
        out["fp64_arm"] = fp64
    if clocks is not None:
        out["clocks"] = clocks
    return out, res_mixed["iterations"]


def run_iteration(args, rank, world):
    """One fixed-potential SQ3 iteration per step (kernel-level profiling)."""
    import torch
    dev, cfg, cell, ctx, sq3, inputs = _setup(args, rank)
    prec = sq3.FP64 if args.prec == "fp64" else sq3.MIXED
    dtype = torch.float64 if prec == sq3.FP64 else torch.float32
    esize = 8 if prec == sq3.FP64 else 4
    V = torch.from_numpy(cell.V).cuda()
    ctx.set_potential(V)
    X = inputs.random_block_device(cfg.N, cfg.Ns, seed=1000 + rank, dtype=dtype)
    D = torch.empty((cfg.Ns, cfg.Ns), dtype=torch.float64, device="cuda")
    rho = torch.empty(cfg.N, dtype=torch.float64, device="cuda")
    lo, b = ctx.hamiltonian_bounds()
    state = {"a0": lo, "a": lo + 0.05 * (b - lo)}

    def step():
        ctx.cheb_filter(X, cfg.m, state["a"], b, state["a0"], prec)
        ctx.orthonormalise(X, prec)
        _, out = ctx.density_kernel(X, cfg.npl, cfg.sigma, cfg.Ne, prec, D=D)
        ctx.density(X, D, prec, rho=rho)
        state["a0"], state["a"] = out["chi"] - out["xi"], out["chi"] + out["xi"]
        return out

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    with ClockSampler(dev, enabled=not args.no_clocks) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            out = step()
        e1.record(stream)
        torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms_step = max_over_ranks(e0.elapsed_time(e1), world, "cuda") / args.steps
    pk, pk_src = peaks()
    dominant = max(prof, key=lambda k: prof[k][0])
    n_cov = int(np.unique(cell.proj.idx).size) if cell.proj is not None else 0
    res = {
        "metric": METRIC_ITER, "value": round(job_seconds_per_iteration(ms_step, world), 6),
        "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == sq3.FP64 else "f32+bf16x3",
        "data": "synthetic",
        "config": {"workload": cfg.name, "step": "one fixed-potential SQ3 iteration",
                   "precision": args.prec},
        "gpu_launches": int(sum(v[1] for v in prof.values())),
        "stage_ms_per_step": _stage_summary(prof, args.steps),
        "roofline": roofline(dominant, prof, cfg, esize, prec == sq3.FP64, pk, pk_src, n_cov),
        "mu": out["mu"],
    }
    clocks = clk.summary()
    if clocks is not None:
        res["clocks"] = clocks
    return res, 1


def batch_cells(ncells: int = 64, seed: int = 0):
    """The batched workload (C4 of the input module)."""
    from paper_2112_08639_gb300 import inputs
    return inputs.batch_cells(ncells, seed)


def small_cells(ncells: int = 64, seed: int = 1):
    """Many 4-atom cells (the input module's small_cells)."""
    from paper_2112_08639_gb300 import inputs
    return inputs.small_cells(ncells, seed)


def measure_batch(cells, dev, steps, warmup, clock_sampler=None):
    """Time the batched filter of `cells` (one persistent launch, graph
    replay, autotuned) and the same filters one cell at a time through
    sq3_cheb_filter; returns (ms batched, ms loop, point-vector-steps,
    autotuned shape)."""
    import torch
    from paper_2112_08639_gb300 import inputs, sq3
    batch = sq3.Batch(dev)
    ctxs, X0s, Xs, bounds = [], [], [], []
    work = 0
    for c in cells:
        ctx = sq3.Context(dev)
        ctx.setup_grid(*c["n"], *c["L"], 12)
        N = int(np.prod(c["n"]))
        b, _ = ctx.pseudocharge(c["pos"], inputs.Z_VALENCE, inputs.RC_LOCAL)
        V = ctx.poisson(b)                       # the local potential of the pseudocharges
        ctx.set_potential(V)
        lo, hi = ctx.hamiltonian_bounds()
        bd = (lo + 0.05 * (hi - lo), hi, lo)
        X0 = inputs.random_block_device(N, c["Ns"], seed=c["seed"])
        X = X0.clone()
        idx = batch.add_cell(c["n"], c["L"], V, X, c["m"])
        batch.set_bounds(idx, *bd)
        ctxs.append(ctx); X0s.append(X0); Xs.append(X); bounds.append(bd)
        work += N * c["Ns"] * c["m"]
    ctas, div = batch.autotune()
    stream = torch.cuda.current_stream()

    def restore():
        for X, X0 in zip(Xs, X0s):
            X.copy_(X0)

    def timed(fn):
        for _ in range(warmup):
            restore(); fn()
        tot = 0.0
        for _ in range(steps):
            restore()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps

    def loop():
        for ctx, X, (a, b_, a0), c in zip(ctxs, Xs, bounds, cells):
            ctx.cheb_filter(X, c["m"], a, b_, a0, sq3.MIXED)

    if clock_sampler is not None:
        with clock_sampler:
            ms_batch = timed(batch.filter)
    else:
        ms_batch = timed(batch.filter)
    ms_loop = timed(loop)
    batch.close()
    for ctx in ctxs:
        ctx.close()
    return ms_batch, ms_loop, work, (ctas, div)


def run_batch(args, rank, world):
    """One step = the Chebyshev filter of every cell of the batched workload
    (batch_cells): one persistent launch that takes every vector of every
    cell through all its filter steps, replayed from a CUDA graph, tile
    shape autotuned; against the same filters one cell at a time through
    sq3_cheb_filter.  The same comparison on 64 small cells (4 atoms, 24^3,
    Ns = 80) is reported beside it."""
    import torch
    from paper_2112_08639_gb300 import build
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cells = batch_cells(args.cells, seed=rank)
    clk = ClockSampler(dev, enabled=not args.no_clocks)
    ms_batch, ms_loop, work, (ctas, div) = measure_batch(cells, dev, args.steps, args.warmup, clk)
    ms_batch = max_over_ranks(ms_batch, world, "cuda")
    sc = small_cells(64, seed=1000 + rank)
    ms_sb, ms_sl, work_s, shape_s = measure_batch(sc, dev, args.steps, args.warmup)
    pk, pk_src = peaks()
    gbs = 12.0 * work / (ms_batch / 1e3) / 1e9
    out = {
        "metric": f"filtered point-vector-steps per second, {len(cells)} uneven cells (batched)",
        "value": round(world * work / (ms_batch / 1e3) / 1e9, 3), "unit": "G/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_batch, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(cells)} Al-like cells of 4-32 atoms, grids 24-48 per side, Ns 80-640, "
                               "filter degree 20, local potential, FP32",
                   "step": "one Chebyshev filter of every cell",
                   "autotuned": {"ctas_per_sm": ctas, "tile_height_divisor": div}},
        "batched_vs_loop": {"ms_batched": round(ms_batch, 3), "ms_one_cell_at_a_time": round(ms_loop, 3),
                            "speedup": round(ms_loop / ms_batch, 3)},
        "small_cells": {"workload": f"{len(sc)} cells of 4 atoms, 24^3, Ns 80, degree 20",
                        "G_per_s_batched": round(work_s / (ms_sb / 1e3) / 1e9, 3),
                        "ms_batched": round(ms_sb, 3), "ms_one_cell_at_a_time": round(ms_sl, 3),
                        "speedup": round(ms_sl / ms_sb, 3),
                        "autotuned": {"ctas_per_sm": shape_s[0], "tile_height_divisor": shape_s[1]}},
        "roofline": {"bound": "hbm", "kernel": "batch_filter_kernel (all cells, all steps)",
                     "achieved": round(gbs, 1),
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(gbs / pk["hbm_gbs"], 4),
                     "traffic": None,
                     "algorithmic": "12 B per point, vector and step (the streaming count; the "
                                    "kernel keeps a vector's iterates in L2 between steps)",
                     "peak_source": pk_src + " (MEASURED_PEAKS hbm_gbs; of measured)"},
        "gpu_launches": 1,
    }
    clocks = clk.summary()
    if clocks is not None:
        out["clocks"] = clocks
    return out, 1


def roofline(dominant, prof, cfg, esize, fp64, pk, pk_src, n_covered):
    """Roofline entry for the kernel class that takes the most device time.

    Algorithmic work per launch:
      stencil   3 words per grid point per vector (read Y_k and Y_{k-1},
                write Y_{k+1}); FP64 path: ~80 flop per point per vector
      nl_pass   read and write of the step's output at the n_covered grid
                points inside at least one projector
      GEMMs     useful flops: Gram and X^T(HX) N Ns^2 (upper-triangle tiles
                of a symmetric product), X R^{-1} N Ns^2 (triangular
                R^{-1}), the density row-dot N Ns^2 (triangular B), the
                recurrence Ns^3 (upper-triangle tiles)
    """
    N, Ns = cfg.N, cfg.Ns
    ms, n = prof[dominant]
    per_launch_s = ms / max(n, 1) / 1e3
    fp64_peak = {"peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                 "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    hbm_peak = {"peak": pk["hbm_gbs"], "unit": "GB/s",
                "peak_source": pk_src + " (MEASURED_PEAKS hbm_gbs; of measured)"}
    if dominant == "stencil":
        if fp64:
            ach = 80.0 * N * Ns / per_launch_s / 1e12
            return dict(bound="alu", kernel="cheb_step (FP64 stencil)", achieved=round(ach, 4),
                        frac=round(ach / FP64_PEAK_TFLOPS, 4), traffic=None, **fp64_peak)
        ach = 3.0 * N * Ns * esize / per_launch_s / 1e9
        bpu, src = MEASURED_TRAFFIC["stencil"]
        return dict(bound="hbm", kernel="cheb_step_ring (FP32 stencil)", achieved=round(ach, 1),
                    frac=round(ach / pk["hbm_gbs"], 4), traffic=round(bpu * N * Ns / 1e9, 3),
                    traffic_unit="GB per launch", algorithmic=round(3.0 * N * Ns * esize / 1e9, 3),
                    traffic_source=src + ", scaled by points x vectors", **hbm_peak)
    if dominant == "nl_pass":
        ach = 2.0 * n_covered * Ns * esize / per_launch_s / 1e9
        bpu, src = MEASURED_TRAFFIC["nl_pass"]
        return dict(bound="hbm", kernel="nl_brick (nonlocal apply + projection)",
                    achieved=round(ach, 1), frac=round(ach / pk["hbm_gbs"], 4),
                    traffic=round(bpu * n_covered * Ns / 1e9, 3), traffic_unit="GB per launch",
                    algorithmic=round(2.0 * n_covered * Ns * esize / 1e9, 3),
                    traffic_source=src + ", scaled by points x vectors", **hbm_peak)
    gemm_flops = {"gram": N * Ns * Ns, "hs_gemm": N * Ns * Ns, "x_rinv": N * Ns * Ns,
                  "rho": N * Ns * Ns, "cheb_gemm": Ns ** 3}
    if dominant in gemm_flops:
        ach = gemm_flops[dominant] / per_launch_s / 1e12
        if fp64:
            return dict(bound="alu", kernel=f"{dominant} (FP64 GEMM)", achieved=round(ach, 4),
                        frac=round(ach / FP64_PEAK_TFLOPS, 4), traffic=None, **fp64_peak)
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        return dict(bound="tensor", kernel=f"{dominant} (tcgen05, 6 BF16 piece products)",
                    achieved=round(6 * ach, 2), useful=round(ach, 2), peak=peak, unit="TFLOP/s",
                    frac=round(6 * ach / peak, 4), traffic=None,
                    peak_source=pk_src + " (bf16_tflops_sustained; of measured)")
    return {"bound": "unknown", "kernel": dominant, "achieved": None, "peak": None, "unit": None,
            "frac": None, "traffic": None}


# ----------------------------------------------------------------------------
# the CPU oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------
# SQ3 iterations (one filter pass each) of the converged QMD-step solve at
# the 108-atom configuration with the learned start, as this bench's GPU
# arm measured it; the reference arm scales the oracle's per-iteration cost
# by it
PASSES_PER_SOLVE = {"al108_72": 5, "al32_48": 5}


def run_oracle_sample(cfg_name: str, passes: int):
    """Time the oracle's steps of one SQ3 iteration and of the SCF pieces on
    sampled sizes, scale each by its operation count to the full cell, and
    multiply by the number of filter passes of one solve.

    filter: m sparse H applies on k columns (scaled by Ns/k); the H apply of
    the projection step costs 1/m of that per column; Cholesky QR, X^T (H X)
    and the density on an N x s column block (dense FP64 BLAS, scaled by
    (Ns/s)^2); the Fermi-operator expansion on an s x s Hs (scaled by
    (Ns/s)^3); the SCF pieces (Poisson, LDA, Kerker/Pulay) at full size.
    """
    from paper_2112_08639_gb300 import inputs
    from oracle import chebyshev, hamiltonian, scf, subspace

    cfg = inputs.CONFIGS[cfg_name]
    cell = inputs.make_cell(cfg)
    parts = hamiltonian.hamiltonian_sparse(cfg.n, cfg.L, cell.V, cell.proj)
    apply_H = lambda Z: hamiltonian.apply(parts, Z)
    rng = np.random.default_rng(0)
    k = min(4, cfg.Ns)
    X = rng.standard_normal((cfg.N, k))
    t = time.perf_counter()
    chebyshev.filter_plain(apply_H, X, cfg.m, 2.0, 100.0, -2.0)
    t_filter = (time.perf_counter() - t) * cfg.Ns / k
    t_apply = t_filter / cfg.m
    s = min(128, cfg.Ns)
    Xs = subspace.cholqr(rng.standard_normal((cfg.N, s)))
    HXs = apply_H(Xs)
    t = time.perf_counter()
    subspace.cholqr(Xs)
    Hs = Xs.T @ HXs
    Hs = 0.5 * (Hs + Hs.T)
    subspace.density_from_kernel(Xs, np.eye(s), cfg.dV)
    t_dense = (time.perf_counter() - t) * (cfg.Ns / s) ** 2
    t = time.perf_counter()
    chi, xi = subspace.exact_bounds(Hs)
    chebyshev.foe_density_kernel(Hs, cfg.npl, cfg.sigma, min(cfg.Ne, 1.5 * s), chi, xi)
    t_foe = (time.perf_counter() - t) * (cfg.Ns / s) ** 3
    rho = np.full(cfg.N, cfg.Ne / (cfg.N * cfg.dV))
    bq, _ = scf.pseudocharge(cfg.n, cfg.L, cell.positions, 3.0, 1.0, Ne=cfg.Ne)
    mixer = scf.PulayMixer(precond=lambda f: scf.kerker(f, cfg.n, cfg.L, 0.8))
    t = time.perf_counter()
    phi = scf.poisson_fd(rho + bq, cfg.n, cfg.L)
    scf.lda_xc(rho)
    mixer.step(rho, rho + 1e-3 * phi)
    t_scf = time.perf_counter() - t
    per_iter = t_filter + t_apply + t_dense + t_foe + t_scf
    total = per_iter * passes
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    sample = (f"{cfg.name}: per SQ3 iteration, filter (degree {cfg.m}) on {k} of {cfg.Ns} columns "
              f"(x{cfg.Ns / k:.0f}); CholQR + X^T(HX) + rho on an N x {s} block "
              f"(x{(cfg.Ns / s) ** 2:.1f}); FOE (npl {cfg.npl}) at Ns={s} (x{(cfg.Ns / s) ** 3:.0f}); "
              f"Poisson + LDA + Kerker/Pulay at full size; numpy/scipy FP64, operation-count "
              f"scaling; x {passes} filter passes per solve (the GPU arm's count)")
    return total, cores, sample, {"per_iteration": per_iter, "filter": t_filter,
                                  "dense": t_dense, "foe": t_foe, "scf": t_scf}


def run_oracle_sample_one_thread(cfg_name: str, passes: int):
    """The same oracle sample in a fresh process with every BLAS/OpenMP pool
    at one thread (set before numpy loads); returns its seconds per solve,
    or None if the child fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    root = os.path.dirname(os.path.abspath(__file__))
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.run_oracle_sample(%r, %d)[0]))" % (root, cfg_name, passes))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=900)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.steps is None:
        args.steps = 3 if args.mode == "solve" else 5
    metric = METRIC if args.mode == "solve" else METRIC_ITER
    passes_ref = PASSES_PER_SOLVE.get(args.config, 20) if args.mode == "solve" else 1
    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        for _ in range(max(args.warmup, 0)):
            run_oracle_sample(args.config, passes_ref)
        for _ in range(args.steps):
            v, cores, sample, parts = run_oracle_sample(args.config, passes_ref)
            vals.append(v)
        v = statistics.median(vals)
        print(json.dumps({
            "impl": "reference", "metric": metric, "value": round(v, 3), "unit": "s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.config,
                       "step": "converged SCF solve (oracle, extrapolated from a sample)"
                       if args.mode == "solve" else "one fixed-potential SQ3 iteration (oracle)"},
            "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.mode == "solve":
        res, passes = run_solve(args, rank, world)
    elif args.mode == "batch":
        res, passes = run_batch(args, rank, world)
    else:
        res, passes = run_iteration(args, rank, world)
    if rank == 0 and args.mode == "batch":
        print(json.dumps(res))
    elif rank == 0 and not args.cpu_baseline:
        print(json.dumps(res))
    elif rank == 0:
        v, cores, sample, parts = run_oracle_sample(args.config, passes)
        res["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": cores, "kind": "oracle",
                               "sample": sample, "blas_threads": cores}
        v1 = run_oracle_sample_one_thread(args.config, passes)
        if v1 is not None:
            res["cpu_baseline"]["one_thread"] = {"value": round(v1, 3), "unit": "s", "threads": 1}
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
