"""Benchmark of the SQ3 hot path on GB300.

One step = one fixed-potential SQ3 iteration of the 108-atom Al-like cell
(72^3 grid, Ns = 2200, filter degree 30, Fermi degree 120, s/p projectors):
Chebyshev filter, Cholesky-QR orthonormalisation, Hs = X^T H X, Lanczos
bounds, Chebyshev Fermi-operator expansion with the Fermi level found on
the device, Ds, and the fused density rho = 2 rowdot(X, X Ds)/dV.  Every step
runs through the C ABI of libsq3 (ctypes binding); inputs are seeded and
synthetic and resident in HBM when the timed region starts (X alone is
larger than L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|mixed]
                    [--config al108_72|al32_48|al4_18] [--impl sq3|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the cell (the single-cell path has no data-parallel exchange), the
timed region is bracketed by barriers, the slowest rank's time is taken, and
`value` is whole-job seconds per iteration (that time / number of replicas).

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
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA peak of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal
# unit count and maximum clock; probed 1.18 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per grid point
# and vector of one launch of the FP32 kernels, from the ncu captures
# summarised in profiles/ (32-atom cell: 110,592 points x 640 vectors); the
# roofline entry scales them to the bench's workload by points x vectors.
MEASURED_TRAFFIC = {
    "stencil": (831.3e6 / (110592 * 640), "profiles/cheb_step_ring_f32_al32_48.md"),
    "nl_pass": (533.1e6 / (110592 * 640), "profiles/nl_brick_f32_al32_48.md"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--prec", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--config", default="al108_72")
    p.add_argument("--impl", default="sq3", choices=["sq3", "reference"])
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-clocks", action="store_true")
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
# the GPU path
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
    """Whole-job time per iteration: the replicas run one cell each, so
    `world` iterations finish in the slowest rank's time per step."""
    return ms_step_slowest / 1e3 / max(world, 1)


def run_sq3(args, rank, world):
    import torch
    from paper_2112_08639_gb300 import build, inputs
    build.build()
    from paper_2112_08639_gb300 import sq3

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfg = inputs.CONFIGS[args.config]
    prec = sq3.FP64 if args.prec == "fp64" else sq3.MIXED
    dtype = torch.float64 if prec == sq3.FP64 else torch.float32
    esize = 8 if prec == sq3.FP64 else 4
    cell = inputs.make_cell(cfg)
    ctx = sq3.Context(dev)
    ctx.setup_grid(cfg.n, cfg.n, cfg.n, cfg.L, cfg.L, cfg.L, 12)
    V = torch.from_numpy(cell.V).cuda()
    ctx.set_potential(V)
    if cell.proj is not None:
        ctx.set_projectors(cell.proj.ptr, cell.proj.idx, cell.proj.val, cell.proj.gamma)
    gen = torch.Generator(device="cuda").manual_seed(1000 + rank)
    X = torch.randn((cfg.Ns, cfg.N), generator=gen, device="cuda", dtype=dtype)
    D = torch.empty((cfg.Ns, cfg.Ns), dtype=torch.float64, device="cuda")
    rho = torch.empty(cfg.N, dtype=torch.float64, device="cuda")

    # spectral bounds for the filter: upper bound b above the FD kinetic
    # maximum (1/2 * 3 * s_max / h^2, s_max = 7.0729 for 12th order) plus the
    # largest potential; damped interval [a, b]; a0 at the lower end.
    b = 0.5 * 3 * 7.0729 / cfg.h ** 2 + float(cell.V.max()) + (
        float(np.max(cell.proj.gamma)) * 4 if cell.proj is not None else 0.0)
    state = {"a0": float(cell.V.min()) - 1.0}
    state["a"] = state["a0"] + 0.05 * (b - state["a0"])

    def step(Xb, Xhost=None):
        if Xhost is None:
            ctx.cheb_filter(Xb, cfg.m, state["a"], b, state["a0"], prec)
        else:   # the block arrives from host memory, its upload overlapping the filter
            ctx.cheb_filter_from_host(Xhost, Xb, cfg.m, state["a"], b, state["a0"], prec)
        ctx.orthonormalise(Xb, prec)
        _, out = ctx.density_kernel(Xb, cfg.npl, cfg.sigma, cfg.Ne, prec, D=D)
        ctx.density(Xb, D, prec, rho=rho)
        state["a0"], state["a"] = out["chi"] - out["xi"], out["chi"] + out["xi"]
        return out

    for _ in range(args.warmup):
        step(X)
    stream = torch.cuda.current_stream()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    with ClockSampler(dev, enabled=not args.no_clocks) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            out = step(X)
        e1.record(stream)
        torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms_total = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    if world > 1:
        torch.distributed.barrier()
    ms_step = ms_total / args.steps

    # end to end through the public API with host buffers: the step's inputs
    # (V and the starting block X) copied from pinned host memory, the step,
    # and rho plus the scalars read back, all inside the timed region.  The
    # block goes up through the filter's host entry point, which copies it in
    # chunks of vectors and filters each chunk as soon as it has landed.
    Xh = X.cpu().pin_memory()
    Vh = V.cpu().pin_memory()
    rho_h = torch.empty(cfg.N, dtype=torch.float64).pin_memory()

    # every end-to-end step starts from the same host block and the same
    # filter bounds (the steps would otherwise alternate between two bound
    # settings, since each one restarts from that block)
    bounds0 = dict(state)

    def e2e_step():
        state.update(bounds0)
        V.copy_(Vh, non_blocking=True)
        ctx.set_potential(V)
        step(X, Xh)
        rho_h.copy_(rho, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()          # untimed: first use of the host buffers and the copy stream
    torch.cuda.synchronize()
    # each step timed on its own (wall clock, synchronised on both sides);
    # the median, so that one host-side hiccup does not set the figure
    e2e_t = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t))
    h2d = Xh.numel() * Xh.element_size() + Vh.numel() * 8
    d2h = cfg.N * 8 + 6 * 8

    launches = int(sum(v[1] for v in prof.values()))
    stage_ms = {k: round(v[0] / args.steps, 3) for k, v in prof.items() if v[1] or v[0]}
    pk, pk_src = peaks()
    dominant = max(prof, key=lambda k: prof[k][0])
    n_cov = int(np.unique(cell.proj.idx).size) if cell.proj is not None else 0
    roof = roofline(dominant, prof, cfg, esize, prec == sq3.FP64, pk, pk_src, args.steps, n_cov)
    clocks = clk.summary()
    res = {
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
        "dtype": "f64" if prec == sq3.FP64 else "f32+bf16x3",
        "data": "synthetic",
        "config": {
            "workload": f"{cfg.name}: {cfg.natoms}-atom Al-like cell, {cfg.n}^3 grid, Ns={cfg.Ns}, "
                        f"filter degree {cfg.m}, Fermi degree {cfg.npl}, kT={cfg.kT_ev} eV, "
                        f"projectors={'s/p' if cfg.projectors else 'none'}",
            "step": "one fixed-potential SQ3 iteration (filter, CholQR, Hs, Lanczos, FOE, Ds, rho)",
            "precision": args.prec,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (X block %.2f GB)" % (cfg.N * cfg.Ns * esize / 1e9),
        },
        "e2e": {"value": round(e2e_s, 6), "unit": "s", "stat": f"median of {len(e2e_t)} steps",
                "steps_s": [round(x, 6) for x in e2e_t], "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "stage_ms_per_step": stage_ms,
        "roofline": roof,
        "mu": out["mu"], "e_band": out["e_band"], "e_ent": out["e_ent"],
    }
    if clocks is not None:
        res["clocks"] = clocks
    return res


def roofline(dominant, prof, cfg, esize, fp64, pk, pk_src, steps, n_covered):
    """Roofline entry for the kernel class that takes the most device time.

    Algorithmic work per launch:
      stencil   3 words per grid point per vector (read Y_k and Y_{k-1},
                write Y_{k+1}); FP64 path: ~80 flop per point per vector
      nl_pass   read and write of the step's output at the n_covered grid
                points inside at least one projector
      GEMMs     useful flops: Gram and X^T(HX) N Ns^2 (upper triangle),
                X R^{-1} N Ns^2 (triangular), X Ds 2 N Ns^2, recurrence 2 Ns^3
    """
    N, Ns = cfg.N, cfg.Ns
    ms, n = prof[dominant]
    per_launch_s = ms / max(n, 1) / 1e3
    fp64_peak = {"peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                 "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    hbm_peak = {"peak": pk["hbm_gbs"], "unit": "GB/s", "peak_source": pk_src + " (MEASURED_PEAKS hbm_gbs)"}
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
    # useful flops per launch: symmetric outputs (Gram, Hs, the recurrence)
    # and triangular B (X R^-1, the density row-dot) count half a full product
    gemm_flops = {"gram": N * Ns * Ns, "hs_gemm": N * Ns * Ns, "x_rinv": N * Ns * Ns,
                  "rho": N * Ns * Ns, "cheb_gemm": Ns ** 3}
    if dominant in gemm_flops:
        ach = gemm_flops[dominant] / per_launch_s / 1e12
        if fp64:
            return dict(bound="alu", kernel=f"{dominant} (FP64 GEMM)", achieved=round(ach, 4),
                        frac=round(ach / FP64_PEAK_TFLOPS, 4), traffic=None, **fp64_peak)
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        # six BF16 piece products are issued per useful FP32-level product
        return dict(bound="tensor", kernel=f"{dominant} (tcgen05, 6 BF16 piece products)",
                    achieved=round(6 * ach, 2), useful=round(ach, 2), peak=peak, unit="TFLOP/s",
                    frac=round(6 * ach / peak, 4), traffic=None,
                    peak_source=pk_src + " (bf16_tflops_sustained)")
    return {"bound": "unknown", "kernel": dominant, "achieved": None, "peak": None, "unit": None,
            "frac": None, "traffic": None}


# ----------------------------------------------------------------------------
# the CPU oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------
def run_oracle_sample(cfg_name: str):
    """Time the oracle's steps of one SQ3 iteration on sampled sizes and scale
    each by its operation count to the full cell.

    filter: m sparse H applies on k columns (scaled by Ns/k); the H apply of
    the projection step costs 1/m of that per column; Cholesky QR, X^T (H X)
    and the density on an N x s column block (dense FP64 BLAS, scaled by
    (Ns/s)^2); the Fermi-operator expansion on an s x s Hs (scaled by
    (Ns/s)^3).
    """
    from paper_2112_08639_gb300 import inputs
    from oracle import chebyshev, hamiltonian, subspace

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
    total = t_filter + t_apply + t_dense + t_foe
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    sample = (f"{cfg.name}: filter (degree {cfg.m}) on {k} of {cfg.Ns} columns (x{cfg.Ns / k:.0f}); "
              f"CholQR + X^T(HX) + rho on an N x {s} block (x{(cfg.Ns / s) ** 2:.1f}); FOE (npl {cfg.npl}) "
              f"at Ns={s} (x{(cfg.Ns / s) ** 3:.0f}); numpy/scipy FP64, operation-count scaling")
    return total, cores, sample, {"filter": t_filter, "apply": t_apply, "dense": t_dense, "foe": t_foe}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.steps is None:
        args.steps = 1 if args.prec == "fp64" else 5
    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        for _ in range(max(args.warmup, 0)):
            run_oracle_sample(args.config)
        for _ in range(args.steps):
            v, cores, sample, parts = run_oracle_sample(args.config)
            vals.append(v)
        v = statistics.median(vals)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.config, "step": "one fixed-potential SQ3 iteration (oracle)"},
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
    res = run_sq3(args, rank, world)
    if rank == 0:
        v, cores, sample, parts = run_oracle_sample(args.config)
        res["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": cores, "kind": "oracle",
                               "sample": sample}
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
