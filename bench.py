"""Benchmark of the PeriDEM time step on GB300.

Default workload: the 50-grain mixed-shape settling aggregate (radii U[1, 1.5] mm,
h = R/15, dt = 5e-8 s, 20x30 mm wall box, seed 1).  One "step" is one full
velocity-Verlet time step of Algorithm 1 over all nodes (displacement update,
contact binning, bond + contact + self-contact + wall forces, velocity update).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).  Under torchrun every rank runs its own seeded
aggregate (independent problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s and bond evals/s vs plain FP64 GPU path at stated error; % HBM peak"
FLOPS_PER_BOND = 17      # algorithmic FP64 ops of one bond evaluation (sqrt, div counted once)


def workload_for(rank: int, args):
    from paper_2108_07212_gb300 import inputs as I
    return I.settling(n_grains=50, seed=1 + rank)


def describe(w, sim=None):
    d = {"workload": f"settling of {w.n_grains} mixed-shape grains (disk/hexagon/triangle/drop/annulus/plus), "
                     f"R~U[1,1.5] mm, h=R/15, dt={w.params['dt']:g} s, box 20x30 mm, gravity 5000 m/s^2"}
    if sim is not None:
        d.update(nodes=int(sim.N), directed_bonds=int(sim.n_bonds))
    return d


# ---------------------------------------------------------------------------


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f".clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
            os.remove(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def fp64_gemm_peak(torch, device):
    """Measured FP64 rate of a cuBLAS DGEMM (TFLOP/s): the FP64 denominator."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=device)
    b = torch.randn(n, n, dtype=torch.float64, device=device)
    for _ in range(2):
        torch.mm(a, b)
    torch.cuda.synchronize()
    best = math.inf
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.mm(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def cpu_baseline(w, budget_s: float = 12.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same workload."""
    from oracle import oracle as O
    P = O.OracleProblem.from_workload(w).init_accel()
    t0 = time.perf_counter()
    P.run(5)
    per = (time.perf_counter() - t0) / 5
    n = max(5, int(budget_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    P.run(n)
    dt = time.perf_counter() - t0
    return {"value": P.N * n / dt, "unit": "node-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} time steps of the full {P.N}-node workload from t=0 (single-threaded C, FP64)"}


# ---------------------------------------------------------------------------


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    w = workload_for(0, args)
    P = O.OracleProblem.from_workload(w).init_accel()
    for _ in range(args.warmup):
        P.run(1)
    t0 = time.perf_counter()
    P.run(args.steps)
    dt = time.perf_counter() - t0
    value = P.N * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w) | {"nodes": int(P.N), "directed_bonds": int(len(P.col))},
            "cpu_baseline": {"value": value, "unit": "node-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} time steps after {args.warmup} warm-up steps"},
            "e2e": {"value": value, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2108_07212_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    prec = B.PD_FP32_SPLIT if args.precision == "fp32" else B.PD_FP64
    w = workload_for(rank, args)
    with torch.cuda.stream(stream):
        sim = B.Simulation(w, precision=prec, device=dev, stream=stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()

    # warm-up
    sim.set_timing(True)
    for _ in range(args.warmup):
        flush_l2()
        sim.step(1)
    stream.synchronize()

    # timed region: L2 flushed before every step, each step bracketed by events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    force_ms = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush_l2()
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
            force_ms.append(sim.kernel_times()["force"])
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    elapsed = sum(step_ms) / 1e3
    if dist is not None:
        t = torch.tensor([elapsed], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    sim.set_timing(False)
    rc, st = sim.status()

    nodes_total = sim.N * world
    value = nodes_total * args.steps / elapsed
    bond_evals = sim.n_bonds * world * args.steps / elapsed

    # end to end through the C ABI with host buffers: per step upload the state
    # (u, v, a) from pinned host memory, advance one step, read positions back
    pin = {f: torch.empty((sim.N, 2), dtype=torch.float64).pin_memory() for f in ("DISP", "VEL", "ACC", "POS")}
    for f in ("DISP", "VEL", "ACC"):
        pin[f].numpy()[:] = sim.get(f)
    e2e_steps = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for f in ("DISP", "VEL", "ACC"):
            sim.set(f, pin[f].numpy())
        sim.step(1)
        out = pin["POS"].numpy()
        B._check(B.load().pd_get_state(sim._ctx, B.FIELDS["POS"], B._ptr(out), out.nbytes, 0))
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": sim.N * world * e2e_steps / e2e_dt, "unit": "node-steps/s",
           "h2d_bytes_per_step": 3 * 16 * sim.N, "d2h_bytes_per_step": 16 * sim.N,
           "steps": e2e_steps}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    fp64_peak = fp64_gemm_peak(torch, dev)
    f_ms = float(np.mean(force_ms))
    flops = FLOPS_PER_BOND * sim.n_bonds
    achieved = flops / (f_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == B.PD_FP64 else "f32+f64",
        "data": "synthetic",
        "config": describe(w, sim) | {"precision": args.precision, "l2": "flushed (256 MB write) before every timed step",
                                      "ranks": "independent seeded aggregates per rank"},
        "bond_evals_per_s": bond_evals,
        "roofline": {"bound": "alu", "kernel": "k_force64", "achieved": achieved, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": None,
                     "note": f"{FLOPS_PER_BOND} algorithmic FP64 ops per directed bond x {sim.n_bonds} bonds per "
                             f"launch / mean CUDA-event duration {f_ms * 1e3:.1f} us; peak = measured cuBLAS DGEMM "
                             "on this GPU (of measured)",
                     "hbm_peak_gbs": peaks.get("hbm_gbs")},
        "force_kernel_us": 1e3 * f_ms,
        "cpu_baseline": cpu_baseline(w) if not args.no_cpu else None,
        "e2e": e2e,
        "clocks": clocks.summary(),
        "gpu_launches": 6 * args.steps,
        "status": int(rc),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
