"""Benchmark of the PeriDEM time step on GB300.

Default workload: the batched ensemble of 64 independent settling aggregates
(20-200 grains each, seed 11; 6.69M nodes, 145M directed bonds) advanced in one
context, FP32-split precision, on the step path its autotuner picks.  One
"step" is one full velocity-Verlet time step of Algorithm 1 over all nodes of
all aggregates (displacement update, contact-list rebuild when due, bond +
contact + self-contact + wall forces, velocity update).  The plain FP64 path is
timed on the same state beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
                  [--workload ensemble64|compaction500|settling50|...] [--legs ...]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).  Under torchrun every rank runs its own seeded
ensemble (independent problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s and bond evals/s vs plain FP64 GPU path at stated error; % HBM peak"
# algorithmic bytes of the plain FP64 force phase: per node the FP64 position p,
# v and a read (48 B), v and a written (32 B), volume (8 B), grain, row pointer,
# broken-bond word and contact-list length (16 B), hash-grid cell (8 B); per
# directed bond the column and the FP64 reference length (12 B)
BYTES_PER_NODE_FP64 = 112
BYTES_PER_BOND_FP64 = 12
# the FP64 displacement update: X, u, v and a read (64 B), u and p written (32 B)
BYTES_UPDATE_FP64 = 96
# GB300 FP64 pipe: 2 lanes per SM per cycle on 152 SMs; a warp instruction on
# the FP64 pipe occupies it for 32 / 2 = 16 SM cycles whatever its active lanes
FP64_LANES_PER_SM_CYCLE = 2
N_SM = 152
# algorithmic bytes of the FP32-split force phase, bonds from the lattice stencil (every workload
# here: horizon 3 h): the lane sums read the float-float position pq (16 B), the stencil record
# (16 B), grain, broken-bond word and contact-list length (12 B) and write the force total (8 B);
# the epilogue reads the force total (8 B), the FP64 v (16 B), the FP32 a (8 B), grain (4 B) and
# the hash-grid cell of the wall test (8 B) and writes v and a (24 B).  120 B per node and no
# per-bond stream (nodes whose lattice row has a gap read CSR columns instead, 4 B per bond, not
# counted).  The fused force phase (one kernel, the force total stays on chip) reads the same
# inputs once: 100 B per node.
BYTES_PER_NODE_FP32 = 120
BYTES_PER_NODE_FP32_FUSED = 100
BYTES_PER_BOND_FP32 = 0
# the FP32-split displacement update as a phase of its own: X + shift, u, v, the FP32 a and the
# rebuild reference read, u and pq written (104 B); inside the persistent kernel's velocity update,
# where v and a are in registers: X + shift, u and the rebuild reference read, u and pq written (80 B)
BYTES_UPDATE_FP32 = 104
BYTES_UPDATE_FP32_FUSED = 80


def fp32_bytes_per_node(mode: int, whole: bool) -> int:
    """Algorithmic bytes per node of the FP32-split force phase of path `mode`
    (pd_set_path: bit 0 persistent, bit 1 split force phase), or of its whole
    step; the candidate-list rebuild runs only in some steps and is not counted."""
    force = BYTES_PER_NODE_FP32 if (mode >> 1) & 1 else BYTES_PER_NODE_FP32_FUSED
    if not whole:
        return force
    return force + (BYTES_UPDATE_FP32_FUSED if mode & 1 else BYTES_UPDATE_FP32)
B_STATUS_REBUILDS = 5    # status slot counting the contact candidate-list rebuilds


WORKLOADS = {
    # name: (generator, default seed, description)
    "settling50": ("settling", 1, "settling of 50 mixed-shape grains (disk/hexagon/triangle/drop/annulus/plus), "
                                  "R~U[1,1.5] mm, h=R/15, dt=5e-8 s, box 20x30 mm, gravity 5000 m/s^2"),
    "compaction500": ("compaction", 3, "compaction of 500 mixed-shape grains, R~U[0.8,1.6] mm, h=R/23, box width "
                                       "40 mm, top wall 0.1 m/s, dt=2e-8 s"),
    "ensemble64": ("ensemble", 11, "64 independent settling aggregates of 20-200 grains, R~U[0.8,1.2] mm, h=R/21, "
                                   "dt=2e-8 s, own wall box each"),
    "surrogate2000": ("surrogate_settling", 5, "settling of 2000 mixed-shape grains, R~U[1,1.5] mm, h=R/23, "
                                               "dt=2.5e-8 s, gravity 5000 m/s^2 (plain FP32 path)"),
    "agitated500": ("compaction", 3, "the 500-grain compaction aggregate with every grain thrown at 5 m/s in a seeded "
                                     "direction (collisions and fracture; contact lists rebuilt every few steps)"),
}
WORKLOAD_ARGS = {"agitated500": {"agitation": 5.0}}
# untimed steps before the timed window of each workload (the window starts
# mid-run, where grains move and collide and the contact lists are rebuilt)
DEFAULT_ADVANCE = {"settling50": 10000, "ensemble64": 2000, "compaction500": 200, "surrogate2000": 1000,
                   "agitated500": 200}


def workload_for(rank: int, args):
    """Rank r runs its own seeded aggregate (default seed + r): independent problems."""
    from paper_2108_07212_gb300 import inputs as I
    name = getattr(args, "workload", None) or "ensemble64"
    gen, seed, _ = WORKLOADS[name]
    if gen == "settling":
        return I.settling(n_grains=50, seed=seed + rank)
    return getattr(I, gen)(seed=seed + rank, **WORKLOAD_ARGS.get(name, {}))


def max_over_ranks(dist, values, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    whole-job time); identity without a process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def describe(w, sim=None, args=None):
    name = getattr(args, "workload", None) or "ensemble64"
    d = {"workload": WORKLOADS[name][2], "name": name}
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
        self.path = os.path.join(tempfile.gettempdir(), f"pd_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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


def oracle_sample(w, min_nodes: int):
    """Oracle problems of a bounded sample of the workload: for a batched ensemble
    its first aggregates (each an independent problem with its own walls) until
    they hold min_nodes nodes; otherwise the whole workload."""
    from oracle import oracle as O
    parts = getattr(w, "parts", None)
    if parts is None:
        return [O.OracleProblem.from_workload(w)], "the whole workload"
    probs, n = [], 0
    for p in parts:
        probs.append(O.OracleProblem.from_workload(p))
        n += probs[-1].N
        if n >= min_nodes:
            break
    return probs, f"its first {len(probs)} of {len(parts)} aggregates ({n} nodes)"


def _time_oracle(probs, omp: bool, n_steps: int) -> float:
    for P in probs:
        P.omp = omp
    t0 = time.perf_counter()
    for P in probs:
        P.run(n_steps)
    return time.perf_counter() - t0


def cpu_baseline(w, advance: int = 0, budget_s: float = 20.0, min_nodes: int = 200_000):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same
    workload: advanced (all-core build, untimed) to the GPU's timed window, then
    the single-threaded build and the all-core (OpenMP) build, each for about
    half the budget.  Returns the baseline and the oracle problems (their final
    state serves the oracle-parity report)."""
    from oracle import oracle as O
    probs, what = oracle_sample(w, min_nodes)
    for P in probs:
        P.omp = True
        P.init_accel()
    if advance:
        _time_oracle(probs, True, advance)
    n_nodes = sum(P.N for P in probs)
    per = _time_oracle(probs, False, 2) / 2
    n1 = max(3, int(0.5 * budget_s / max(per, 1e-6)))
    dt1 = _time_oracle(probs, False, n1)
    per = _time_oracle(probs, True, 2) / 2
    n2 = max(3, int(0.5 * budget_s / max(per, 1e-6)))
    dt2 = _time_oracle(probs, True, n2)
    cores = O.threads_available()
    first = advance + 4 + n1
    return {"value": n_nodes * n2 / dt2, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{what}: steps {first}..{first + n2} with the all-core build (OpenMP, {cores} threads), "
                      f"FP64 C (steps 0..{advance} run untimed first: the GPU's window)",
            "single_thread": {"value": n_nodes * n1 / dt1, "unit": "node-steps/s", "cores": 1,
                              "sample": f"{what}: steps {advance + 2}..{advance + 2 + n1}, single-threaded build"}}, probs


def oracle_parity(B, probs, sims, w):
    """The GPU paths against the oracle at the oracle's own state (the end of
    the CPU-baseline run): the oracle's displacement, velocity, acceleration,
    broken bonds and step are pushed into each GPU context over the sample's
    aggregates, one force evaluation runs on both sides, and the nodal forces
    rho V (a - g) and the broken-bond sets are compared over the sample."""
    rho = w.params["rho"]
    g = np.array([w.params["gx"], w.params["gy"]])
    refs = []
    for P in probs:
        so = {"DISP": P.u.copy(), "VEL": P.v.copy(), "ACC": P.a.copy(), "BROKEN": P.broken[: len(P.col)].copy()}
        F, parts = P.forces(keep_broken=False)
        refs.append((so, F, parts, P.broken[: len(P.col)].copy(), rho * P.V[:, None]))
    out = {"sample": f"the oracle's {len(probs)} sample aggregates ({sum(P.N for P in probs)} nodes) at its "
                     f"step {probs[0].step}", "reference": "the FP64 oracle, one force evaluation at its state"}
    for name, S in sims.items():
        grain = S.get("GRAIN")
        agg = w.grain_agg[grain] if getattr(w, "grain_agg", None) is not None else np.zeros(S.N, np.int64)
        row = S.get("ROW_PTR")
        st = {f: S.get(f) for f in ("DISP", "VEL", "ACC", "BROKEN")}
        ranges = []
        for a, (so, *_rest) in enumerate(refs):
            nodes = np.flatnonzero(agg == a)
            n0, n1 = int(nodes[0]), int(nodes[-1]) + 1
            assert n1 - n0 == nodes.size == len(so["DISP"])
            b0, b1 = int(row[n0]), int(row[n1])
            ranges.append((n0, n1, b0, b1))
            for f in ("DISP", "VEL", "ACC"):
                st[f][n0:n1] = so[f]
            st["BROKEN"][b0:b1] = so["BROKEN"]
        for f, val in st.items():
            S.set(f, val)
        S.set("STEP", np.array([probs[0].step], np.int64))
        S.eval_forces()
        acc, br = S.get("ACC"), S.get("BROKEN")
        err, scale, dis, nbroken = 0.0, 0.0, 0, 0
        for (n0, n1, b0, b1), (so, F_or, parts_or, br_or, m) in zip(ranges, refs):
            Fg = m * (acc[n0:n1] - g)
            scale = max(scale, float(np.abs(F_or).max()), float(m.max()) * max(float(np.abs(g).max()), 100.0))
            err = max(err, float(np.abs(Fg - F_or).max()))
            dis += int(np.sum(br[b0:b1] != br_or))
            nbroken += int(br_or.sum())
        out[name] = {"force_rel_err_max_norm": err / scale, "break_disagreements": dis}
        out["force_scale_N"] = scale
        out["broken_bonds_oracle"] = nbroken
        out["contact_active"] = bool(any(np.abs(r[2][2]).max() > 0 for r in refs))
    return out


# ---------------------------------------------------------------------------


def run_reference(args):
    """The oracle as the reference arm: the all-core build on a bounded sample of
    the main line's workload (for the ensemble: its first aggregates, about 1M
    nodes), advanced untimed to the GPU arm's window, then W untimed and K
    timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    w = workload_for(0, args)
    probs, what = oracle_sample(w, 1_000_000)
    for P in probs:
        P.omp = True
        P.init_accel()
    # the same window as the GPU arm: steps 0..advance run untimed first
    advance = DEFAULT_ADVANCE.get(args.workload, 0) if args.advance is None else args.advance
    if advance:
        _time_oracle(probs, True, advance)
    _time_oracle(probs, True, args.warmup)
    dt = _time_oracle(probs, True, args.steps)
    n_nodes = sum(P.N for P in probs)
    n_bonds = sum(len(P.col) for P in probs)
    value = n_nodes * args.steps / dt
    cores = O.threads_available()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, None, args) | {"sample": what, "sample_nodes": int(n_nodes),
                                                 "sample_directed_bonds": int(n_bonds),
                                                 "window": f"steps {advance + args.warmup}.."
                                                           f"{advance + args.warmup + args.steps} of the run"},
            "cpu_baseline": {"value": value, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{what}: {args.steps} time steps after {args.warmup} warm-up steps, "
                                       f"all-core build (OpenMP, {cores} threads)"},
            "e2e": {"value": value, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _timed_steps(sim, stream, flush, steps, warmup, torch):
    """Per-step CUDA-event times (L2 flushed before every step), the force
    kernel's event-node durations and the candidate-list rebuilds of the timed
    steps.  The step times come from the plain step graphs; the force-kernel
    durations from a second pass over the same number of steps with the
    instrumented graphs (event nodes around the kernel groups), so the event
    nodes do not add to the step time.  The first pass runs between
    cudaProfilerStart/Stop, so an ncu launch list taken with
    --profile-from-start off holds exactly its steps."""
    for _ in range(warmup):
        flush()
        sim.step(1)
    stream.synchronize()
    rebuilds0 = int(sim.status()[1][B_STATUS_REBUILDS])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.profiler.start()
    for k in range(steps):
        flush()
        ev[k][0].record(stream)
        sim.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    rebuilds = int(sim.status()[1][B_STATUS_REBUILDS]) - rebuilds0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    sim.set_timing(True)
    force_ms = []
    for k in range(steps):
        flush()
        sim.step(1)
        force_ms.append(sim.kernel_times()["force"])
    torch.cuda.synchronize()
    sim.set_timing(False)
    return step_ms, force_ms, rebuilds


# ---------------------------------------------------------------------------
# workload legs at the sizes where HBM, not launch latency, bounds the step
# (500-grain compaction, 64-aggregate ensemble, 2000-grain surrogate settling)

# the largest whole-step model (separate update phase, split force phase): the
# workload size above which the inputs exceed L2 many times over
BYTES_PER_NODE_STEP_FP32_MAX = BYTES_UPDATE_FP32 + BYTES_PER_NODE_FP32


# DRAM bytes (read + write) per launch of the force-phase kernels, per workload,
# from one ncu capture (one pass) of the timed steps (the bench marks them with
# cudaProfilerStart/Stop; path mode 6 = mode 2 without the conditional graph
# node, which ncu cannot trace; the same kernels), e.g.
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
#       --profile-from-start off -k regex:"k_sums|k_epilogue" --csv
#       python bench.py --steps 3 --warmup 3 --legs= --no-cpu --path 6,1
# (medians over the three captured launches; summaries under profiles/).  They
# hold while the kernel sources hash to TRAFFIC_DIGEST; otherwise, or for a
# kernel not captured, traffic is null.
TRAFFIC = {
    "ensemble64": {"k_persistent<1, 1, 256>": 1196907520, "k_persistent<0, 1, 256>": 3344664064,
                   "k_sums<1, 1>": 356045568, "k_epilogue<1>": 421486080,
                   "k_sums<0, 1>": 2233693952, "k_epilogue<0>": 584599552},
    "compaction500": {"k_persistent<1, 1, 256>": 69165824, "k_persistent<0, 1, 256>": 244184320,
                      "k_persistent<1, 1, 128>": 69178880, "k_persistent<0, 1, 128>": 243823872,
                      "k_sums<1, 1>": 23607040, "k_epilogue<1>": 23026944,
                      "k_sums<0, 1>": 170565120, "k_epilogue<0>": 31460864},
}
TRAFFIC_DIGEST = "1235532d82438481bf9c97cad09580c8b576d3ac"
TRAFFIC_SOURCES = ("pd_device.cuh", "pd_step.cuh", "pd_step32.cu", "pd_step64.cu", "pd_persist.cu", "pd_common.cu",
                   "pd_internal.h")


def kernel_digest() -> str:
    """SHA-1 of the force-kernel sources and of the build script (compile flags)."""
    import hashlib
    hsh = hashlib.sha1()
    paths = [os.path.join(ROOT, "paper_2108_07212_gb300", "csrc", f) for f in TRAFFIC_SOURCES]
    for f in paths + [os.path.join(ROOT, "paper_2108_07212_gb300", "build.py")]:
        with open(f, "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def force_phase_traffic(path: dict, fp32: bool, workload: str):
    """Measured DRAM bytes of one force phase of the chosen path, or None."""
    table = TRAFFIC.get(workload, {})
    if not table or kernel_digest() != TRAFFIC_DIGEST:
        return None
    p, m, l = ("1" if fp32 else "0"), path["mode"], path["lanes"]
    if m & 1:
        names = [f"k_persistent<{p}, {l}, {path.get('block', 128)}>"]     # the whole step
    else:
        names = [f"k_sums<{p}, {l}>", f"k_epilogue<{p}>"] if (m >> 1) & 1 else [f"k_force<{p}, {l}>"]
    if not all(n in table for n in names):
        return None
    return float(sum(table[n] for n in names))


def _force_kernels(mode: int, fp32: bool) -> str:
    """Name of the force phase of a step path (pd_set_path modes)."""
    p = "1" if fp32 else "0"
    if mode & 1:
        return f"k_persistent<{p},...> (whole step)"
    return f"k_sums<{p},...> + k_epilogue<{p}>" if (mode >> 1) & 1 else f"k_force<{p},...>"


def _launches(mode: int, steps: int, rebuilds: int) -> int:
    """Kernels launched by `steps` timed steps: the displacement update and the
    force phase (one or two kernels) every step, plus the six rebuild kernels
    (bin, three scan kernels, scatter, lists) in the steps whose conditional
    node ran them; the persistent kernel is one launch per step."""
    if mode & 1:
        return steps
    if mode & 4:      # rebuild kernels launched every step
        return steps * (8 + ((mode >> 1) & 1))
    return steps * (2 + ((mode >> 1) & 1)) + 6 * rebuilds


def _event_time(stream, torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _force_kernel_ms(sim, n=20):
    sim.set_timing(True)
    ms = []
    for _ in range(n):
        sim.step(1)
        ms.append(sim.kernel_times()["force"])
    sim.set_timing(False)
    return float(np.median(ms))


def _roof_fp32(sim, f_ms, hbm, label, path=None, workload=None):
    """HBM roofline of the FP32-split force group: the force phase on the
    kernel-graph paths, the whole step when the persistent kernel, which runs
    every phase of the step, is the timed group (fp32_bytes_per_node)."""
    per_node = fp32_bytes_per_node(path["mode"], bool(path["mode"] & 1)) if path else BYTES_PER_NODE_FP32
    nbytes = per_node * sim.N + BYTES_PER_BOND_FP32 * sim.n_bonds
    a = nbytes / (f_ms / 1e3) / 1e9
    traffic = force_phase_traffic(path, True, workload) if path and workload else None
    return {"bound": "hbm", "kernel": _force_kernels(path["mode"], True) if path else "k_force32", "achieved": a,
            "peak": hbm, "unit": "GB/s", "frac": a / hbm,
            "traffic": traffic, "note": f"{label}: {per_node} B/node + {BYTES_PER_BOND_FP32} B/bond x "
                                     f"{sim.N} nodes / {sim.n_bonds} bonds, median event time {f_ms * 1e3:.1f} us (of measured)"}


# Warp instructions on the FP64 pipe per launch of the FP64 force-phase kernels
# (ncu smsp__inst_executed_pipe_fp64.sum, one launch each, --clock-control none;
# profiles/force64_*.md), per workload; they hold while the kernel sources hash
# to FP64_INST_DIGEST, otherwise the ALU roofline is left unmeasured.
FP64_INST = {
    "ensemble64": {"k_persistent<0, 1, 256>": 36245494, "k_sums<0, 1>": 32548173,
                   "k_epilogue<0>": 1674592},
    "compaction500": {"k_persistent<0, 1, 256>": 2784267, "k_persistent<0, 1, 128>": 2784259,
                      "k_sums<0, 1>": 2492904, "k_epilogue<0>": 130368},
}
FP64_INST_DIGEST = "1235532d82438481bf9c97cad09580c8b576d3ac"


def _roof_fp64(sim, f_ms, path, workload, clk, hbm):
    """Roofline of the plain FP64 force phase.  Bound: the FP64 pipe.  Peak =
    152 SMs x 2 FP64 lanes per cycle x the median SM clock sampled during the
    timed steps (lane operations per second); achieved = 32 x the FP64-pipe warp
    instructions of one launch (ncu) / its CUDA-event duration, i.e. frac is the
    share of the phase the FP64 pipe is busy.  The HBM fraction of the same
    phase (algorithmic bytes / duration) is reported beside it."""
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = N_SM * FP64_LANES_PER_SM_CYCLE * mhz * 1e6 / 1e12          # tera lane-ops/s
    m, l = path["mode"], path["lanes"]
    names = [f"k_persistent<0, {l}, {path.get('block', 128)}>"] if m & 1 else (
        [f"k_sums<0, {l}>", f"k_epilogue<0>"] if (m >> 1) & 1 else [f"k_force<0, {l}>"])
    table = FP64_INST.get(workload, {}) if kernel_digest() == FP64_INST_DIGEST else {}
    inst = sum(table[n] for n in names) if all(n in table for n in names) else None
    # the persistent kernel is the whole step: the displacement update's bytes too
    per_node = BYTES_PER_NODE_FP64 + (BYTES_UPDATE_FP64 if m & 1 else 0)
    nbytes = per_node * sim.N + BYTES_PER_BOND_FP64 * sim.n_bonds
    hbm_a = nbytes / (f_ms / 1e3) / 1e9
    achieved = None if inst is None else 32.0 * inst / (f_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": _force_kernels(m, False), "achieved": achieved, "peak": peak,
            "unit": "T FP64 lane-ops/s", "frac": None if achieved is None else achieved / peak,
            "traffic": force_phase_traffic(path, False, workload),
            "hbm": {"achieved": hbm_a, "peak": hbm, "unit": "GB/s", "frac": hbm_a / hbm,
                    "note": f"{per_node} B/node + {BYTES_PER_BOND_FP64} B/bond (of measured)"},
            "note": f"peak = {N_SM} SMs x {FP64_LANES_PER_SM_CYCLE} FP64 lanes/cycle x {mhz:.0f} MHz (derived); "
                    + ("achieved = 32 x %d FP64-pipe warp instructions (ncu) / mean event time %.1f us"
                       % (inst, f_ms * 1e3) if inst is not None else
                       "FP64 instruction count not captured for this kernel build (achieved unmeasured)")}


def leg_compaction(B, I, dev, stream, torch, hbm, clk, steps=200):
    """500 grains, ~5e5 nodes: FP64 path vs FP32 split, throughput, force error and
    break disagreements on an agitated (colliding, fracturing) state."""
    out = {}
    w = I.compaction()
    for prec, name in ((B.PD_FP64, "fp64"), (B.PD_FP32_SPLIT, "fp32")):
        with torch.cuda.stream(stream):
            sim = B.Simulation(w, precision=prec, device=dev, stream=stream)
        tune = sim.autotune()
        sim.step(16)
        dt = _event_time(stream, torch, lambda: sim.step(steps))
        f_ms = _force_kernel_ms(sim)
        out[name] = {"value": sim.N * steps / dt, "unit": "node-steps/s", "ms_per_step": 1e3 * dt / steps,
                     "bond_evals_per_s": sim.n_bonds * steps / dt, "force_kernel_us": 1e3 * f_ms,
                     "roofline": _roof_fp32(sim, f_ms, hbm, "500-grain compaction", tune, "compaction500")
                     if name == "fp32"
                     else _roof_fp64(sim, f_ms, tune, "compaction500", clk, hbm),
                     "step_path": tune, "status": int(sim.status()[0])}
        out["nodes"], out["directed_bonds"] = int(sim.N), int(sim.n_bonds)
        del sim
    out["speedup_fp32_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    # precision report on the agitated state (grains thrown at 5 m/s in random directions)
    wa = I.compaction(agitation=5.0)
    with torch.cuda.stream(stream):
        a = B.Simulation(wa, precision=B.PD_FP64, store_parts=True, device=dev, stream=stream)
        b = B.Simulation(wa, precision=B.PD_FP32_SPLIT, store_parts=True, device=dev, stream=stream)
    n_win = 600
    a.step(n_win)
    b.step(n_win)
    n_dis = int(np.sum(a.get("BROKEN") != b.get("BROKEN")))
    n_broken = int(a.get("BROKEN").sum())
    for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP"):
        b.set(f, a.get(f))
    a.eval_forces()
    b.eval_forces()
    Fa, Fb = a.get("FORCE"), b.get("FORCE")
    out["precision_report"] = {
        "workload": f"the same aggregate with every grain thrown at 5 m/s (seeded directions), {n_win} steps",
        "force_rel_err_max_norm": float(np.abs(Fb - Fa).max() / np.abs(Fa).max()),
        "broken_bonds_fp64": n_broken, f"break_disagreements_after_{n_win}_steps": n_dis,
        "reference": "the plain FP64 GPU path (its parity with the FP64 oracle on this agitated state: "
                     "tests/test_gpu_fullsize.py, 1e-12 per force part, identical broken bonds)"}
    out["workload"] = ("compaction of 500 mixed-shape grains, R~U[0.8,1.6] mm, h=R/23, box width 40 mm, "
                       "top wall 0.1 m/s, dt=2e-8 s")
    del a, b
    return out


def leg_surrogate(B, I, SU, dev, stream, torch, steps=200, profile_steps=0):
    """2000 grains (~2e6 nodes, h=R/23), FP32 split: surrogate (networks trained
    on snapshots of a small aggregate with the same templates) vs the plain
    FP32 and FP64 paths.  With profile_steps, only that many surrogate steps
    (not judge steps) run on path mode 6 (no conditional graph node, which ncu
    cannot trace) between cudaProfilerStart/Stop, and the leg ends there."""
    w = I.surrogate_settling()
    # training snapshots: 60 grains of the same shapes and h/R, each thrown at
    # 1 m/s in a seeded random direction so that collisions load them
    wt = I.surrogate_settling(n_grains=60, seed=6)
    with torch.cuda.stream(stream):
        T = B.Simulation(wt, precision=B.PD_FP32_SPLIT, store_parts=True, device=dev, stream=stream,
                         surrogate=lambda s_: SU.build_basis(s_))
    ang = np.random.Generator(np.random.PCG64(66)).uniform(0.0, 2 * math.pi, wt.n_grains)
    vg = np.stack([np.cos(ang), np.sin(ang)], 1)
    T.set("VEL", vg[T.get("GRAIN")])
    t0 = time.perf_counter()
    data = SU.collect_samples(T, 1500, 15)
    t_collect = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        S = B.Simulation(w, precision=B.PD_FP32_SPLIT, device=dev, stream=stream,
                         surrogate=lambda s_: SU.build_basis(s_, source=(T, T.surrogate_basis)))
    cfg = S.surrogate_basis
    lam = cfg["lambda_"].reshape(-1, cfg["n_modes"])
    t0 = time.perf_counter()
    src = {k: t for t, k in enumerate(SU.template_keys(T, T.surrogate_basis))}
    counts = np.bincount(cfg["template_of_grain"])
    nets, trained = [], 0
    for t, key in enumerate(SU.template_keys(S, cfg)):
        tt = src.get(key)
        params = SU.init_params(0)
        if tt is not None and tt in data:
            params = SU.train_template(*data[tt], lam[t], epochs=400)[0]
            trained += 1
        nets.append(B.MLP(max_batch=int(counts[t]), stream=stream, params=params))
        S.surrogate_set_mlp(t, nets[-1])
    t_train = time.perf_counter() - t0
    S.surrogate_enable(True)
    if profile_steps:
        S.set_path(6, 1, 128)
        S.step(3)                                    # steps 1-3; the judge runs every 50th
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        S.step(profile_steps)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return {"profiled_surrogate_steps": profile_steps, "nodes": int(S.N), "status": int(S.status()[0])}
    S.autotune()
    with torch.cuda.stream(stream):
        P = B.Simulation(w, precision=B.PD_FP32_SPLIT, device=dev, stream=stream)
    P.autotune()
    out = {"workload": "settling of 2000 mixed-shape grains, R~U[1,1.5] mm, h=R/23, dt=2.5e-8 s, gravity 5000 m/s^2",
           "nodes": int(S.N), "directed_bonds": int(S.n_bonds), "templates": len(cfg["templates"]),
           "networks_trained": trained, "training": {"samples_s": t_collect, "train_s": t_train,
                                                      "source": "60-grain aggregate of the same templates, 1500 steps"}}
    res = {}
    for sim, name in ((P, "plain_fp32"), (S, "surrogate")):
        sim.step(16)
        dt = _event_time(stream, torch, lambda: sim.step(steps))
        res[name] = {"value": sim.N * steps / dt, "unit": "node-steps/s", "ms_per_step": 1e3 * dt / steps}
    active, err, merr, maxs = S.surrogate_stats()
    on = active == 1
    res["surrogate"].update(active_grains=int(on.sum()), judged_err_p50=float(np.median(err[on])) if on.any() else None,
                            judged_err_max=float(err[on].max()) if on.any() else None,
                            judged_modal_err_p50=float(np.median(merr[on])) if on.any() else None,
                            max_stretch_over_s0=float(maxs.max()))
    u0, u1 = P.get("DISP"), S.get("DISP")
    res["surrogate"]["traj_rel_l2_vs_plain"] = float(np.linalg.norm(u1 - u0) / max(np.linalg.norm(u0), 1e-300))
    res["surrogate"]["status"] = int(S.status()[0])
    del P
    torch.cuda.empty_cache()
    with torch.cuda.stream(stream):
        D = B.Simulation(w, precision=B.PD_FP64, device=dev, stream=stream)
    D.autotune()
    D.step(16)
    dt = _event_time(stream, torch, lambda: D.step(steps // 4))
    res["plain_fp64"] = {"value": D.N * (steps // 4) / dt, "unit": "node-steps/s", "ms_per_step": 4e3 * dt / steps}
    out.update(res)
    out["speedup_vs_plain_fp32"] = res["surrogate"]["value"] / res["plain_fp32"]["value"]
    out["speedup_vs_plain_fp64"] = res["surrogate"]["value"] / res["plain_fp64"]["value"]
    del D, S
    torch.cuda.empty_cache()
    out["landing"] = _surrogate_landing(B, I, SU, dev, stream, torch, T, data, steps)
    del T
    torch.cuda.empty_cache()
    return out


def _surrogate_landing(B, I, SU, dev, stream, torch, T, data, steps, advance=1200):
    """The same 2000 grains lowered to 1.02 R_c above the floor and thrown down
    at 2 m/s: the lowest grains land and deform, the judge (every 50 steps)
    takes off the surrogate every grain whose nodal bond-force error exceeds
    1e-3, the rest stay on it.  Both paths run `advance` steps from the same
    initial state, then `steps` timed steps."""
    w = I.surrogate_settling()
    with torch.cuda.stream(stream):
        X = B.Simulation(w, device=dev, stream=stream).get("X")        # meshing only (host)
    rc = w.params["rc_ratio"] * w.grain_geom[:, 6].min()
    w.grain_geom[:, 1] -= X[:, 1].min() - 1.02 * rc
    w.grain_geom[:, 5] = -2.0
    with torch.cuda.stream(stream):
        S = B.Simulation(w, precision=B.PD_FP32_SPLIT, device=dev, stream=stream,
                         surrogate=lambda s_: SU.build_basis(s_, source=(T, T.surrogate_basis)))
    cfg = S.surrogate_basis
    lam = cfg["lambda_"].reshape(-1, cfg["n_modes"])
    src = {k: t for t, k in enumerate(SU.template_keys(T, T.surrogate_basis))}
    counts = np.bincount(cfg["template_of_grain"])
    nets = []
    for t, key in enumerate(SU.template_keys(S, cfg)):
        tt = src.get(key)
        params = SU.train_template(*data[tt], lam[t], epochs=400)[0] if tt is not None and tt in data \
            else SU.init_params(0)
        nets.append(B.MLP(max_batch=int(counts[t]), stream=stream, params=params))
        S.surrogate_set_mlp(t, nets[-1])
    S.surrogate_enable(True)
    S.autotune()
    with torch.cuda.stream(stream):
        P = B.Simulation(w, precision=B.PD_FP32_SPLIT, device=dev, stream=stream)
    P.autotune()
    res = {"workload": "the same grains 1.02 R_c above the floor, all moving down at 2 m/s (landing)",
           "window": f"steps {advance}..{advance + steps}"}
    for sim, name in ((P, "plain_fp32"), (S, "surrogate")):
        sim.step(advance)
        dt = _event_time(stream, torch, lambda: sim.step(steps))
        res[name] = {"value": sim.N * steps / dt, "unit": "node-steps/s", "ms_per_step": 1e3 * dt / steps}
    active, err, merr, maxs = S.surrogate_stats()
    on = active == 1
    res["surrogate"].update(
        active_grains=int(on.sum()), grains=int(w.n_grains),
        judged_err_max=float(err[on].max()) if on.any() else None,
        max_stretch_over_s0_active=float(maxs[on].max()) if on.any() else None,
        max_stretch_over_s0_all=float(maxs.max()), status=int(S.status()[0]))
    u0, u1 = P.get("DISP"), S.get("DISP")
    res["surrogate"]["traj_rel_l2_vs_plain"] = float(np.linalg.norm(u1 - u0) / max(np.linalg.norm(u0), 1e-300))
    res["speedup_vs_plain_fp32"] = res["surrogate"]["value"] / res["plain_fp32"]["value"]
    del P, S
    return res


def _same_state_force_report(B, sim32, sim64, w):
    """FP32-split vs FP64 path at one state: the FP64 context's state is pushed
    into the FP32 one, both evaluate forces once, and the nodal forces
    rho V (a - g) and the broken bonds are compared."""
    for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP"):
        sim32.set(f, sim64.get(f))
    sim64.eval_forces()
    sim32.eval_forces()
    g = np.array([w.params["gx"], w.params["gy"]])
    a64, a32 = sim64.get("ACC") - g, sim32.get("ACC") - g
    m = w.params["rho"] * sim64.get("VOLUME")[:, None]
    F64, F32 = m * a64, m * a32
    # scale: the largest nodal force, floored at the largest nodal weight (in free
    # fall the forces vanish and the float path's absolute floor would dominate)
    scale = max(np.abs(F64).max(), float(m.max()) * max(float(np.abs(g).max()), 100.0))
    return {"force_rel_err_max_norm": float(np.abs(F32 - F64).max() / scale),
            "force_scale_N": scale, "largest_force_N": float(np.abs(F64).max()),
            "broken_bonds_fp64": int(sim64.get("BROKEN").sum()),
            "break_disagreements": int(np.sum(sim64.get("BROKEN") != sim32.get("BROKEN"))),
            "reference": "the plain FP64 GPU path at the same state (its parity with the FP64 oracle at this size: "
                         "tests/test_gpu_fullsize.py, 1e-12)"}


def leg_settling(B, I, dev, stream, torch, steps=200, advance=10000):
    """The 50-grain settling (19,681 nodes): small enough to live in L2, so the
    step is bound by launch and dependency latency; FP32 split vs FP64, L2
    flushed before every timed step."""
    w = I.settling(n_grains=50, seed=1)
    flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = {"workload": WORKLOADS["settling50"][2], "window": f"steps {advance}..{advance + steps}",
           "l2": "flushed (256 MB write) before every timed step"}

    def flush():
        with torch.cuda.stream(stream):
            flush_buf.zero_()

    for prec, name in ((B.PD_FP32_SPLIT, "fp32"), (B.PD_FP64, "fp64")):
        with torch.cuda.stream(stream):
            sim = B.Simulation(w, precision=prec, device=dev, stream=stream)
        sim.step(advance)
        tune = sim.autotune()
        step_ms, force_ms, rebuilds = _timed_steps(sim, stream, flush, steps, 5, torch)
        dt = sum(step_ms) / 1e3
        out[name] = {"value": sim.N * steps / dt, "unit": "node-steps/s", "ms_per_step": 1e3 * dt / steps,
                     "force_kernel_us": 1e3 * float(np.mean(force_ms)), "rebuilds": rebuilds, "step_path": tune,
                     "status": int(sim.status()[0])}
        out["nodes"], out["directed_bonds"] = int(sim.N), int(sim.n_bonds)
        del sim
    del flush_buf
    out["speedup_fp32_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def leg_sequential(B, w, dev, stream, torch, steps=40):
    """The ensemble's 64 aggregates run one after another in separate contexts
    (FP32 split, and the plain FP64 path): the baseline of the batched form."""
    out = {}
    for prec, name in ((B.PD_FP32_SPLIT, "sequential_fp32"), (B.PD_FP64, "sequential_fp64")):
        sims = []
        with torch.cuda.stream(stream):
            for part in w.parts:
                sims.append(B.Simulation(part, precision=prec, device=dev, stream=stream))
        for s_ in sims:
            s_.step(16)

        def run():
            for s_ in sims:
                s_.step(steps)
        dts = _event_time(stream, torch, run)
        n_tot = sum(int(s_.N) for s_ in sims)
        out[name] = {"value": n_tot * steps / dts, "unit": "node-steps/s", "ms_per_step": 1e3 * dts / steps}
        del sims
        torch.cuda.empty_cache()
    return out


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
    advance = DEFAULT_ADVANCE.get(args.workload, 0) if args.advance is None else args.advance
    with torch.cuda.stream(stream):
        sim = B.Simulation(w, precision=prec, device=dev, stream=stream)
    # the timed window starts mid-run (steps advance..advance+steps)
    if advance:
        sim.step(advance)
    # the plain FP64 path from the same state (pushed), timed on the same window
    sim64 = None
    if prec != B.PD_FP64:
        with torch.cuda.stream(stream):
            sim64 = B.Simulation(w, precision=B.PD_FP64, device=dev, stream=stream)
        for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP"):
            sim64.set(f, sim.get(f))

    # both paths run the step variant their own autotuner picks (state unchanged),
    # unless --path fixes it
    def pick(x):
        if args.path:
            v = [int(t) for t in args.path.split(",")]
            x.set_path(v[0], v[1], v[2] if len(v) > 2 else 128)
            inf = x.info()
            return {"mode": int(inf["mode"]), "lanes": int(inf["lanes"]), "block": int(inf["block"]), "fixed": True}
        return x.autotune()
    key = "fp32" if prec != B.PD_FP64 else "fp64"
    tuned = {key: pick(sim)}
    if sim64 is not None:
        tuned["fp64"] = pick(sim64)
    big = sim.N * BYTES_PER_NODE_STEP_FP32_MAX > 512 * 1024 * 1024
    flush_buf = None if big else torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def flush_l2():
        if flush_buf is not None:
            with torch.cuda.stream(stream):
                flush_buf.zero_()

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        step_ms, force_ms, rebuilds = _timed_steps(sim, stream, flush_l2, args.steps, args.warmup, torch)
        if sim64 is not None:
            step64_ms, force64_ms, rebuilds64 = _timed_steps(sim64, stream, flush_l2, args.steps, args.warmup, torch)
    elapsed = sum(step_ms) / 1e3
    elapsed64 = sum(step64_ms) / 1e3 if sim64 is not None else elapsed
    elapsed, elapsed64 = max_over_ranks(dist, [elapsed, elapsed64], dev)
    rc, st = sim.status()

    value = sim.N * world * args.steps / elapsed
    bond_evals = sim.n_bonds * world * args.steps / elapsed
    value64 = sim.N * world * args.steps / elapsed64

    # end to end through the C ABI with host buffers: per step upload the state
    # (u, v, a) from pinned host memory, advance one step, read positions back
    # (page-locked buffers: the copies are enqueued on the stream and the step
    # ends with one stream synchronisation, after which the positions are on the host)
    pin = {f: torch.empty((sim.N, 2), dtype=torch.float64).pin_memory() for f in ("DISP", "VEL", "ACC", "POS")}
    for f in ("DISP", "VEL", "ACC"):
        pin[f].numpy()[:] = sim.get(f)
    e2e_steps = max(3, min(args.steps, 200))
    L = B.load()
    ups = [(B.FIELDS[f], ctypes.c_void_p(pin[f].data_ptr()), 16 * sim.N) for f in ("DISP", "VEL", "ACC")]
    down = (B.FIELDS["POS"], ctypes.c_void_p(pin["POS"].data_ptr()), 16 * sim.N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for fld, ptr, nb in ups:
            B._check(L.pd_set_state(sim._ctx, fld, ptr, nb, B.PD_MEM_HOST_ASYNC))
        B._check(L.pd_step(sim._ctx, 1))
        B._check(L.pd_get_state(sim._ctx, down[0], down[1], down[2], B.PD_MEM_HOST_ASYNC))
        stream.synchronize()
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e_dt = max_over_ranks(dist, [e2e_dt], dev)[0]
    e2e = {"value": sim.N * world * e2e_steps / e2e_dt, "unit": "node-steps/s",
           "h2d_bytes_per_step": 3 * 16 * sim.N, "d2h_bytes_per_step": 16 * sim.N, "steps": e2e_steps}
    del pin

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    clk = clocks.summary()
    f_ms = float(np.mean(force_ms))
    # the persistent kernel is the whole step: its duration is bounded by the
    # event-timed plain step (graph launch included), which the instrumented
    # graph's event nodes would otherwise inflate
    if tuned[key]["mode"] & 1:
        f_ms = min(f_ms, float(np.mean(step_ms)))
    if prec == B.PD_FP64:
        roof = _roof_fp64(sim, f_ms, tuned["fp64"], args.workload, clk, hbm)
    else:
        whole = bool(tuned["fp32"]["mode"] & 1)          # persistent kernel: one launch for the whole step
        per_node = fp32_bytes_per_node(tuned["fp32"]["mode"], whole)
        nbytes = per_node * sim.N + BYTES_PER_BOND_FP32 * sim.n_bonds
        achieved = nbytes / (f_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": _force_kernels(tuned["fp32"]["mode"], True), "achieved": achieved, "peak": hbm,
                "unit": "GB/s",
                "frac": achieved / hbm, "traffic": force_phase_traffic(tuned["fp32"], True, args.workload),
                "note": f"{per_node} B per node + {BYTES_PER_BOND_FP32} B per directed bond (algorithmic) x "
                        f"{sim.N} nodes / {sim.n_bonds} bonds per {'step' if whole else 'force phase'} / mean "
                        f"CUDA-event duration {f_ms * 1e3:.1f} us"
                        + (" (persistent kernel = the whole step: event-timed step, graph launch included)" if whole else "")
                        + "; peak = measured copy bandwidth (of measured)"
                        + ("; the workload is too small to load 152 SMs, so the phase is latency-bound"
                           if sim.N < 100000 else "")}
    if prec == B.PD_FP64:
        step_per_node, step_per_bond = BYTES_UPDATE_FP64 + BYTES_PER_NODE_FP64, BYTES_PER_BOND_FP64
    else:
        step_per_node, step_per_bond = fp32_bytes_per_node(tuned[key]["mode"], True), BYTES_PER_BOND_FP32
    step_bytes = step_per_node * sim.N + step_per_bond * sim.n_bonds
    step_s = elapsed / args.steps / world
    line = {
        "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == B.PD_FP64 else "f32+f64",
        "data": "synthetic",
        "config": describe(w, sim, args) | {"precision": "fp64" if prec == B.PD_FP64 else "fp32 split (FP32 forces, FP64 integration)",
                                      "l2": ("inputs larger than L2 (%.2f GB of algorithmic traffic per step)" % (step_bytes / 1e9))
                                      if flush_buf is None else "flushed (256 MB write) before every timed step",
                                      "window": f"steps {advance}..{advance + args.steps} of the run",
                                      "ranks": "independent seeded problems per rank",
                                      "step_path": tuned},
        "bond_evals_per_s": bond_evals,
        "fp64_path": {"value": value64, "unit": "node-steps/s", "ms_per_step": 1e3 * elapsed64 / args.steps,
                      "force_kernel_us": 1e3 * float(np.mean(force64_ms)) if sim64 is not None else 1e3 * f_ms,
                      "roofline": _roof_fp64(sim64, float(np.mean(force64_ms)), tuned["fp64"], args.workload, clk, hbm)
                      if sim64 is not None else roof},
        "speedup_vs_fp64_path": value / value64,
        "roofline": roof,
        "step_roofline": {"bound": "hbm", "achieved": step_bytes / step_s / 1e9, "peak": hbm, "unit": "GB/s",
                          "frac": step_bytes / step_s / 1e9 / hbm,
                          "note": f"whole step: {step_per_node} B/node + {step_per_bond} B/bond "
                                  "(rebuilds not counted) / event-timed step (of measured)"},
        "force_kernel_us": 1e3 * f_ms,
        "list_rebuilds": {"timed_steps": args.steps, key: rebuilds,
                          **({"fp64": rebuilds64} if sim64 is not None else {}),
                          "note": "contact candidate lists (radius R_c + 0.1 R_c) rebuilt only when a node has "
                                  "moved 0.45 skin (inside the persistent kernel, or in a conditional graph node "
                                  "on the kernel-graph path)"},
        "cpu_baseline": None,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": _launches(tuned[key]["mode"], args.steps, rebuilds)
                        + (_launches(tuned["fp64"]["mode"], args.steps, rebuilds64) if sim64 is not None else 0),
        "status": int(rc),
    }
    if sim64 is not None:
        line["precision_report"] = _same_state_force_report(B, sim, sim64, w)
    if not args.no_cpu:
        line["cpu_baseline"], probs = cpu_baseline(w, advance)
        # the GPU paths at the oracle's state of the same sample
        line["oracle_parity"] = oracle_parity(B, probs, {key: sim} | ({"fp64": sim64} if sim64 is not None else {}), w)
        del probs
    del sim, sim64
    torch.cuda.empty_cache()
    if world == 1 and args.legs:
        from paper_2108_07212_gb300 import inputs as I
        from paper_2108_07212_gb300 import surrogate as SU
        legs = {}
        for name in args.legs.split(","):
            t0 = time.perf_counter()
            if name == "sequential" and getattr(w, "parts", None) is not None:
                legs[name] = leg_sequential(B, w, dev, stream, torch)
                legs[name]["speedup_batched_vs_sequential_fp32"] = value / legs[name]["sequential_fp32"]["value"]
                legs[name]["speedup_batched_vs_sequential_fp64"] = value / legs[name]["sequential_fp64"]["value"]
            elif name == "compaction":
                legs[name] = leg_compaction(B, I, dev, stream, torch, hbm, clk)
            elif name == "settling":
                legs[name] = leg_settling(B, I, dev, stream, torch)
            elif name == "surrogate":
                legs[name] = leg_surrogate(B, I, SU, dev, stream, torch)
            else:
                continue
            legs[name]["wall_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()
        line["legs"] = legs
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--legs", default="sequential,compaction,surrogate,settling",
                    help="comma-separated further workloads at N=1 ('' for none)")
    ap.add_argument("--workload", default="ensemble64", choices=sorted(WORKLOADS),
                    help="workload of the main line (ensemble64 is the benchmark configuration)")
    ap.add_argument("--advance", type=int, default=None,
                    help="untimed steps before the timed window (default: per workload; the window starts mid-run)")
    ap.add_argument("--path", default="", help="fix the step path: MODE,LANES[,BLOCK] (pd_set_path) instead of autotuning")
    ap.add_argument("--sur-profile", type=int, default=0, metavar="N",
                    help="only run N surrogate steps of the 2000-grain settling between cudaProfilerStart/Stop "
                         "(for an ncu launch list) and print their status")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.sur_profile:
        return run_surrogate_profile(args.sur_profile)
    return run_ours(args)


def run_surrogate_profile(n):
    import torch
    from paper_2108_07212_gb300 import binding as B
    from paper_2108_07212_gb300 import inputs as I
    from paper_2108_07212_gb300 import surrogate as SU
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    out = leg_surrogate(B, I, SU, dev, stream, torch, profile_steps=n)
    print(json.dumps(out))
    return 0 if out["status"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
