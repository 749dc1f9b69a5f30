#!/usr/bin/env python
"""Particle-steps/s of the weakly-compressible SPH hot path on GB300.

Workload (default): the 3D dam break at dp = 0.0025 -- tank 1.6 x 0.67 x 0.6,
water column 0.4 x 0.67 x 0.3 (160 x 268 x 120 = 5 145 600 fluid particles on a
lattice with seeded +-0.01 dp jitter), 3 open-top wall layers (1 847 172 wall
particles), Wendland C2 with h = 1.3 dp, rho0 = 1000, g = 9.81,
c0 = 10 sqrt(2 g H), mixed precision (float pair arithmetic, double state).

One bench step = sph_step(SUBSTEPS) = SUBSTEPS acoustic steps (default 10),
which always spans at least two advection steps, so every stage of the hot
path (cell keys, radix sort, reorder, cell offsets, density summation,
viscous force, both half-steps, pressure and density relaxation, time-step
reductions) runs inside every bench step.  value = fluid particles x acoustic
steps / device time, summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Inputs stay resident in HBM (about 1.5 GB of state, far above the 129 MB L2,
so no L2 flush is needed between steps).  Under torchrun (N > 1) the tank is
split into slabs along x over the ranks (strong scaling; the ranks exchange
ghost particles and reduce the velocity maximum every acoustic step, see
paper_2603_11868_gb300/slab.py); --replicas runs N independent replicas
instead (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s, 5M-particle 3D dam break, FP32-mixed vs FP64 on one GB300"
SUBSTEPS = 10

# Algorithmic bytes per fluid particle and launch of each stage's method work
# (mixed precision, 3D): every per-particle array of the method's state read
# or written once (positions and density in double, velocity with its
# compensation 24 B, pair data as one 32-byte float record per particle),
# neighbour records read once (re-reads are meant to hit L2), about 6 B of
# static wall records per fluid particle for each loop that reads walls, and
# nothing for the neighbour lists, which are this design's choice rather than
# the method's.  The first-half drift of the density stage is fused into the
# pressure kernel, so its bytes (read x and v 36, write x 24 and the records
# 32) move from the density relaxation to the pressure stage.
ALG_BYTES_PER_PARTICLE_3D = {
    "keys": 32,                 # read x 24; write key, index 8
    "sort": 60,                 # 3 passes x (key + index read and write) + histograms
    "reorder": 132,             # gather and write the state, write the records
    "offsets": 6,               # sorted keys, about 0.5 cells per particle
    "density_sum": 40,
    "viscous": 44,
    "half1": 112,               # read x 24, v 12, rho 8, drho 4; write x 24, rho 8, records 32
    "pressure": 92 + 6 + 92,    # records 32, a_prior 12, v 24 r + 24 w; walls; fused drift
    "density_relax": 52 + 6,    # records 32, drho 4, rho 8 r + 8 w; walls
    "control": 0,
}
# bytes per fluid particle this implementation's layout moves beyond the
# method's (the drift check of the lists reads the rebuild offsets and the
# budget, 16 B, wherever particles move; the key of the binned cell 4 B)
# (the fused drift re-reads no velocity, 12 B less); half1 reads the velocity
# state in double (12 B more)
LAYOUT_EXTRA_BYTES = {"pressure": 4 + 16 - 12, "density_relax": 4, "half1": 12 + 4 + 16,
                      "viscous": 4}
WALL_RECORD_BYTES_3D = 16  # one float4 per wall particle, read once per loop
# neighbour-list bytes per list entry and launch of the stages that use the
# lists: the loops read each entry once; the rebuild writes and then reads
# them once (list build + density summation)
LIST_ENTRY_BYTES = {"pressure": 4, "density_relax": 4, "viscous": 4, "density_sum": 8}


def code_only(text: str) -> str:
    """C++ source with comments and whitespace removed: what a compiled kernel
    depends on (string literals here hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return re.sub(r"\s+", "", text)


def source_fingerprint() -> str:
    """Fingerprint of the kernel sources' code (comments and layout ignored)."""
    h = hashlib.sha1()
    for f in ("sph_stages.cuh", "sph_nsearch.cu", "sph_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2603_11868_gb300", "csrc", f)) as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:12]


# Counters of one launch of the named stage from an ncu capture of a smaller
# case of the same geometry and kernel (3D dam break at dp = 0.005, 643 200
# fluid particles), keyed by the fingerprint of the kernel sources' code it was
# taken on (comments and layout ignored); a stale fingerprint reports them as
# null.  DRAM traffic is scaled
# to the bench's launch by the fluid count (traffic per particle does not
# depend on size at fixed h / dp), warp instructions by the list entries
# (nearly all instructions are spent per entry).
NCU_CAPTURES = {
    ("pressure", "5cdecf4501c5"): {"fluid": 643200, "dram_bytes": 294713088 + 22424832,
                                   "warp_inst": 134546052, "list_entries_per_particle": None},
}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 5]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[2 + k].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def apply_tuning(obj, args):
    """--tuning B,R,L sets block size, radix bits and lists directly (for
    profiling runs); otherwise the autotuner picks them (unless disabled)."""
    from paper_2603_11868_gb300 import sph
    if args.tuning:
        blk, radix, lists = (int(v) for v in args.tuning.split(","))
        obj.set_option(sph.SPH_OPT_BLOCK, blk)
        obj.set_option(sph.SPH_OPT_RADIX_BITS, radix)
        obj.set_option(sph.SPH_OPT_NEIGHBOUR_LIST, lists)
        return {"block": blk, "radix_bits": radix, "neighbour_list": lists, "trials": 0}
    if args.no_autotune:
        return None
    return sph.tune(obj, args.substeps, cache=args.tune_cache)


def replica_value(el: float, units: float, dist, device) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: the units every rank
    processed, summed, over the slowest rank's time (no collective on the data
    path; these two reductions only aggregate the measurement)."""
    if dist is None:
        return units / el, el
    import torch
    t = torch.tensor([el], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def shard_tanks(sizes, ranks: int) -> list[list[int]]:
    """Tanks of a batch dealt to ranks, largest first, each to the rank with
    the fewest particles so far; each rank's tanks in ascending order."""
    sizes = np.asarray(sizes, dtype=np.float64)
    order = np.argsort(-sizes, kind="stable")
    load = np.zeros(ranks)
    out: list[list[int]] = [[] for _ in range(ranks)]
    for t in order:
        r = int(np.argmin(load))
        out[r].append(int(t))
        load[r] += sizes[t]
    return [sorted(o) for o in out]


def make_workload(name: str, dp: float | None = None):
    from paper_2603_11868_gb300 import cases
    if dp is not None:
        return cases.dam_break_3d(dp=dp, seed=2), f"3D dam break, dp={dp}"
    if name == "dam_break_3d_5m":
        return cases.dam_break_3d(dp=0.0025, seed=2), "3D dam break, dp=0.0025"
    if name == "dam_break_3d_80k":
        return cases.dam_break_3d(dp=0.01, seed=1), "3D dam break, dp=0.01"
    if name == "dam_break_2d":
        return cases.dam_break_2d(), "2D dam break, dp=0.025"
    if name == "dam_break_obstacle_3d_56m":
        # the largest particle count of the paper's runs (dam break with an
        # obstacle, 56 M particles): 56.3 M fluid + 8.4 M wall particles
        return (cases.dam_break_obstacle_3d(dp=0.0022),
                "3D dam break with obstacle, dp=0.0022")
    raise SystemExit(f"unknown workload {name}")


def cpu_oracle_sample(seconds_cap: float = 30.0) -> dict:
    """The FP64 oracle as it stands, serial, on the host: the same 3D dam break
    at dp = 0.01 (80 400 fluid + 120 234 wall particles: same lattice, h / dp,
    wall layers and per-particle neighbour counts as the 5.1 M workload), one
    initial bin/sort + acoustic steps (with their rebuilds) until about 10 s."""
    from oracle import oracle
    from paper_2603_11868_gb300 import cases
    case = cases.dam_break_3d(dp=0.01, seed=1)
    o = oracle.Oracle.from_case(case)
    t0 = time.perf_counter()
    steps = 0
    while steps < 200:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > 10.0 or el * (steps + 1) / steps > seconds_cap:
            break
    el = time.perf_counter() - t0
    return {"value": case.n * steps / el, "unit": "particle-steps/s", "cores": 1,
            "kind": "oracle",
            "sample": f"serial FP64 oracle, 3D dam break dp=0.01 ({case.n} fluid + {case.nw} "
                      f"wall), {steps} acoustic steps incl. rebuilds, {el:.1f} s"}


def roofline_of(stage: str, launch_s: float, n: int, nw: int, list_entries: float,
                clocks: dict, mixed: bool) -> dict:
    """HBM roofline of one stage's launch from its algorithmic bytes, with the
    bytes this design adds (list entries, layout) and the ncu DRAM traffic as
    overheads, and its issue-slot roofline: warp instructions per launch over
    what the SMs can issue in the launch time (4 schedulers per SM, one warp
    instruction each per cycle, at the SM clock sampled during the run)."""
    import torch
    peaks = measured_peaks()
    alg = ALG_BYTES_PER_PARTICLE_3D.get(stage, 0) * n
    list_bytes = LIST_ENTRY_BYTES.get(stage, 0) * list_entries
    layout = LAYOUT_EXTRA_BYTES.get(stage, 0) * n
    if stage in ("density_sum", "viscous", "pressure", "density_relax"):
        layout += WALL_RECORD_BYTES_3D * nw - 6 * n   # the actual wall records vs the 6 B allowance
    achieved = alg / launch_s / 1e9
    cap = NCU_CAPTURES.get((stage, source_fingerprint())) if mixed else None
    traffic = cap["dram_bytes"] / cap["fluid"] * n if cap else None
    issue = None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clocks.get("sm_mhz") if clocks else None
    if cap and cap.get("warp_inst") and mhz:
        e_cap = cap.get("list_entries_per_particle")
        scale = (n * (list_entries / n) / (cap["fluid"] * e_cap)) if e_cap else n / cap["fluid"]
        inst = cap["warp_inst"] * scale
        slots = 4.0 * sms * mhz * 1e6 * launch_s
        issue = {"warp_inst_per_launch": inst, "sm_count": sms, "sm_mhz": mhz,
                 "issue_slots_per_launch": slots, "frac": inst / slots,
                 "scaled_by": "list entries" if e_cap else "fluid particles"}
    return {"bound": "hbm", "kernel": stage, "achieved": achieved, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "peak_source": peaks["source"], "bytes_per_launch": alg,
            "avg_launch_ms": launch_s * 1e3,
            "list_entries_per_particle": list_entries / n,
            "overhead": {"list_entry_bytes": list_bytes, "layout_extra_bytes": layout,
                         "traffic_over_algorithmic": (traffic / alg) if traffic else None},
            "issue": issue}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    warm = max(0, args.warmup)
    from oracle import oracle
    from paper_2603_11868_gb300 import cases
    case = cases.dam_break_3d(dp=0.01, seed=1)
    o = oracle.Oracle.from_case(case)
    # each reference step: one acoustic step of the sample (bounded CPU work)
    o.step(warm)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    value = case.n * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": warm,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "3D dam break (serial FP64 oracle on host cores; bounded "
                               "sample dp=0.01, 80 400 fluid + 120 234 wall)",
                   "precision": "fp64", "sample_fluid": case.n},
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"{args.steps} acoustic steps of the dp=0.01 3D dam break"},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_steps(solver, steps, substeps, torch):
    """Device time of `steps` bench steps (events on the caller's stream,
    which waits on the library's stream)."""
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        solver.step(substeps)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def measure_nsearch(steps: int, warmup: int) -> dict:
    """Neighbour-search microbenchmark: 2^24 particles uniform in the unit cube
    (seeded), h such that each particle has 57 others within 2h on average;
    cell keys + radix sort + reorder + cell offsets + one density pass, with
    float64 and float32 positions, timed per stage."""
    import torch
    from paper_2603_11868_gb300 import cases, sph

    case = cases.uniform_cube(n=1 << 24, seed=3, neighbours=57.0)
    res = {"n": case.n, "h": case.h}
    for label, dt, fp32 in (("f64", torch.float64, False), ("f32", torch.float32, True)):
        dev = [torch.tensor(np.ascontiguousarray(case.fluid[:, k]), dtype=dt, device="cuda")
               for k in range(3)]
        ns = sph.NeighbourSearch(3, case.lo, case.hi, case.h, fp32=fp32)
        for _ in range(warmup):
            ns.run(*dev, timed=False)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(st)
            for _ in range(steps):
                ns.run(*dev, timed=False)
            e1.record(st)
            e1.synchronize()
        el = e0.elapsed_time(e1) / 1e3 / steps
        stages = {k: 0.0 for k in ns.STAGES}
        for _ in range(3):
            for k, v in ns.run(*dev).items():
                stages[k] += v / 3
        res[label] = {"particles_per_s": case.n / el, "ms_per_run": el * 1e3,
                      "stage_ms": {k: round(v, 4) for k, v in stages.items()},
                      "clocks": clk.summary()}
        ns.close()
        del dev
    return res


def run_nsearch(args):
    import torch
    from paper_2603_11868_gb300 import build, sph

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    sph.load()
    res = measure_nsearch(args.steps, args.warmup)
    if rank == 0:
        line = {"metric": "neighbour-search particles/s (keys + radix sort + reorder + offsets "
                          "+ density pass), 16M uniform",
                "value": res["f32"]["particles_per_s"], "unit": "particles/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": res["f32"]["ms_per_run"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 positions",
                "data": "synthetic",
                "config": {"workload": f"uniform cube, {res['n']} particles, h={res['h']:.6g}, "
                                       f"{57} neighbours within 2h on average",
                           "l2": "inputs larger than L2 (no flush)"},
                "f32": res["f32"], "f64": res["f64"], "clocks": res["f32"]["clocks"]}
        print(json.dumps(line), flush=True)
    return 0


def batched_cases(n_tanks: int = 256, dp: float = 0.01):
    """256 independent 2D dam-break tanks, fluid counts log-uniform in
    [1 000, 64 000] (seeded), dp = 0.01, 4 wall layers each."""
    from paper_2603_11868_gb300 import cases
    sizes = cases.batched_tank_sizes(n_tanks, seed=4)
    return [cases.batched_tank(n, dp=dp, seed=100 + k) for k, n in enumerate(sizes)]


def measure_batched(args, steps: int, warmup: int, dist=None, rank: int = 0, ws: int = 1,
                    local: int = 0) -> dict:
    """Batched tanks: every tank advances one acoustic step (its own length)
    per graph launch; value = total fluid particles x acoustic steps / time."""
    import torch
    from paper_2603_11868_gb300 import sph

    cs = batched_cases(args.tanks)
    n_all = sum(c.n for c in cs)
    if ws > 1:  # independent tanks: each rank advances its share, no collective
        cs = [cs[t] for t in shard_tanks([c.n for c in cs], ws)[rank]]
    b = sph.Batch(cs, precision=args.precision)
    n, nw = b.n, b.nw
    tuning = apply_tuning(b, args)
    for _ in range(warmup):
        b.step(args.substeps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        el = time_steps(b, steps, args.substeps, torch)
    sph.sph_batch_synchronize(b.b, 60.0)
    value, el = replica_value(el, n * steps * args.substeps, dist, "cuda")
    stages, rebuilds = b.profile(2 * args.substeps)
    per_step = {k: v / (2 * args.substeps) for k, v in stages.items()}
    kernels = sph.sph_batch_kernels_per_step(b.b)
    sc = b.scalars()
    b.close()
    return {"value": value, "unit": "particle-steps/s", "ms_per_step": el / steps * 1e3,
            "steps": steps, "warmup": warmup, "n_all": n_all, "tanks_rank0": len(cs),
            "fluid_rank0": n, "wall_rank0": nw,
            "acoustic_steps_per_bench_step": args.substeps,
            "stage_ms_per_acoustic_step": {k: round(v, 4) for k, v in per_step.items()},
            "advection_steps_begun_per_acoustic_step": rebuilds / (2 * args.substeps),
            "gpu_launches": kernels * args.substeps * steps,
            "kernels_per_acoustic_step": kernels,
            "tank_time_spread": [float(np.min(sc["t"])), float(np.max(sc["t"]))],
            "tuning": tuning, "clocks": clk.summary()}


def run_batched(args):
    import torch
    from paper_2603_11868_gb300 import build, sph

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    sph.load()
    r = measure_batched(args, args.steps, args.warmup, dist, rank, ws, local)
    if rank == 0:
        line = {"metric": "particle-steps/s, 256 batched 2D dam-break tanks (1k-64k particles "
                          "each), FP32-mixed",
                "value": r["value"], "unit": "particle-steps/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 pair / f64 state" if args.precision == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": f"{args.tanks} tanks, {r['n_all']} fluid particles over "
                                       f"{ws} rank(s) (rank 0: {r['tanks_rank0']} tanks, "
                                       f"{r['fluid_rank0']} fluid + {r['wall_rank0']} wall), "
                                       f"dp=0.01, {args.substeps} acoustic steps per bench step",
                           "parallelism": f"tanks sharded over {ws} rank(s)",
                           "l2": "state larger than L2 (no flush)"}}
        line.update({k: r[k] for k in ("acoustic_steps_per_bench_step",
                                       "stage_ms_per_acoustic_step",
                                       "advection_steps_begun_per_acoustic_step", "gpu_launches",
                                       "kernels_per_acoustic_step", "tank_time_spread", "tuning",
                                       "clocks")})
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_slab(args):
    """The headline workload as one tank split into slabs along x over the N
    ranks (paper_2603_11868_gb300/slab.py): each rank advances its own
    particles and ghost copies of its neighbours'; after every acoustic step
    the ranks all-reduce the velocity maximum and refresh the ghosts, and at
    every advection-step boundary they hand over the particles that changed
    slab.  value = the tank's fluid particles x acoustic steps / the slowest
    rank's time: strong scaling (the total work is fixed)."""
    import torch
    import torch.distributed as dist
    from paper_2603_11868_gb300 import build, slab, sph

    ws, rank, local = dist_env()
    ndev = torch.cuda.device_count()
    torch.cuda.set_device(local % ndev)
    backend = args.slab_backend
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=torch.device("cuda", local % ndev))
        device = f"cuda:{local % ndev}"
    else:
        dist.init_process_group("gloo")
        device = "cpu"
    build.build()
    sph.load()
    case, wname = make_workload(args.workload, args.dp)
    n, nw = case.n, case.nw
    t_e0 = time.perf_counter()
    eng = slab.LibraryEngine(case, args.precision, device_rows=backend == "nccl")
    r = slab.SlabRank(case, rank, ws, eng)
    setup_s = time.perf_counter() - t_e0
    slab.run_distributed(r, args.warmup * args.substeps, dist, device)
    torch.cuda.synchronize()
    dist.barrier()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local % ndev) as clk:
        e0.record(st)
        slab.run_distributed(r, args.steps * args.substeps, dist, device)
        e1.record(st)
        e1.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    t = torch.tensor([el], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    el = float(t.item())
    acoustic = args.steps * args.substeps
    value = n * acoustic / el
    # end to end: the set-up that uploads this rank's particles, the steps, and
    # the owned state read back to the host
    t_b = time.perf_counter()
    slab.run_distributed(r, args.substeps, dist, device)
    gid, own = r.owned_state()
    torch.cuda.synchronize()
    e2e_s = setup_s + (time.perf_counter() - t_b) * args.steps
    t = torch.tensor([e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_s = float(t.item())
    counts = torch.tensor([r.n_own, r.n_gl + r.n_gr], dtype=torch.float64, device=device)
    tot = counts.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    kps = sph.sph_kernels_per_step(eng.ctx)
    eng.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": f"{wname}: {n} fluid + {nw} wall particles, "
                                   f"{args.substeps} acoustic steps per bench step",
                       "precision": args.precision, "fluid_particles": n,
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"slabs along x over {ws} ranks, halo "
                                      f"{slab.HALO_CELLS} cells, {backend}"},
            "slabs": {"cuts": [float(c) for c in r.cuts[1:-1]],
                      "ghosts_over_owned": float(tot[1].item() / tot[0].item())},
            "e2e": {"value": n * acoustic / e2e_s, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": "set-up upload and final owned-state read, amortised over the "
                            "timed steps"},
            "gpu_launches": int(kps * acoustic) if kps > 0 else None,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    from paper_2603_11868_gb300 import build, sph

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    sph.load()
    case, wname = make_workload(args.workload, args.dp)
    solver = sph.Solver(case, precision=args.precision)
    n, nw = case.n, case.nw
    # launch configuration picked by the library's autotuner (trials run from a
    # snapshot that is restored afterwards, before the warm-up)
    tuning = apply_tuning(solver, args)
    mean_nb = None
    if rank == 0 and not args.quick:
        cf, cw, _ = solver.neighbour_stats()
        mean_nb = float(cf.mean() + cw.mean())
    for _ in range(args.warmup):
        solver.step(args.substeps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        el = time_steps(solver, args.steps, args.substeps, torch)
    acoustic = args.steps * args.substeps
    value, el = replica_value(el, n * acoustic, dist, "cuda")
    if dist:
        dist.barrier()
    clocks = clk.summary()
    kps = solver.kernels_per_step()
    sc = solver.scalars()

    # per-stage device times (stage-by-stage launches with events on the
    # library stream; the state keeps advancing) -> dominant kernel roofline
    prof_steps = 2 * args.substeps
    ms, rebuilds = solver.profile_stages(prof_steps)
    per_step = {k: v / prof_steps for k, v in ms.items()}
    rebuild_stages = ("keys", "sort", "reorder", "offsets", "density_sum", "viscous")
    launches = {k: (rebuilds if k in rebuild_stages else prof_steps) for k in ms}
    dom = max(ms, key=lambda k: ms[k])
    list_entries = float(solver.list_lengths().astype(np.float64).sum())
    roofline = roofline_of(dom, ms[dom] / 1e3 / max(1, launches[dom]), n, nw, list_entries,
                           clocks, args.precision == "mixed")

    # FP64 path on the same workload for the speed-up (fewer steps)
    fp64 = None
    if args.precision == "mixed" and not args.quick and rank == 0:
        s64 = sph.Solver(case, precision="fp64")
        s64.step(args.substeps)
        el64 = time_steps(s64, args.fp64_steps, args.substeps, torch)
        fp64 = n * args.fp64_steps * args.substeps / el64
        s64.close()

    # end to end through the C ABI: pinned host input -> set_particles ->
    # sph_step -> sph_get_fields -> pinned host output, every bench step
    e2e = None
    if not args.quick:
        d = case.dim
        pin_in = {k: torch.empty(sh, dtype=torch.float64, pin_memory=True).numpy()
                  for k, sh in (("pos", (n, d)), ("vel", (n, d)), ("rho", (n,)))}
        pin_in["pos"][:] = case.fluid
        pin_in["vel"][:] = 0.0
        pin_in["rho"][:] = case.rho0
        outbuf = torch.empty(n * (2 * d + 1), dtype=torch.float64, pin_memory=True).numpy()
        L = sph.load()
        mask = sph.SPH_F_POS | sph.SPH_F_VEL | sph.SPH_F_RHO
        ptr = lambda a: a.ctypes.data  # noqa: E731
        e2e_steps = max(2, args.steps // 5)

        def e2e_step():
            rc = L.sph_set_particles(solver.ctx, sph.SPH_FLUID, n, ptr(pin_in["pos"]),
                                     ptr(pin_in["vel"]), ptr(pin_in["rho"]))
            rc = rc or L.sph_step(solver.ctx, args.substeps)
            rc = rc or L.sph_get_fields(solver.ctx, mask, ptr(outbuf))
            if rc:
                raise RuntimeError(f"e2e step failed: {rc} {sph.sph_last_error(solver.ctx)}")

        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        el_e2e = time.perf_counter() - t0
        if dist:
            t = torch.tensor([el_e2e], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el_e2e = float(t.item())
        e2e = {"value": ws * n * e2e_steps * args.substeps / el_e2e, "unit": "particle-steps/s",
               "h2d_bytes_per_step": n * (2 * d + 1) * 8,
               "d2h_bytes_per_step": n * (2 * d + 1) * 8}

    solver.close()
    # the batched-tank and neighbour-search workloads, timed after the headline
    # on one GPU (their own values, clocks and times; not part of `value`)
    extras = {}
    if ws == 1 and not args.quick and not args.no_extras:
        torch.cuda.empty_cache()
        b = measure_batched(args, steps=20, warmup=3, local=local)
        extras["batched_256"] = {
            "metric": "particle-steps/s, 256 batched 2D dam-break tanks (1k-64k particles "
                      "each), FP32-mixed", "fluid_particles": b["n_all"],
            **{k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup",
                                 "acoustic_steps_per_bench_step", "kernels_per_acoustic_step",
                                 "gpu_launches", "tuning", "clocks")}}
        torch.cuda.empty_cache()
        ns = measure_nsearch(steps=5, warmup=3)
        extras["nsearch_16m"] = {
            "metric": "neighbour-search particles/s (keys + radix sort + reorder + offsets + "
                      "density pass), 16M uniform, float positions",
            "value": ns["f32"]["particles_per_s"], "unit": "particles/s",
            "ms_per_step": ns["f32"]["ms_per_run"], "steps": 5, "warmup": 3,
            "stage_ms": ns["f32"]["stage_ms"], "clocks": ns["f32"]["clocks"],
            "f64": {"value": ns["f64"]["particles_per_s"], "ms_per_step": ns["f64"]["ms_per_run"],
                    "stage_ms": ns["f64"]["stage_ms"]}}
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.quick and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": f"{wname}: {n} fluid + {nw} wall particles, "
                                   f"{args.substeps} acoustic steps per bench step",
                       "precision": args.precision, "fluid_particles": n,
                       "wall_particles": nw, "acoustic_steps_timed": acoustic,
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline,
            "stage_ms_per_step": {k: round(v, 4) for k, v in per_step.items()},
            "rebuilds_per_step": rebuilds / prof_steps,
            "clocks": clocks,
            # 4 kernels every step, the rest of the step's kernels in the steps
            # that begin an advection step (the graph's conditional node)
            "gpu_launches": int(round(acoustic * (4 + (kps - 4) * rebuilds / prof_steps)))
            if kps > 0 else None,
            "kernels_per_acoustic_step": kps,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fp64_value": fp64,
            "speedup_vs_fp64": (value / ws / fp64) if fp64 else None,
            "gpips": (value * mean_nb * 2 / 1e9) if mean_nb else None,
            # the same throughput counting wall particles too
            "fluid_and_wall_steps_per_s": value * (n + nw) / n,
            "sim_time": sc["t"], "source_fingerprint": source_fingerprint(), "tuning": tuning,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="dam_break_3d_5m",
                    choices=["dam_break_3d_5m", "dam_break_3d_80k", "dam_break_2d",
                             "dam_break_obstacle_3d_56m", "nsearch_16m", "batched_256"])
    ap.add_argument("--dp", type=float, default=None,
                    help="3D dam break at this spacing instead of the named workload")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--substeps", type=int, default=SUBSTEPS)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="main number only")
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1 ranks, N independent replicas instead of one tank split "
                         "into slabs")
    ap.add_argument("--slab-backend", choices=["nccl", "gloo"], default="nccl",
                    help="transport of the slab split: nccl (device rows) or gloo (host "
                         "arrays; ranks may share a GPU)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-tank and neighbour-search lines nested in the default line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch configuration")
    ap.add_argument("--tanks", type=int, default=256,
                    help="tank count of the batched workload (the bench line is 256)")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of autotuner choices keyed by GPU and problem (reused "
                         "when present, written after tuning)")
    ap.add_argument("--tuning", default=None,
                    help="block,radix_bits,lists: fixed launch configuration, no autotuner")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "nsearch_16m":
        return run_nsearch(args)
    if args.workload == "batched_256":
        return run_batched(args)
    if dist_env()[0] > 1 and not args.replicas:
        return run_slab(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
