#!/usr/bin/env python
"""Benchmark of the GB300 SPH-IDIC step: gas+dust particle-updates per second.

Default workload: the 3D periodic box, 128^3 gas + 128^3 dust particles
(4,194,304 in total), h = 1.2 dx (about 58 neighbours), 128^3 cells,
t_stop = 1e-4, FP32 state and pair sums with FP32 cell sums. A step is one
full pass of the path (binning, density, force, implicit cell drag, update).
The default times the workload's 100-step run (after 5 warm-up steps): the
particles leave their initial lattice as the run goes on and the pair sums
slow down with the disorder, so a shorter window would flatter the step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload box3d|dustyshock|column2d]
                  [--impl ours|reference] [--cell-acc fp32|fp64] [--part all|isph|mk|batch]
                  [--no-cpu-baseline] [--no-e2e] [--no-clocks] [--no-adjoint] [--no-batch]
                  [--no-schemes] [--no-fp64-cells]

``--part`` runs one part alone (one drag scheme, or the batched ensemble) and
prints its object: a short program for profiling that part's kernels.

Prints one JSON line (rank 0). Timed region: barrier + synchronize on both
sides, CUDA events on the library's stream, max over ranks. The state of the
default workload (~300 MB per step of traffic) is larger than L2, so L2 is not
flushed. N > 1 runs one independent replica per GPU (weak scaling; the step
has no data-path collective). ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "gas+dust particle-updates/s per TFSPH step; % HBM roofline; adjoint/fwd time"
UNIT = "particle-updates/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["box3d", "dustyshock", "column2d"], default="box3d")
    ap.add_argument("--cell-acc", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-schemes", action="store_true")
    ap.add_argument("--no-fp64-cells", action="store_true")
    ap.add_argument("--part", choices=["all", "isph", "mk", "batch"], default="all",
                    help="run one part alone (one drag scheme, or the batched ensemble) and print its "
                         "object: a short program for profiling that part's kernels")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# Distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend: str):
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend, rank=self.rank, world_size=self.world)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if self.pg is None:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.pg is None:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def make_workload(name: str, scale: int = 0):
    import workloads
    if name == "box3d":
        nside = scale or 128
        w = workloads.box3d(nside=nside, precision=0)
        desc = (f"3D periodic box [0,1)^3, {nside}^3 gas + {nside}^3 dust, Gaussian random velocity "
                f"fields (k^-2, rms 0.1 cs), h=1.2dx (~58 neighbours), {nside}^3 cells, t_stop=1e-4")
    elif name == "dustyshock":
        nl = scale or 177778
        w = workloads.dustyshock(n_left=nl, n_right=max(1, nl // 8), precision=0)
        desc = (f"1D dusty Sod shock tube with walls, {w.n_gas} gas (incl. frozen walls) + {w.n_dust} dust, "
                f"rho 1/0.125, p 1/0.1, gamma 1.4, dust-to-gas 1, t_stop log-uniform 1e-5..1, cell 2h")
    else:
        nside = scale or 512
        w = workloads.column2d(nside=nside, precision=0)
        desc = (f"2D dust settling column, {nside}^2 gas (+ frozen walls) + {nside}^2 dust, g=(0,-1), "
                f"t_stop log-uniform 1e-3..1e-1, cell 2h")
    return w, desc


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: str):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.dev, f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        smax.append(float(parts[2]))
                    except ValueError:
                        continue
                    for nm, val in zip(names, parts[5:9]):
                        if val.lower() == "active":
                            reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# Roofline bookkeeping (algorithmic bytes / flops per phase)
# ---------------------------------------------------------------------------
def algorithmic(phase: str, w, info, nb_mean: float) -> tuple[str, float]:
    """(bound, algorithmic bytes or flops of one launch of the phase's kernel).

    Bytes count each array the kernel must touch once (FP32 state: V4 = 16 B);
    flops count neighbour pairs only (density 20, force 35 flops per pair).
    """
    ng, nd = w.n_gas, w.n_dust
    n = ng + nd
    nc = info.n_cells_total
    if phase == "count":
        return "hbm", 4.0 * n + 2 * 8.0 * nc
    if phase == "scan":
        return "hbm", 2 * (4.0 + 4.0 + 4.0) * nc
    if phase == "scatter":
        return "hbm", 16.0 * n + 2 * 12.0 * nc
    if phase == "gather":
        return "hbm", 84.0 * n
    if phase == "drag":
        return "hbm", (16 + 16 + 16 + 16 + 16 + 4) * ng + (16 + 16 + 16 + 16 + 4) * nd + 2 * 8.0 * nc
    if phase == "density":
        return "alu", 20.0 * nb_mean * ng
    if phase == "force":
        return "alu", 35.0 * nb_mean * ng
    raise ValueError(phase)


def step_model_bytes(w, info) -> float:
    """Algorithmic bytes of one step (FP32 state): sort 16 B, gather 56 B (gas)
    or 64 B (dust), density 16 B (gas), force + drag + update + next key 56 B
    per particle-update, plus the cell ranges of both phases (start and end,
    4 B each, per cell). Each of the step's three global dependencies (binning
    -> density -> force and drag) costs one round trip through HBM; reuse of
    neighbour data from shared memory or L2 is not counted."""
    return 144.0 * w.n_gas + 136.0 * w.n_dust + 2 * 2 * 4.0 * info.n_cells_total


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


_BIN = ("bin.cu", "sort_ops.cuh")
_PAIR = ("sph.cu", "pair.cuh")
PHASE_SOURCE = {"count": _BIN, "scan": _BIN, "scatter": _BIN, "gather": _BIN,
                "density": _PAIR, "force": _PAIR, "drag": ("drag.cu", "drag_ops.cuh")}


def kernel_source_hash(phase: str) -> str:
    """sha256 of the phase's kernel sources and the shared internal header,
    without comments and blank space: an edit of the comments alone leaves
    the recorded counters valid, any change of the code does not."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1908_01682_gb300", "csrc")
    hsh = hashlib.sha256()
    for f in PHASE_SOURCE[phase] + ("tfsph_internal.cuh",):
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        hsh.update(" ".join(src.split()).encode())
    return hsh.hexdigest()


def recorded_traffic(workload: str, phase: str):
    """DRAM bytes (read + write) per launch of the phase's kernel from the
    committed ncu summary, or None when absent or taken on other source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        ent = rec[workload][phase]
    except (OSError, ValueError, KeyError):
        return None
    if ent.get("source_sha256") != kernel_source_hash(phase):
        return None
    return float(ent["dram_bytes_per_launch"])


def fp32_alu_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 FMA pipes: 128 lanes per SM, 2 flops per FMA."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands
# ---------------------------------------------------------------------------
def oracle_sample(workload: str, scale: int):
    import oracle
    w, desc = make_workload(workload, scale)
    q = w.params
    p = oracle.Params(dim=q["dim"], lo=q["lo"], hi=q["hi"], periodic=q["periodic"], h=q["h"],
                      cell_size=q["cell_size"], m_gas=q["m_gas"], m_dust=q["m_dust"], eos=q["eos"],
                      cs=q["cs"], gamma=q["gamma"], av_alpha=q["av_alpha"], av_beta=q["av_beta"],
                      tstar_mode=q["tstar_mode"], path_fp32=1)
    s = oracle.make_state(p, w.gx, w.gv, w.dx, w.du, w.tstop, ge=w.ge, frozen=w.frozen)
    return oracle, p, s, w, desc


def cpu_baseline(workload: str, scale: int, single_scale: int) -> tuple[dict, tuple]:
    """The oracle timed on all host cores (one step of the workload itself)
    and on one core (one step of a smaller sample of the same workload).
    Also returns the all-core step's inputs and results, for the per-field
    errors of the GPU step."""
    oracle, p, s, w, desc = oracle_sample(workload, scale)
    oracle.build()
    cores = oracle.set_threads(oracle.omp_threads())
    t0 = time.perf_counter()
    r = oracle.step(p, s, w.tau, w.g)
    dt = time.perf_counter() - t0
    n = w.n_gas + w.n_dust
    out = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"1 FP64 oracle step of {desc} ({n} particles), {dt:.2f} s wall, {cores} threads"}
    _, p1, s1, w1, desc1 = oracle_sample(workload, single_scale)
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.step(p1, s1, w1.tau, w1.g)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    n1 = w1.n_gas + w1.n_dust
    out["single_thread"] = {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"1 FP64 oracle step of {desc1} ({n1} particles), {dt1:.2f} s wall"}
    return out, (oracle, p, s, r, w)


def field_errors(b, ctx_params, orc_run) -> dict:
    """Normwise error, ||x - x_ref|| / ||x_ref||, of every field of one GPU
    step of the workload against the oracle's step from the same inputs
    (densities before the step; positions as minimum images on periodic axes)."""
    import numpy as np

    oracle, p, s, r, w = orc_run
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    with b.Context(ctx_params, f32(w.gx), f32(w.gv), f32(w.dx), f32(w.du), f32(w.tstop), ge=f32(w.ge),
                   frozen=w.frozen) as c:
        rho_g = c.field(b.TFSPH_FIELD_RHO_G).astype(np.float64)
        rho_d = c.field(b.TFSPH_FIELD_RHO_D).astype(np.float64)
        c.step(w.tau, w.g)
        got = {k: c.field(f).astype(np.float64) for k, f in
               (("x_g", b.TFSPH_FIELD_POS_G), ("v_g", b.TFSPH_FIELD_VEL_G), ("x_d", b.TFSPH_FIELD_POS_D),
                ("u_d", b.TFSPH_FIELD_VEL_D))}
    ref_rho_d = oracle.density(p, w.dx, p.m_dust)[0]

    def nw(a, ref, pos=False):
        d = np.asarray(a, np.float64) - np.asarray(ref, np.float64)
        if pos:
            for k in range(w.dim):
                if w.params["periodic"][k]:
                    L = w.params["hi"][k] - w.params["lo"][k]
                    d[k] -= L * np.round(d[k] / L)
        return float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))

    return {"rho_g": nw(rho_g, r.rho_g), "rho_d": nw(rho_d, ref_rho_d), "x_g": nw(got["x_g"], s.gx, True),
            "v_g": nw(got["v_g"], s.gv), "x_d": nw(got["x_d"], s.dx, True), "u_d": nw(got["u_d"], s.du),
            "metric": "normwise ||gpu - oracle|| / ||oracle|| after one step from the workload's inputs"}


def run_reference(args, dist: Dist):
    """The oracle timed as the reference arm (rank 0 only)."""
    if dist.rank != 0:
        return
    scale = {"box3d": 48, "dustyshock": 20000, "column2d": 128}[args.workload]
    oracle, p, s, w, desc = oracle_sample(args.workload, scale)
    oracle.build()
    for _ in range(args.warmup):
        oracle.step(p, s, w.tau, w.g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(p, s, w.tau, w.g)
    dt = time.perf_counter() - t0
    n = w.n_gas + w.n_dust
    value = n * args.steps / dt
    cores = oracle.omp_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": desc, "particles": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed FP64 oracle steps of {desc}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def run_ours(args, dist: Dist):
    import numpy as np
    import torch

    from paper_1908_01682_gb300 import binding as b

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device; the GPU path has no CPU fallback")
    torch.cuda.set_device(dist.local_rank % torch.cuda.device_count())
    if args.part != "all":
        out = run_batch(b, args) if args.part == "batch" else run_schemes(b, args, only=args.part)
        if dist.rank == 0:
            print(json.dumps({"part": args.part, "result": out}), flush=True)
        return
    visible = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    dev_index = visible[dist.local_rank % len(visible)] if visible else str(torch.cuda.current_device())

    w, desc = make_workload(args.workload)
    cell_acc = b.TFSPH_CELL_ACC_FP32 if args.cell_acc == "fp32" else b.TFSPH_CELL_ACC_FP64
    p = b.params_from_dict(w.params, cell_acc=cell_acc)
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    ctx = b.Context(p, f32(w.gx), f32(w.gv), f32(w.dx), f32(w.du), f32(w.tstop), ge=f32(w.ge), frozen=w.frozen)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    info = ctx.info()
    n = w.n_gas + w.n_dust

    # neighbour statistics of the input (for the algorithmic flop count)
    nb_mean = float(np.mean(ctx.debug(b.TFSPH_DEBUG_NEIGH_COUNT))) if w.n_gas else 0.0

    # warm-up; the state before the last warm-up step is kept so that the
    # profiled pass below replays exactly the timed steps (a snapshot carries
    # its state's binning, density and force, which that last warm-up step
    # consumes, so the timed region starts from a plain state)
    for _ in range(max(0, args.warmup - 1)):
        ctx.step(w.tau, w.g)
    snap = ctx.save_state()
    ctx.step(w.tau, w.g)
    torch.cuda.synchronize()

    # ---- timed region (headline) ----
    clocks = Clocks(dev_index)
    if not args.no_clocks:
        clocks.start()
    launches0 = ctx.info().launches
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.step(w.tau, w.g)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop() if not args.no_clocks else {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
    launches = ctx.info().launches - launches0
    ctx.sync()
    ms_total_max = dist.max(ms_total)
    ms_per_step = ms_total_max / args.steps
    value = dist.sum(n * args.steps) / (ms_total_max / 1e3)

    # ---- profiled pass over the same steps: per-phase CUDA events on the same stream ----
    ctx.load_state(snap)
    ctx.step(w.tau, w.g)
    del snap
    ctx.profile(True)
    for _ in range(args.steps):
        ctx.step(w.tau, w.g)
    phase_ms, psteps, _ = ctx.profile_read()
    ctx.profile(False)
    phase_avg = {k: v / max(1, psteps) for k, v in phase_ms.items()}
    dominant = max(phase_avg, key=phase_avg.get)
    bound, amount = algorithmic(dominant, w, info, nb_mean)
    pk, pk_src = peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    if bound == "hbm":
        achieved = amount / (phase_avg[dominant] * 1e-3) / 1e9
        peak = float(pk.get("hbm_gbs", 6800.0))
        unit = "GB/s"
    else:
        # the clock the pair kernels ran at; without samples, the maximum SM
        # clock (the peaks file's clock under load is that of a power-capped
        # GEMM, lower than an FP32 ALU kernel runs at)
        mhz, mhz_src = clk.get("sm_mhz"), "SM clock sampled during the timed steps"
        if not mhz:
            mhz, mhz_src = float(pk.get("sm_max_mhz", 2070.0) or 2070.0), "maximum SM clock (clocks not sampled)"
        achieved = amount / (phase_avg[dominant] * 1e-3) / 1e12
        peak = fp32_alu_peak_tflops(sm_count, mhz)
        unit = "TFLOP/s"
    step_bytes = step_model_bytes(w, info)
    roof = {"kernel": dominant, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": recorded_traffic(args.workload, dominant),
            "peak_source": pk_src if bound == "hbm" else
            f"derived: 128 FP32 FMA lanes x 2 flops x {sm_count} SMs x {mhz:.0f} MHz ({mhz_src})",
            "step_hbm_frac": (step_bytes / (ms_per_step * 1e-3) / 1e9) / float(pk.get("hbm_gbs", 6800.0)),
            "step_algorithmic_bytes": step_bytes,
            "step_model": "144 B per gas + 136 B per dust particle-update + 2 phases x 2 x 4 B per cell"}

    # ---- the same run with FP64 cell sums and drag factors (the precision mode
    # that keeps the stiff limit); the headline above uses the FP32 cell sums
    # of this workload's configuration ----
    cells_fp64 = None
    if cell_acc == b.TFSPH_CELL_ACC_FP32 and not args.no_fp64_cells:
        p64 = b.params_from_dict(w.params, cell_acc=b.TFSPH_CELL_ACC_FP64)
        with b.Context(p64, f32(w.gx), f32(w.gv), f32(w.dx), f32(w.du), f32(w.tstop), ge=f32(w.ge),
                       frozen=w.frozen) as c64:
            c64.set_stream(stream)
            for _ in range(args.warmup):
                c64.step(w.tau, w.g)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                c64.step(w.tau, w.g)
            e1.record(stream)
            torch.cuda.synchronize()
            c64.profile(True)
            for _ in range(min(args.steps, 10)):
                c64.step(w.tau, w.g)
            pm, ps, _ = c64.profile_read()
        cells_fp64 = {"ms_per_step": e0.elapsed_time(e1) / args.steps,
                      "drag_ms": pm.get("drag", 0.0) / max(1, ps),
                      "note": "same steps with FP64 cell sums, slip and drag factors (cell_acc FP64)"}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(b, ctx, w, args, dist)

    adj = None
    if not args.no_adjoint:
        adj = run_adjoint(b, args)

    batch = None
    if not args.no_batch:
        batch = run_batch(b, args)

    schemes = None
    if not args.no_schemes:
        schemes = run_schemes(b, args)

    cpu = None
    errors = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        single = {"box3d": 48, "dustyshock": 40000, "column2d": 128}[args.workload]
        cpu, orc_run = cpu_baseline(args.workload, 0, single)
        errors = field_errors(b, p, orc_run)
        del orc_run

    ctx.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n_gas": w.n_gas, "n_dust": w.n_dust,
                   "cells": int(info.n_cells_total), "cell_sums": args.cell_acc, "tau": w.tau,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{dist.world}"},
        "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
        "roofline": roof,
        "kernel_ms": {k: round(v, 5) for k, v in phase_avg.items()},
        "cell_sums_fp64": cells_fp64,
        "adjoint": adj,
        "batched": batch,
        "drag_schemes": schemes,
        "cpu_baseline": cpu,
        "errors": errors,
    }
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def run_adjoint(b, args):
    """Adjoint cost on the settling column (512^2 gas + 512^2 dust, FP32):
    loss = squared error of the final binned dust density (64 x 64 bins,
    cloud in cell) against a seeded target profile after 500 steps
    checkpointed every 50, gradients with respect to the per-particle t_stop
    and the initial velocities. Forward = the rollout with its checkpoints and
    the loss; backward = the loss gradient, the per-segment recompute and the
    step adjoints. CUDA events on the library's stream around each."""
    import numpy as np
    import torch

    from paper_1908_01682_gb300 import adjoint

    w, desc = make_workload("column2d")
    p = b.params_from_dict(w.params)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    nsteps, every, nb = 500, 50, (64, 64)
    stream = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    with b.Context(p, f32(w.gx), f32(w.gv), f32(w.dx), f32(w.du), f32(w.tstop), frozen=w.frozen) as c:
        c.set_stream(stream)
        dev = lambda a: torch.tensor(f32(a), device="cuda")
        grid = adjoint.profile_grid(c, nb)
        rho0 = adjoint.dust_profile(grid, dev(w.dx))
        rng = np.random.default_rng(8)
        target = rho0 * torch.tensor(1.0 + 0.1 * rng.standard_normal(rho0.numel()), device="cuda")
        roll = adjoint.Rollout(c, w.tau, w.g, nsteps, checkpoint_every=every, frozen=w.frozen)

        def forward_backward(timed):
            ts = dev(w.tstop).requires_grad_()
            gv0 = dev(w.gv).requires_grad_()
            du0 = dev(w.du).requires_grad_()
            gx0, dx0 = dev(w.gx), dev(w.dx)
            torch.cuda.synchronize()
            if timed:
                e0.record(stream)
            _, _, dxf, _ = adjoint.TFSPHRollout.apply(ts, gv0, du0, roll, gx0, dx0)
            loss = adjoint.DustProfileLoss.apply(dxf, target, grid)
            if timed:
                e1.record(stream)
            loss.backward()
            if timed:
                e2.record(stream)
            torch.cuda.synchronize()
            return float(loss), ts.grad, gv0.grad, du0.grad

        forward_backward(False)  # warm-up of both directions (allocates the snapshot buffers)
        loss, gts, ggv, gdu = forward_backward(True)
        fwd, bwd = e0.elapsed_time(e1), e1.elapsed_time(e2)
        finite = bool(torch.isfinite(gts).all() and torch.isfinite(ggv).all() and torch.isfinite(gdu).all())
    return {"workload": desc, "steps": nsteps, "checkpoint_every": every,
            "loss": "squared error of the 64 x 64 cloud-in-cell dust density after the rollout vs a seeded target",
            "gradients": "d loss / d t_stop (per particle), d loss / d initial gas and dust velocities",
            "forward_ms": fwd, "backward_ms": bwd, "ratio": bwd / fwd, "loss_value": loss,
            "gradients_finite": finite,
            "timing": "CUDA events on the library's stream; forward includes the checkpoints and the loss"}


def run_batch(b, args):
    """Batched ensemble: 256 independent 1D dusty waves of 1k-64k particles
    each (log-uniform sizes, t_stop and amplitudes), stepped as one batch in
    its autotuned launch form (graph replay), against the same instances
    stepped one single context after another on the same stream. CUDA events
    on that stream around each timed loop."""
    import types

    import numpy as np
    import torch

    import workloads

    stream = torch.cuda.current_stream()
    ws = workloads.ensemble1d(precision=0)
    cell_acc = b.TFSPH_CELL_ACC_FP32 if args.cell_acc == "fp32" else b.TFSPH_CELL_ACC_FP64
    taus = [w.tau for w in ws]
    ng = sum(w.n_gas for w in ws)
    nd = sum(w.n_dust for w in ws)
    n = ng + nd
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    items = [(b.params_from_dict(w.params, cell_acc=cell_acc), w.gx, w.gv, w.dx, w.du, w.tstop) for w in ws]
    bsteps, lsteps = 100, 10
    forms = {}
    with b.Batch(items, stream=stream) as bt:
        bt.step(taus, nsteps=0)
        # every launch form at 256 threads, timed from the same state (the
        # autotuner below restores the state it found)
        for name, mode, bps in (("kernels", b.TFSPH_BATCH_KERNELS, 1), ("tiled", b.TFSPH_BATCH_TILED, 1),
                                ("persistent", b.TFSPH_BATCH_PERSISTENT, 4)):
            bt.config(mode, 256, bps)
            bt.step(nsteps=2)
            forms[name] = timed(lambda k: bt.step(nsteps=k), 10)
        bt.sync()
        bt.close()
    with b.Batch(items, stream=stream) as bt:
        bt.step(taus, nsteps=0)
        pick = bt.autotune(steps=10)
        bt.step(nsteps=args.warmup)
        launches0 = bt.info().launches
        batched_ms = timed(lambda k: bt.step(nsteps=k), bsteps)
        info = bt.info()
        bt.sync()
        ncells = int(info.n_cells)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    ctxs = []
    try:
        for w in ws:
            c = b.Context(b.params_from_dict(w.params, cell_acc=cell_acc), f32(w.gx), f32(w.gv), f32(w.dx),
                          f32(w.du), f32(w.tstop))
            c.set_stream(stream)
            ctxs.append(c)

        def looped(k):
            for _ in range(k):
                for c, w in zip(ctxs, ws):
                    c.step(w.tau, w.g)

        looped(args.warmup)
        looped_ms = timed(looped, lsteps)
    finally:
        for c in ctxs:
            c.close()
    wsum = types.SimpleNamespace(n_gas=ng, n_dust=nd)
    step_bytes = step_model_bytes(wsum, types.SimpleNamespace(n_cells_total=ncells))
    pk, pk_src = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    return {
        "workload": f"{len(ws)} independent 1D periodic dusty waves, 1k-64k particles each (log-uniform), "
                    f"t_stop log-uniform 1e-5..1, amplitudes 1e-5..1e-3, h=1.2dx, cell 2h, FP32",
        "instances": len(ws), "particles": n, "cells": ncells,
        "form": {"mode": {b.TFSPH_BATCH_PERSISTENT: "persistent", b.TFSPH_BATCH_TILED: "tiled"}.get(
                     pick["mode"], "kernels"),
                 "block": pick["block"], "blocks_per_sm": pick["blocks_per_sm"], "graph": bool(info.graph),
                 "tile": (f"{pick['block']} consecutive particles per CTA, their cells +- R staged in shared memory"
                          if pick["mode"] == b.TFSPH_BATCH_TILED else "none (global-memory walk)"),
                 "picked_by": "tfsph_batch_autotune over forms x CTA sizes (x CTAs per SM, persistent)"},
        "forms_ms_per_step_at_256_threads": forms,
        "batched_ms_per_step": batched_ms, "looped_ms_per_step": looped_ms,
        "speedup_vs_looped": looped_ms / batched_ms,
        "value": n / (batched_ms * 1e-3), "unit": UNIT,
        "launches_per_step": (info.launches - launches0) / bsteps,
        "hbm_frac": (step_bytes / (batched_ms * 1e-3) / 1e9) / hbm, "hbm_peak_gbs": hbm,
        "steps": {"batched": bsteps, "looped": lsteps},
    }


def run_schemes(b, args, only=None):
    """The other two drag schemes of the paper on the same 3D box: ISPH
    (Sec. 2.2) and MK (Sec. 2.1, explicit: run at tau = t_stop / 2, inside its
    stability limit). CUDA events on the stream around 20 steps after 3."""
    import numpy as np
    import torch

    w, desc = make_workload(args.workload)
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    stream = torch.cuda.current_stream()
    cell_acc = b.TFSPH_CELL_ACC_FP32 if args.cell_acc == "fp32" else b.TFSPH_CELL_ACC_FP64
    out = {}
    for name, drag in (("isph", b.TFSPH_DRAG_ISPH), ("mk", b.TFSPH_DRAG_MK)):
        if only is not None and name != only:
            continue
        tau = w.tau if drag == b.TFSPH_DRAG_ISPH else 0.5 * float(np.min(w.tstop))
        p = b.params_from_dict(w.params, cell_acc=cell_acc, drag=drag)
        with b.Context(p, f32(w.gx), f32(w.gv), f32(w.dx), f32(w.du), f32(w.tstop), ge=f32(w.ge),
                       frozen=w.frozen) as c:
            c.set_stream(stream)
            for _ in range(3):
                c.step(tau, w.g)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            steps = 20
            e0.record(stream)
            for _ in range(steps):
                c.step(tau, w.g)
            e1.record(stream)
            torch.cuda.synchronize()
            c.sync()
            ms = e0.elapsed_time(e1) / steps
            c.profile(True)
            for _ in range(5):
                c.step(tau, w.g)
            ph, ps, _ = c.profile_read()
            c.profile(False)
        n = w.n_gas + w.n_dust
        out[name] = {"ms_per_step": ms, "value": n / (ms * 1e-3), "unit": UNIT, "tau": tau,
                     "drag_phase_ms": ph["drag"] / max(1, ps),
                     "note": "drag phase = cross-phase sums + particle update (+ dust density for ISPH)"}
    out["workload"] = desc
    return out


def run_e2e(b, ctx, w, args, dist):
    """Same metric through the public API with page-locked host buffers: the
    state lives on the host and every step uploads it (tfsph_set_state),
    steps, and reads the new state back into the same buffers, so the timed
    steps follow the same trajectory as the device-timed run (W untimed
    steps from the initial state, then K timed ones)."""
    import numpy as np
    import torch

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = a
        return t

    keep = [pinned(w.gx), pinned(w.gv), pinned(w.dx), pinned(w.du), pinned(w.tstop)]
    ge = pinned(w.ge) if w.ge is not None else None
    gx, gv, dx, du, ts = (t.numpy() for t in keep)
    outs = {b.TFSPH_FIELD_POS_G: gx, b.TFSPH_FIELD_VEL_G: gv, b.TFSPH_FIELD_POS_D: dx, b.TFSPH_FIELD_VEL_D: du}
    if ge is not None:
        outs[b.TFSPH_FIELD_ENERGY_G] = ge.numpy()
    h2d = 4 * (gx.size + gv.size + dx.size + du.size + ts.size + (w.n_gas if ge is not None else 0)) + \
        (w.n_gas if w.frozen is not None else 0)
    d2h = sum(4 * a.size for a in outs.values())

    def one():
        ctx.set_state(gx, gv, dx, du, ts, ge=None if ge is None else ge.numpy(), frozen=w.frozen)
        ctx.step(w.tau, w.g)
        for f, a in outs.items():
            ctx.field(f, out=a)

    for _ in range(max(1, args.warmup)):
        one()
    k = max(1, args.steps)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        one()
    torch.cuda.synchronize()
    dt = dist.max(time.perf_counter() - t0)
    dist.barrier()
    n = w.n_gas + w.n_dust
    return {"value": dist.sum(n * k) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": k, "ms_per_step": dt / k * 1e3}


def main(argv=None):
    args = parse_args(argv)
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)  # rank 0 only; the other ranks exit without work
        return
    import torch
    dist.init("nccl" if torch.cuda.is_available() else "gloo")
    try:
        run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
