#!/usr/bin/env python
"""Benchmark of the two-scale (LSQP) multigrid solve on one GB300.

Workload (default): the 3840-macro shell r in [0.55, 1] (icosahedron refined
twice on the surface, 4 radial layers, 3 tetrahedra per prism) refined to
N = 64 intervals per macro edge (168,428,034 nodes, 167,117,310 unknowns),
FP64, LSQP surrogate q = 2 on S_l = M_2, right-hand side uniform[-1, 1]
(seed 0).  One step is the whole path: the surrogate fit (sampling + least
squares) followed by V(3,3) cycles from u = 0 until the relative residual is
<= 1e-8.

value: stencil-row updates per second over the step (GLUP/s): every smoother
update, residual row and convergence-check row on levels N >= 8, divided by
the step's device time; the N = 4 coarse solve is not counted.

Reported beside it: the smoother alone (one full sweep of the finest level,
LSQP and IFEM), the dominant kernel's roofline (finest-level cell-interior
LSQP smoother, FP64 pipe bound), the end-to-end number through host buffers,
and the CPU oracle timed on a sample of the same workload.

--impl reference times the CPU oracle (the only reference this method has)
on the host cores, on the same workload, each step a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
T_START = time.perf_counter()
sys.path.insert(0, ROOT)

METRIC = "GLUP/s surrogate smoother vs IFEM; V-cycle s to 1e-8 residual; p50/p99 latency"
WORKLOADS = {
    # name: (tang, layers, L, description)
    "shell3840_N64": (2, 4, 6, "3840 macro cells (icosahedral shell, 2 surface refinements, 4 layers), "
                               "N=64 intervals per macro edge, r in [0.55, 1]"),
    "shell3840_N128": (2, 4, 7, "3840 macro cells (icosahedral shell, 2 surface refinements, 4 layers), "
                                 "N=128 intervals per macro edge, r in [0.55, 1]"),
    "shell1920_N64": (2, 2, 6, "1920 macro cells (icosahedral shell, 2 surface refinements, 2 layers), N=64, "
                               "r in [0.55, 1]"),
    "shell480_N64": (1, 2, 6, "480 macro cells (icosahedral shell, 1 surface refinement, 2 layers), N=64, "
                              "r in [0.55, 1]"),
    "shell480_N128": (1, 2, 7, "480 macro cells (icosahedral shell, 1 surface refinement, 2 layers), N=128, "
                               "r in [0.55, 1]"),
    "shell60_N16": (0, 1, 4, "60 macro cells (icosahedral shell, 1 layer), N=16, r in [0.55, 1]"),
}
HBM_FALLBACK_GBS = 6800.0    # profiling recipe's fallback, used only when MEASURED_PEAKS.json is absent
LSQP_FLOPS = {1: 44, 2: 59, 3: 74}   # Table 4.2: 29 + 15 q flops per stencil-based update
# FP64 flops of Eq. 5.1 once the weights are known (Table 4.2's CONS count:
# 14 multiply-adds and the division by the centre weight, here a multiply
# by its reciprocal).  The LSQP kernels issue exactly these on the FP64 pipe;
# the 15 q flops of the weight recurrence run in exact integer arithmetic.
STENCIL_FLOPS = 29


def hbm_peak():
    """(GB/s, note): MEASURED_PEAKS.json's copy bandwidth, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return float(json.load(open(path))["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, copy)"
        except (KeyError, ValueError):
            pass
    return HBM_FALLBACK_GBS, "of fallback (profiling recipe, no MEASURED_PEAKS.json)"


def measure_peaks(hhg, stream=None):
    """FP64 and FP32 multiply-add throughput of this GPU now (hhg_peak_rate:
    independent FMA chains on every SM, best of three ~150 ms runs)."""
    out = {}
    for name, kind in (("fp64_fma_per_s", hhg.PEAK_FP64_FMA), ("fp32_fma_per_s", hhg.PEAK_FP32_FMA)):
        out[name] = hhg.hhg_peak_rate(kind, stream)[0]
    out["fp64_tflops"] = 2 * out["fp64_fma_per_s"] / 1e12
    out["fp32_tflops"] = 2 * out["fp32_fma_per_s"] / 1e12
    return out


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="shell3840_N64")
    p.add_argument("--q", type=int, default=2)
    p.add_argument("--j", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--mode", choices=["solve", "smoother", "serve", "variants", "discretisation", "batch", "peaks",
                                      "traffic", "mixed"],
                   default="solve",
                   help="solve: the whole path per step (default); smoother: finest-level sweeps only "
                        "(for profiling the smoother kernels)")
    p.add_argument("--op", choices=["lsqp", "ifem"], default="lsqp", help="operator for --mode smoother")
    p.add_argument("--smooth-cfg", type=int, default=None,
                   help="--mode smoother, mixed precision: pin the FP32 smoother configuration of the finest "
                        "level (-1 per-colour kernel, 0..3 staged; default: the tuner's choice)")
    p.add_argument("--precision", choices=["f64", "mixed"], default="f64",
                   help="f64: FP64 V-cycles; mixed: FP32 V-cycles inside FP64 iterative refinement")
    p.add_argument("--serve-requests", type=int, default=48,
                   help="requests of the serving stream reported beside the solve (0 = skip)")
    p.add_argument("--serve-batch-rhs", type=int, default=8,
                   help="continuous batching of the serving stream: right-hand sides per merged solve (1 = off)")
    p.add_argument("--disc-max-nodes", type=float, default=25e6,
                   help="--mode discretisation: largest level (total nodes) of the study")
    p.add_argument("--disc-cells", type=str, default="60,480,3840,30720",
                   help="--mode discretisation: macro meshes (cell counts) of the study")
    p.add_argument("--disc-min-level", type=int, default=2,
                   help="--mode discretisation: first level L (N = 2^(L+2))")
    p.add_argument("--compare-f64", action="store_true",
                   help="with --precision mixed: also time one plain FP64 solve and report the speedup")
    p.add_argument("--no-mixed-c3", action="store_true",
                   help="skip the mixed-precision vs FP64 solve on the N=128 shell reported beside the default line")
    p.add_argument("--batch-rhs", type=int, default=32, help="--mode batch: right-hand sides of the batched solve")
    p.add_argument("--nrhs", type=int, default=1, help="--mode smoother: right-hand sides smoothed together")
    p.add_argument("--fp64-kernel", type=int, default=0, choices=[0, 1, 2],
                   help="FP64 surrogate kernels: 0 = per node (default), 1 = runs, one launch per colour, "
                        "2 = runs with the cell-resident sweep")
    p.add_argument("--ncu-report", type=str, default=None,
                   help="--mode traffic: ncu report (.ncu-rep) holding DRAM counters of one launch of the kernel")
    p.add_argument("--traffic-key", type=str, default="lsqp_node_smooth_f64",
                   help="--mode traffic: record key (kernel) in profiles/traffic.txt")
    p.add_argument("--traffic-source", type=str, default="cell.cu",
                   help="--mode traffic: source file of the kernel (its hash gates the record)")
    p.add_argument("--traffic-scale", type=float, default=8.0,
                   help="--mode traffic: captured launch -> one sweep of the bench workload (launches per sweep x "
                        "units ratio)")
    return p.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (replicas only: every rank solves its own shell)
# ----------------------------------------------------------------------------

def dist_init(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or (self.uuid and parts[0] != self.uuid):
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def source_hash(path):
    """Hash of a CUDA source's code: comments removed and whitespace
    collapsed, so the traffic record survives documentation edits but not a
    change to the code it was captured from."""
    import re
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = " ".join(src.split())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def traffic_record(kernel: str, workload: str):
    """ncu DRAM bytes of one sweep (all its launches) of `kernel` on
    `workload`, if recorded for the current kernel source (profiles/traffic.txt,
    written by profiles/traffic_record.py from an ncu capture); None when
    absent or when the source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(f"{kernel}@{workload}")
    if not rec:
        return None
    if source_hash(os.path.join(ROOT, "paper_1608_06473_gb300", "csrc", rec["source"])) != rec.get("code_sha256_16"):
        return None
    return rec["dram_bytes_per_sweep"]


def run_ours(args, rank, world, local):
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic

    torch.cuda.set_device(local)
    tang, layers, L, desc = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    s = hhg.Shell(0.55, 1.0, tang, layers, L, stream=stream)
    hhg.hhg_set_fp64_kernel(s.handle, args.fp64_kernel)
    n_total, n_free = s.num_nodes()
    free_per_level = {l: s.num_nodes(l)[1] for l in range(2, L + 1)}
    f = torch.from_numpy(synthetic.uniform(n_total, synthetic.SEED_F)).cuda()
    u = torch.zeros(n_total, dtype=torch.float64, device="cuda")
    op = hhg.HHG_OP_LSQP
    dtype = hhg.HHG_F32 if args.precision == "mixed" else hhg.HHG_F64
    nu1 = nu2 = 3

    def step(fv, uv):
        s.fit(args.q, args.j, stream=stream)
        if isinstance(uv, torch.Tensor) and uv.is_cuda:
            uv.zero_()
        rel, cycles, _ = s.vcycle(fv, uv, nu1, nu2, max_cycles=60, rtol=1e-8, op=op, dtype=dtype, stream=stream)
        return rel[0], cycles

    def updates(cycles):
        per_cycle = sum((nu1 + nu2 + 1) * free_per_level[l] for l in range(3, L + 1)) + free_per_level[L]
        return cycles * per_cycle + free_per_level[L]

    log("shell set up (%d nodes)" % n_total)
    # arithmetic peaks of this GPU, measured now (roofline denominators)
    peaks = measure_peaks(hhg, stream)
    log("peaks measured")
    hbm_gbs, hbm_note = hbm_peak()

    for _ in range(args.warmup):
        step(f, u)
    torch.cuda.synchronize()
    log("warm-up steps done")

    props = torch.cuda.get_device_properties(local)
    uuid = "GPU-" + str(props.uuid) if hasattr(props, "uuid") else None
    clocks = ClockSampler(uuid)
    hhg.hhg_timing(s.handle, True)
    launches0 = hhg.hhg_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    tot_updates, cyc_list, rels = 0, [], []
    for _ in range(args.steps):
        rel, cycles = step(f, u)
        tot_updates += updates(cycles)
        cyc_list.append(cycles)
        rels.append(rel)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = hhg.hhg_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world)
    sm_ms, sm_n = hhg.hhg_timing_read(s.handle, hhg.HHG_T_CELL_SMOOTH)
    breakdown = {}
    for name, tid in hhg.TIMERS.items():
        ms_t, cnt = hhg.hhg_timing_read(s.handle, tid)
        breakdown[name] = {"ms_per_step": ms_t / args.steps, "count_per_step": cnt / args.steps}
    hhg.hhg_timing(s.handle, False)

    # smoother alone: one sweep of the finest level (all 10 steps)
    sdt = torch.float32 if args.precision == "mixed" else torch.float64

    def sweep_glups(opcode, reps):
        uu = torch.from_numpy(synthetic.uniform(n_total, synthetic.SEED_U)).cuda().to(sdt)
        ff = f.to(sdt)
        s.smooth(ff, uu, 1, op=opcode, dtype=dtype, stream=stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.smooth(ff, uu, reps, op=opcode, dtype=dtype, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        return n_free * reps / (a.elapsed_time(b) * 1e-3) / 1e9

    log("timed steps done")
    g_lsqp = sweep_glups(hhg.HHG_OP_LSQP, 3)
    g_ifem = sweep_glups(hhg.HHG_OP_IFEM, 1)
    log("smoother sweeps timed")
    f64_solve = None
    if args.precision == "mixed" and args.compare_f64:
        u.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rel64, cyc64, _ = s.vcycle(f, u, nu1, nu2, max_cycles=60, rtol=1e-8, op=op, dtype=hhg.HHG_F64, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        f64_solve = {"s": a.elapsed_time(b) * 1e-3, "cycles": cyc64, "relres": float(rel64[0])}

    # end to end through host buffers (pinned): H2D of f and u, D2H of u per step
    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(synthetic.uniform(n_total, synthetic.SEED_F)).pin_memory()
        ke = max(1, min(args.steps, 5))
        uhs = [torch.zeros(n_total, dtype=torch.float64).pin_memory() for _ in range(ke)]   # u0 = 0 per step
        # one untimed step through host buffers first: the library allocates
        # its device staging buffers for host vectors on the first such call
        step(fh, torch.zeros(n_total, dtype=torch.float64).pin_memory())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_upd = 0
        for uh in uhs:
            rel, cycles = step(fh, uh)
            e_upd += updates(cycles)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": e_upd * world / te / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": 16 * n_total,
               "d2h_bytes_per_step": 8 * n_total, "steps": ke, "warmup": 1}

    # the dominant kernel: the finest level's cell-interior smoother, timed
    # per sweep (one cell-resident launch, or 4 colour launches)
    N = 2 ** L
    n_cells = 20 * 4 ** tang * layers * 3
    units_per_sweep = n_cells * (N - 1) * (N - 2) * (N - 3) // 6
    sweep_s = sm_ms * 1e-3 / max(sm_n, 1)
    k64, lps, tkey = fp64_smoother_name(s, L, args.q)
    if args.precision == "mixed":
        cfg32 = hhg.hhg_tuning(s.handle, L)[0]
        lps = 1 if 0 <= cfg32 <= 5 or cfg32 == 7 else 4
    common = {"sweeps": sm_n, "launches": lps * sm_n, "avg_sweep_ms": sweep_s * 1e3,
              "avg_launch_ms": sweep_s * 1e3 / lps, "units_per_sweep": units_per_sweep,
              "units_per_launch": units_per_sweep / lps}
    if args.precision == "f64":
        achieved = STENCIL_FLOPS * units_per_sweep / sweep_s / 1e12
        traffic = traffic_record(tkey, args.workload)
        roofline = {"kernel": k64,
                    "bound": "alu", "achieved": achieved, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                    "frac": achieved / peaks["fp64_tflops"],
                    "traffic": traffic / lps if traffic else None,
                    "peak_note": "of measured: FP64 FMA throughput of this GPU measured in this run "
                                 "(hhg_peak_rate, 2 flops per FMA)",
                    "algorithmic": "29 FP64 flops per update (Eq. 5.1 with known weights: 14 FMA + 1 multiply by "
                                   "the centre reciprocal; the kernel issues exactly these on the FP64 pipe)",
                    "paper_flops": {"per_update": LSQP_FLOPS[args.q],
                                    "tflops": LSQP_FLOPS[args.q] * units_per_sweep / sweep_s / 1e12,
                                    "note": "Table 4.2 (29 + 15 q, weights included); the 15 q weight flops run in "
                                            "exact integer arithmetic here, so this rate is not bounded by the FP64 "
                                            "pipe"},
                    "dram": {"algorithmic_gbs": 24 * units_per_sweep / sweep_s / 1e9,
                             "measured_gbs": (traffic / sweep_s / 1e9) if traffic else None,
                             "traffic_per_sweep": traffic,
                             "peak_gbs": hbm_gbs, "peak_note": hbm_note,
                             "frac": ((traffic / sweep_s / 1e9) / hbm_gbs) if traffic else None}}
    else:
        achieved = 12 * units_per_sweep / sweep_s / 1e9
        cfg = hhg.hhg_tuning(s.handle, L)[0]
        kname = smoother32_name(cfg, args.q)
        roofline = {"kernel": kname,
                    "bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": achieved / hbm_gbs,
                    "traffic": None,
                    "peak_note": hbm_note,
                    "algorithmic": "12 B per update (FP32 u read, f read, u written)"}
    roofline.update(common)
    value = tot_updates * world / (ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if args.precision == "f64" else "f32 (inner cycles) + f64 (refinement)",
           "data": "synthetic",
           "config": {"workload": args.workload, "shell": desc, "op": "lsqp", "q": args.q, "j": args.j,
                      "precision": args.precision,
                      "cycle": "V(3,3)", "rtol": 1e-8, "unknowns": n_free, "nodes": n_total,
                      "l2": "inputs larger than L2 (each FP64 vector %.2f GB)" % (8 * n_total / 1e9),
                      "parallelism": "replicas" if world > 1 else "single"},
           "clocks": clk, "gpu_launches": launches, "roofline": roofline, "peaks": peaks,
           "e2e": e2e,
           "smoother_glups": {"lsqp": g_lsqp, "ifem": g_ifem, "lsqp_over_ifem": g_lsqp / g_ifem},
           "vcycle_s_to_1e-8": ms * 1e-3 / args.steps, "cycles": cyc_list, "final_relres": max(rels),
           "breakdown": breakdown, "f64_solve": f64_solve,
           "smoother_tuning": ({str(l): hhg.hhg_tuning(s.handle, l)[0] for l in range(3, L + 1)}
                               if args.precision == "mixed" else None),
           "speedup_over_f64_solve": (f64_solve["s"] / (ms * 1e-3 / args.steps)) if f64_solve else None}
    s.close()
    del f, u
    torch.cuda.empty_cache()
    return out


def log(msg):
    """Progress of the bench on stderr (the JSON line goes to stdout)."""
    print("[bench %7.1f s] %s" % (time.perf_counter() - T_START, msg), file=sys.stderr, flush=True)


def sub_json(extra, timeout_s):
    """Runs this script again with `extra` arguments in a child process (its
    own CUDA context, after this process has released its device memory) and
    returns the last JSON line it prints; a child that fails or runs past
    timeout_s gives {"error": ...} instead, so the bench line is always
    printed."""
    cmd = [sys.executable, os.path.abspath(__file__), *extra]
    try:
        res = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"error": "did not finish within %d s" % timeout_s, "args": extra}
    lines = [x for x in res.stdout.splitlines() if x.startswith("{")]
    if res.returncode != 0 or not lines:
        tail = res.stderr.strip().splitlines()
        return {"error": "exit %d: %s" % (res.returncode, tail[-1] if tail else ""), "args": extra}
    return json.loads(lines[-1])


def fp64_smoother_name(s, L, q):
    """(name, launches per sweep, traffic-record key) of the FP64 cell
    smoother the library runs on level L of shell s."""
    import paper_1608_06473_gb300 as hhg
    variant, cs = hhg.hhg_fp64_kernel(s.handle, L)
    if cs:
        return ("lsqp_resident_sweep<double,%d> (finest level; one launch per sweep, each cell's interior in the "
                "shared memory of a cluster of %d CTAs)" % (q, cs), 1, "lsqp_resident_f64")
    if variant == hhg.FP64_NODES:
        return ("lsqp_node_kernel<%d,SMOOTH> (finest level; one sweep = 4 colour launches)" % q, 4,
                "lsqp_node_smooth_f64")
    return ("lsqp_run64_kernel<%d,SMOOTH> (finest level; one sweep = 4 colour launches, a thread per run of a "
            "line)" % q, 4, "lsqp_run64_smooth_f64")


def smoother32_name(cfg, q):
    """The FP32 cell smoother kernel of tuner configuration cfg."""
    if cfg >= 7:
        return ("lsqp_resident_sweep<float,%d> (finest level, one launch per sweep, each cell's interior in the "
                "shared memory of a thread-block cluster)" % q)
    if cfg >= 6:
        return ("lsqp_chunk32_smooth<%d> (finest level, one launch per colour; a thread takes up to 4 points of a "
                "line)" % q)
    if cfg >= 4:
        return ("lsqp_wave32_smooth<%d,%d> (finest level, one launch per sweep: plane wavefront per cell, u in place "
                "through L1/L2)" % (q, 128 if cfg == 4 else 256))
    if cfg >= 0:
        return ("lsqp_stage32_smooth<%d> (finest level, one launch per sweep, planes staged in shared memory; "
                "configuration %d)" % (q, cfg))
    return "lsqp_node32_%skernel<%d,SMOOTH> (finest level, one launch per colour)" % ("x2_" if cfg == -2 else "", q)


def mixed_vs_f64(workload, q, j):
    """The mixed-precision solve (FP32 surrogate evaluation, smoother and
    transfers in V-cycles inside FP64 iterative refinement, FP64 fit and
    coarsest solve) against the plain FP64 solve on the same shell and
    right-hand side: V(3,3) to relative residual 1e-8 from u = 0, each timed
    with CUDA events after a warm-up solve (fit excluded from the solve time,
    reported apart), the difference of the two solutions, and the FP32
    smoother's rate at this size."""
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic
    tang, layers, L, desc = WORKLOADS[workload]
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    s = hhg.Shell(0.55, 1.0, tang, layers, L, stream=stream)
    n_total, n_free = s.num_nodes()
    f = torch.from_numpy(synthetic.uniform(n_total, synthetic.SEED_F)).cuda()
    out = {"workload": workload, "shell": desc, "nodes": n_total, "unknowns": n_free, "cycle": "V(3,3)",
           "rtol": 1e-8}
    sol = {}
    log("N = 128 shell set up")
    for name, dtype in (("mixed", hhg.HHG_F32), ("f64", hhg.HHG_F64)):
        uu = torch.zeros_like(f)
        a, b = ev(), ev()
        a.record(stream)
        s.fit(q, j, stream=stream)
        b.record(stream)
        s.vcycle(f, uu, 3, 3, max_cycles=60, rtol=1e-8, dtype=dtype, stream=stream)   # warm-up
        torch.cuda.synchronize()
        fit_s = a.elapsed_time(b) * 1e-3
        uu.zero_()
        hhg.hhg_timing(s.handle, True)
        torch.cuda.synchronize()
        a.record(stream)
        rel, cyc, _ = s.vcycle(f, uu, 3, 3, max_cycles=60, rtol=1e-8, dtype=dtype, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        sm_ms, sm_n = hhg.hhg_timing_read(s.handle, hhg.HHG_T_CELL_SMOOTH)
        hhg.hhg_timing(s.handle, False)
        out[name] = {"solve_s": a.elapsed_time(b) * 1e-3, "fit_s": fit_s, "cycles": cyc, "relres": float(rel[0]),
                     "cell_sweep_ms": sm_ms / max(sm_n, 1)}
        log("N = 128 %s solves done" % name)
        sol[name] = uu
    out["speedup_over_f64_solve"] = out["f64"]["solve_s"] / out["mixed"]["solve_s"]
    out["mixed_vs_f64_rel_l2"] = float(torch.linalg.vector_norm(sol["mixed"] - sol["f64"]) /
                                       torch.linalg.vector_norm(sol["f64"]))
    N = 2 ** L
    units = 20 * 4 ** tang * layers * 3 * (N - 1) * (N - 2) * (N - 3) // 6
    hbm_gbs, hbm_note = hbm_peak()
    sweep = out["mixed"]["cell_sweep_ms"] * 1e-3
    cfg = hhg.hhg_tuning(s.handle, L)[0]
    out["fp32_smoother"] = {"tuned_cfg": cfg, "kernel": smoother32_name(cfg, q), "cell_sweep_ms": sweep * 1e3,
                            "glups": units / sweep / 1e9,
                            "algorithmic_gbs": 12 * units / sweep / 1e9, "hbm_frac": 12 * units / sweep / 1e9 / hbm_gbs,
                            "peak_note": hbm_note}
    out["f64_smoother"] = {"cell_sweep_ms": out["f64"]["cell_sweep_ms"],
                           "glups": units / (out["f64"]["cell_sweep_ms"] * 1e-3) / 1e9}
    s.close()
    del f, sol
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------
# CPU oracle (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(workload, n_cells, sweeps, seed=7):
    """Oracle LSQP multicolour Gauss-Seidel sweeps over the interior rows of a
    seeded sample of macro cells of the workload's shell; returns (updates,
    seconds) of the sweeps alone (assembly and fit excluded)."""
    import synthetic
    from oracle import local as LO
    from oracle import mesh as M
    tang, layers, L, _ = WORKLOADS[workload]
    sh = M.make_shell(tang=tang, layers=layers)
    N = 2 ** L
    col = LO.colour_of(N)
    upd, sec = 0, 0.0
    for c in synthetic.sample(sh.nC, n_cells, seed):
        rows, cols, W = LO.interior_rows(sh, N, int(c), "lsqp")
        idx = np.unique(np.concatenate([rows, cols.ravel()]))
        lr, lc = np.searchsorted(idx, rows), np.searchsorted(idx, cols)
        u = synthetic.uniform(len(idx), synthetic.SEED_U)
        f = synthetic.uniform(len(idx), synthetic.SEED_F)
        t0 = time.perf_counter()
        for _ in range(sweeps):
            LO.interior_colour_steps(lr, lc, W, col, u, f)
        sec += time.perf_counter() - t0
        upd += sweeps * len(rows)
    return upd, sec


def _oracle_worker(job):
    workload, sweeps, seed = job
    return oracle_sample(workload, 1, sweeps, seed=seed)


def host_info():
    model = None
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_c1_vcycle(N=16):
    """Seconds of one V(3,3) cycle of the full oracle (global CSR operators,
    sparse direct coarse solve) on the 60-cell shell at N (16 by default),
    LSQP q = 2, from u = 0 with the seed-0 right-hand side (hierarchy
    assembly excluded)."""
    import synthetic
    from oracle import mesh as M
    from oracle import mg
    H = mg.build_hierarchy(M.make_shell(), N, "lsqp", 2, 2)
    n = H.levels[-1].n_total
    f = synthetic.uniform(n, synthetic.SEED_F)
    t0 = time.perf_counter()
    H.vcycle(len(H.ops) - 1, np.zeros(n), f)
    return time.perf_counter() - t0


def cpu_baseline(workload, n_cells=6, sweeps=60):
    """The oracle timed on this host: one core on a bounded sample of the
    workload (LSQP multicolour GS sweeps over the interior rows of seeded
    macro cells), the same on every core (one process per core, spawned, each
    sweeping its own seeded cell), and one full-oracle V-cycle at 60 cells,
    N = 16."""
    import multiprocessing as mp
    upd, sec = oracle_sample(workload, n_cells, sweeps)
    host = host_info()
    cores = host["nproc"] or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(workload, sweeps, 50 + k) for k in range(cores)])
    all_upd = sum(r[0] for r in res)
    all_sec = max(r[1] for r in res)
    return {"value": upd / sec / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle LSQP multicolour GS, {sweeps} sweeps over the interior rows of {n_cells} seeded "
                      f"macro cells of {workload} (FP64 NumPy, one core; assembly and fit excluded)",
            "seconds": sec, "host": host,
            "all_cores": {"value": all_upd / all_sec / 1e9, "unit": "GLUP/s", "cores": cores,
                          "sample": f"{cores} spawned processes, each {sweeps} sweeps over one seeded macro cell "
                                    f"of {workload}; total updates / slowest process's sweep time"},
            "c1_vcycle_s": oracle_c1_vcycle(),
            "c1_vcycle_note": "one V(3,3) cycle of the full oracle, 60 cells, N = 16, LSQP q = 2 (one core)",
            "shell60_N32_vcycle_s": oracle_c1_vcycle(32),
            "shell60_N32_vcycle_note": "one V(3,3) cycle of the full oracle, 60 cells, N = 32 (337,986 nodes), "
                                       "LSQP q = 2 (one core; hierarchy assembly excluded)"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    n_cells, sweeps = 2, 20
    for _ in range(args.warmup):
        oracle_sample(args.workload, 1, 2)
    upd, sec = 0, 0.0
    for k in range(args.steps):
        a, b = oracle_sample(args.workload, n_cells, sweeps, seed=11 + k)
        upd += a
        sec += b
    v = upd / sec / 1e9
    tang, layers, L, desc = WORKLOADS[args.workload]
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "shell": desc, "op": "lsqp", "q": 2, "j": 2},
            "cpu_baseline": {"value": v, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step: {sweeps} oracle LSQP GS sweeps over {n_cells} seeded macro cells",
                             "host": host_info()},
            "e2e": {"value": v, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


SERVE_RADII = [0.35 + 0.05 * k for k in range(8)]   # inner radii of the request stream (8-point grid)
SERVE_LEVELS = [4, 5, 6, 7]                          # N = 16 .. 128 on the 60-macro shell


def serve_run(n_requests, rate_hz=200.0, seed=2024, max_inflight=4, warm_fraction=0.5, max_batch_rhs=16,
              hbm_budget_gb=96.0):
    """Poisson stream of shell solves through the library's request loop
    (hhg_server_*): levels 4-7 and inner radius (from an 8-point grid in
    [0.35, 0.7]) drawn uniformly, 1-8 right-hand sides uniform[-1, 1] each,
    mixed precision to relative residual 1e-8, under an HBM budget.  A
    `warm_fraction` of the 32 (radius, level) hierarchies is built before the
    timed stream; the others are built inside it, evicting idle hierarchies
    when the budget requires.  max_batch_rhs > 1 turns on continuous batching
    (queued requests of one key merged into one batched solve).  Returns, from
    the library's own per-request stamps, end-to-end latency, queue wait
    (submit to start) and service time (start to end) percentiles,
    throughput, and the builds and evictions during the stream."""
    import paper_1608_06473_gb300 as hhg
    import synthetic
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    reqs = [(float(SERVE_RADII[rng.integers(8)]), int(SERVE_LEVELS[rng.integers(4)]), int(rng.integers(1, 9)))
            for _ in range(n_requests)]
    pool = {}   # right-hand sides per level (the vector length depends on the level only): 8 seeded vectors

    def rhs(ri, L, nr):
        if L not in pool:
            n, _ = hhg.hhg_problem_nodes(ri, 1.0, 0, 1, L)
            pool[L] = np.stack([synthetic.uniform(n, 900 + b) for b in range(8)])
        return pool[L][:nr]

    keys = [(ri, L) for ri in SERVE_RADII for L in SERVE_LEVELS]
    warm_keys = keys[::int(round(1 / warm_fraction))] if warm_fraction > 0 else []
    srv = hhg.Server(hbm_budget_bytes=int(hbm_budget_gb * 1e9), max_inflight=max_inflight, dtype=hhg.HHG_F32,
                     rtol=1e-8, max_batch_rhs=max_batch_rhs)
    try:
        ts = [srv.submit(rhs(ri, L, 1), r_inner=ri, L=L) for ri, L in warm_keys]
        for t in ts:
            srv.wait(t)
        st0 = srv.stats()
        log("serving: %d hierarchies built before the stream" % len(ts))
        for ri, L, nr in reqs:
            rhs(ri, L, nr)
        t0 = time.perf_counter()
        tickets = []
        for (ri, L, nr), g in zip(reqs, gaps):
            t0 += g
            dt = t0 - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(rhs(ri, L, nr), r_inner=ri, L=L))
        infos, worst = [], 0.0
        for t in tickets:
            _, rel, info = srv.wait(t)
            worst = max(worst, float(rel.max()))
            infos.append(info)
        stats = srv.stats()
        log("serving: %d requests done" % len(tickets))
    finally:
        srv.close()
    lat = np.array([i["t_end"] - i["t_submit"] for i in infos])
    wait = np.array([i["t_start"] - i["t_submit"] for i in infos])
    svc = np.array([i["t_end"] - i["t_start"] for i in infos])
    span = max(i["t_end"] for i in infos) - min(i["t_submit"] for i in infos)
    n_rhs = sum(nr for _, _, nr in reqs)
    pct = lambda x, q: float(np.percentile(x, q))
    return {"requests": n_requests, "arrival_rate_hz": rate_hz, "max_inflight": max_inflight,
            "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99), "mean_latency_s": float(lat.mean()),
            "p50_queue_wait_s": pct(wait, 50), "p99_queue_wait_s": pct(wait, 99),
            "p50_service_s": pct(svc, 50), "p99_service_s": pct(svc, 99),
            "throughput_req_s": n_requests / span, "throughput_rhs_s": n_rhs / span,
            "offered_load_note": "arrivals (%g req/s) exceed the measured throughput, so end-to-end latency is "
                                 "mostly queue wait; service time is the solve itself (with a build when the "
                                 "hierarchy was not resident)" % rate_hz,
            "worst_relres": worst,
            "reused": int(sum(i["reused"] for i in infos)),
            "built_in_stream": stats["built"] - st0["built"], "evicted_in_stream": stats["evicted"] - st0["evicted"],
            "prebuilt_keys": len(warm_keys), "keys": len(keys), "hbm_budget_gb": hbm_budget_gb,
            "resident_hierarchies": stats["resident"],
            "max_batch_rhs": max_batch_rhs,
            "merged_requests": int(sum(i["batch_rhs"] > nr for i, (_, _, nr) in zip(infos, reqs))),
            "mean_batch_rhs": float(np.mean([i["batch_rhs"] for i in infos])),
            "resident_gb": stats["bytes"] / 1e9,
            "workload": "Poisson arrivals (mean %g req/s) of shell solves on the 60-macro icosahedral shell, "
                        "levels 4-7 (N=16..128) and r_inner in {0.35,0.40,...,0.70} drawn uniformly, 1-8 "
                        "right-hand sides uniform[-1,1]; mixed precision, V(3,3) to 1e-8; HBM budget %g GB; "
                        "%d of %d hierarchies built before the stream, the rest inside it"
                        % (rate_hz, hbm_budget_gb, len(warm_keys), len(keys))}


def run_variants(args):
    """V(3,3) solves to 1e-8 of the method variants on the workload (FP64):
    LSQP q = 1, 2, 3 (j = 2), IPOLY, IFEM, and double discretisation (LSQP
    smoothing, IFEM residuals, stopped on the updates).  Per variant: the fit
    time, the solve time (CUDA events), cycles and the mean convergence
    factor."""
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic
    tang, layers, L, desc = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    s = hhg.Shell(0.55, 1.0, tang, layers, L, stream=stream)
    n_total, n_free = s.num_nodes()
    f = torch.from_numpy(synthetic.uniform(n_total, synthetic.SEED_F)).cuda()
    u = torch.zeros_like(f)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {}
    plan = [("lsqp_q1", hhg.HHG_OP_LSQP, ("lsqp", 1)), ("lsqp_q2", hhg.HHG_OP_LSQP, ("lsqp", 2)),
            ("lsqp_q3", hhg.HHG_OP_LSQP, ("lsqp", 3)), ("ipoly", hhg.HHG_OP_LSQP, ("ipoly", 2)),
            ("dd_lsqp_q2", hhg.HHG_OP_DD, ("lsqp", 2)), ("ifem", hhg.HHG_OP_IFEM, None)]
    s.fit(2, 2, stream=stream)
    s.vcycle(f, u, max_cycles=2, rtol=0.0, stream=stream, raise_on_noconv=False)   # warm-up
    for name, op, fit in plan:
        a, b = ev(), ev()
        a.record(stream)
        if fit and fit[0] == "lsqp":
            s.fit(fit[1], 2, stream=stream)
        elif fit:
            s.fit_ipoly(stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        t_fit = a.elapsed_time(b) * 1e-3
        u.zero_()
        a.record(stream)
        rel, cycles, st = s.vcycle(f, u, max_cycles=60, rtol=1e-8, op=op, stream=stream, raise_on_noconv=False)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) * 1e-3
        out[name] = {"fit_s": t_fit, "solve_s": sec, "cycles": cycles, "relres": float(rel[0]),
                     "rate": float(rel[0]) ** (1.0 / max(cycles, 1)),
                     "stop": "updates" if op == hhg.HHG_OP_DD else "residual"}
    s.close()
    return {"mode": "variants", "workload": args.workload, "shell": desc, "unknowns": n_free, "cycle": "V(3,3)",
            "rtol": 1e-8, "variants": out}


DISC_MESHES = {60: (0, 1), 480: (1, 2), 3840: (2, 4), 30720: (3, 8)}   # cells: (surface refinements, layers)
DISC_VARIANTS = ("fem", "lsqp_q1", "lsqp_q2", "lsqp_q3", "ipoly_q1", "ipoly", "ipoly_q3", "lsqp_dd", "ipoly_dd",
                 "cons", "cons_dd")


def run_discretisation(args):
    """The accuracy study of Sec. 4 (Table 4.1 and the DD / CONS comparison
    of Sec. 4.2) on the GPU: for the 60-, 480-, 3840- and 30720-cell shells
    (r in [0.55, 1]) and levels L = 2.. (N = 2^(L+2)) up to --disc-max-nodes,
    the exact solution u of Sec. 4 and f = -Laplace(u) at the nodes, the
    vertex-quadrature load vector (hhg_load_vector), 10 V(3,3) cycles from
    u = 0 per variant, and e = h^(3/2) ||I(u) - v||_2 over all nodes with
    h = H/N and the macro mesh size H = 1 for the 60-cell shell, halved by
    each macro refinement.  Variants: FEM (exact operator), LSQP q = 1, 2, 3, IPOLY q = 1, 2, 3, LSQP DD
    and IPOLY DD (surrogate relaxation, exact residuals), CONS (the operator
    of the unprojected domain, compared with u at its own nodes) and CONS DD
    (relaxation with the unprojected stencils in the cell interiors).  dev =
    e / e_FEM - 1; Table 4.1 sets entries with |dev| > 0.1 in italics."""
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic
    r1, r2 = 0.55, 1.0
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    rows = []
    for cells in [int(c) for c in args.disc_cells.split(",")]:
        tang, layers = DISC_MESHES[cells]
        for Lp in range(args.disc_min_level, 7):
            N = 2 ** (Lp + 2)
            n_total, _ = hhg.hhg_problem_nodes(r1, r2, tang, layers, Lp + 2)
            if n_total > args.disc_max_nodes:
                break
            row = {"cells": cells, "L": Lp, "N": N, "nodes": n_total, "e": {}, "dev": {}, "solve_s": {}}
            for unproj in (False, True):
                s = hhg.Shell(r1, r2, tang, layers, Lp + 2, stream=stream, unprojected=unproj)
                X = torch.from_numpy(s.node_coords()).cuda()
                ue, fe = synthetic.manufactured(X, r1, r2, xp=torch)
                del X
                b = torch.empty_like(fe)
                s.load_vector(fe, b, stream=stream)
                del fe
                u = torch.empty_like(b)
                plan = ([("cons", hhg.HHG_OP_LSQP, ("lsqp", 2))] if unproj else
                        [("fem", hhg.HHG_OP_IFEM, None), ("lsqp_q1", hhg.HHG_OP_LSQP, ("lsqp", 1)),
                         ("lsqp_q2", hhg.HHG_OP_LSQP, ("lsqp", 2)), ("lsqp_q3", hhg.HHG_OP_LSQP, ("lsqp", 3)),
                         ("lsqp_dd", hhg.HHG_OP_DD, ("lsqp", 2)), ("ipoly_q1", hhg.HHG_OP_LSQP, ("ipoly", 1)),
                         ("ipoly_q3", hhg.HHG_OP_LSQP, ("ipoly", 3)), ("ipoly", hhg.HHG_OP_LSQP, ("ipoly", 2)),
                         ("ipoly_dd", hhg.HHG_OP_DD, ("ipoly", 2)), ("cons_dd", hhg.HHG_OP_DD, ("cons", 2))])
                for name, op, fit in plan:
                    if fit and fit[0] == "lsqp":
                        s.fit(fit[1], 2, stream=stream)
                    elif fit and fit[0] == "ipoly":
                        s.fit_ipoly(fit[1], stream=stream)
                    elif fit:
                        s.fit_cons(fit[1], 2, stream=stream)
                    u.zero_()
                    a, z = ev(), ev()
                    a.record(stream)
                    s.vcycle(b, u, max_cycles=10, rtol=0.0, op=op, stream=stream, raise_on_noconv=False)
                    z.record(stream)
                    torch.cuda.synchronize()
                    row["solve_s"][name] = a.elapsed_time(z) * 1e-3
                    row["e"][name] = (2.0 ** -tang / N) ** 1.5 * float(torch.linalg.vector_norm(ue - u))
                s.close()
                del ue, b, u
                torch.cuda.empty_cache()
            for name in DISC_VARIANTS:
                row["dev"][name] = row["e"][name] / row["e"]["fem"] - 1
            rows.append(row)
            print(json.dumps({"cells": cells, "L": Lp, "e": row["e"]}), file=sys.stderr, flush=True)
    return {"mode": "discretisation", "radii": [r1, r2], "cycles": "10 x V(3,3) from u = 0",
            "h": "H/N, H = 1, 1/2, 1/4, 1/8 for 60, 480, 3840, 30720 cells",
            "load_vector": "vertex quadrature (hhg_load_vector)", "rows": rows}


BATCH_RADII = [0.35 + 0.05 * k for k in range(8)]   # inner radii of the 8-shell group


def run_batch(args):
    """The batched configuration: (A) --batch-rhs Gaussian right-hand sides
    (sigma = 1, seeds 100 + b) on the 3840-macro shell at N = 32, solved
    together (every node's weights formed once for all of them) by
    mixed-precision V(3,3) cycles (FP32 smoothing, transfers and surrogate,
    FP64 refinement and coarsest solve) replayed from a CUDA graph, to
    relative residual 1e-8 each; against the same solve of right-hand side 0
    alone.  (B) 8 shells of inner radius 0.35 .. 0.70 (3840 macros each) as
    one hierarchy per level, levels 4, 5, 6 (every kernel launch spans the 8
    shells of a level), one Gaussian right-hand side per shell.  Times are
    CUDA events around the solve after a warm-up solve; the fit is timed
    apart."""
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    tang, layers = 2, 4

    def solve(s, F, nrhs, free_per_level, L):
        U = torch.zeros_like(F)
        s.vcycle(F, U, 3, 3, max_cycles=60, rtol=1e-8, dtype=hhg.HHG_F32, nrhs=nrhs, stream=stream)   # warm-up
        U.zero_()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        rel, cyc, _ = s.vcycle(F, U, 3, 3, max_cycles=60, rtol=1e-8, dtype=hhg.HHG_F32, nrhs=nrhs, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) * 1e-3
        per_cycle = sum(7 * free_per_level[l] for l in range(3, L + 1)) + free_per_level[L]
        upd = nrhs * (cyc * per_cycle + free_per_level[L])
        return {"s": sec, "cycles": cyc, "max_relres": float(np.max(rel)), "glups": upd / sec / 1e9,
                "s_per_rhs": sec / nrhs}

    out = {"mode": "batch"}
    L = 5
    s = hhg.Shell(0.55, 1.0, tang, layers, L, stream=stream)
    n_total, n_free = s.num_nodes()
    fpl = {l: s.num_nodes(l)[1] for l in range(2, L + 1)}
    a, b = ev(), ev()
    a.record(stream)
    s.fit(2, 2, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    nb = args.batch_rhs
    F = torch.from_numpy(synthetic.batch(n_total, nb, "gaussian")).cuda()
    one = solve(s, F[0].clone(), 1, fpl, L)
    many = solve(s, F, nb, fpl, L)
    out["A"] = {"shell": "3840 macro cells, N=32, r in [0.55, 1]", "nodes": n_total, "unknowns": n_free,
                "nrhs": nb, "rhs": "Gaussian sigma=1, seeds 100+b", "fit_s": a.elapsed_time(b) * 1e-3,
                "single": one, "batched": many,
                "per_rhs_speedup": one["s"] / many["s_per_rhs"],
                "graphs": "V-cycles 2.. replayed from one CUDA graph"}
    s.close()
    del F
    torch.cuda.empty_cache()
    rows = []
    for Lg in (4, 5, 6):
        radii = [(ri, 1.0) for ri in BATCH_RADII]
        g = hhg.Shell.group(radii, tang, layers, Lg, stream=stream)
        nt, nf = g.num_nodes()
        fpl = {l: g.num_nodes(l)[1] for l in range(2, Lg + 1)}
        a, b = ev(), ev()
        a.record(stream)
        g.fit(2, 2, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        Fg = torch.from_numpy(synthetic.gaussian(nt, synthetic.SEED_BATCH0)).cuda()
        r = solve(g, Fg, 1, fpl, Lg)
        r.update({"L": Lg, "N": 2 ** Lg, "shells": len(radii), "macro_cells": 8 * 3840, "nodes": nt,
                  "unknowns": nf, "fit_s": a.elapsed_time(b) * 1e-3})
        rows.append(r)
        g.close()
        del Fg
        torch.cuda.empty_cache()
    out["B"] = {"shells": "8 shells, r_inner = 0.35, 0.40, ..., 0.70, r_outer = 1, 3840 macro cells each, one "
                          "hierarchy per level (every launch spans the 8 shells)", "levels": rows,
                "total_s": sum(r["s"] for r in rows)}
    return out


def run_traffic(args):
    """Writes the DRAM traffic record the bench's roofline reads
    (profiles/traffic.txt): dram__bytes_read.sum + dram__bytes_write.sum of
    the first launch in an ncu report, times --traffic-scale (launches per
    sweep x the bench workload's units over the captured launch's), keyed by
    kernel and workload and gated by the hash of the kernel source's code
    (comments and whitespace excluded)."""
    import csv
    import io
    res = subprocess.run(["ncu", "-i", args.ncu_report, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True)
    rows = list(csv.reader(io.StringIO(res.stdout)))
    hdr, units, first = rows[0], rows[1], rows[2]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    val = lambda name: float(first[hdr.index(name)]) * scale[units[hdr.index(name)]]
    per_launch = val("dram__bytes_read.sum") + val("dram__bytes_write.sum")
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    recs = json.load(open(path)) if os.path.exists(path) else {}
    key = f"{args.traffic_key}@{args.workload}"
    recs[key] = {"source": args.traffic_source,
                 "code_sha256_16": source_hash(os.path.join(ROOT, "paper_1608_06473_gb300", "csrc",
                                                            args.traffic_source)),
                 "dram_bytes_per_sweep": per_launch * args.traffic_scale,
                 "captured_launch_bytes": per_launch, "scale": args.traffic_scale,
                 "kernel": first[hdr.index("Kernel Name")] if "Kernel Name" in hdr else None,
                 "note": "written by bench.py --mode traffic from %s" % os.path.basename(args.ncu_report)}
    with open(path, "w") as fh:
        json.dump(recs, fh, indent=1)
    return {"mode": "traffic", "key": key, **recs[key]}


def run_peaks(args):
    import torch

    import paper_1608_06473_gb300 as hhg
    torch.cuda.init()
    out = measure_peaks(hhg)
    out["int32_imad_per_s"] = hhg.hhg_peak_rate(hhg.PEAK_INT32_IMAD)[0]
    out["hbm"] = dict(zip(("gbs", "note"), hbm_peak()))
    out["mode"] = "peaks"
    return out


def run_smoother(args):
    """Finest-level smoother only: setup, fit, `warmup` sweeps, then `steps`
    sweeps timed with CUDA events on the launching stream, over --nrhs
    right-hand sides at once (u ~ U[-1, 1] seed 1 + b, f ~ U[-1, 1] seed b)."""
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic
    tang, layers, L, desc = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    s = hhg.Shell(0.55, 1.0, tang, layers, L, stream=stream)
    n_total, n_free = s.num_nodes()
    hhg.hhg_set_fp64_kernel(s.handle, args.fp64_kernel)
    opcode = hhg.HHG_OP_LSQP if args.op == "lsqp" else hhg.HHG_OP_IFEM
    if opcode == hhg.HHG_OP_LSQP:
        s.fit(args.q, args.j, stream=stream)
    dt = torch.float32 if args.precision == "mixed" else torch.float64
    dtype = hhg.HHG_F32 if args.precision == "mixed" else hhg.HHG_F64
    nb = args.nrhs
    f = torch.from_numpy(np.stack([synthetic.uniform(n_total, synthetic.SEED_F + b) for b in range(nb)])).cuda().to(dt)
    u = torch.from_numpy(np.stack([synthetic.uniform(n_total, synthetic.SEED_U + b) for b in range(nb)])).cuda().to(dt)
    if nb == 1:
        f, u = f[0].contiguous(), u[0].contiguous()
    if args.smooth_cfg is not None and args.precision == "mixed":
        s.smooth(f, u.clone(), 1, op=opcode, dtype=dtype, nrhs=nb, stream=stream)   # allocates and tunes FP32
        hhg.hhg_set_tuning(s.handle, L, args.smooth_cfg)
    s.smooth(f, u, args.warmup, op=opcode, dtype=dtype, nrhs=nb, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s.smooth(f, u, args.steps, op=opcode, dtype=dtype, nrhs=nb, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    tuning = hhg.hhg_tuning(s.handle, L) if args.precision == "mixed" else None
    s.close()
    return {"mode": "smoother", "op": args.op, "precision": "f32" if args.precision == "mixed" else "f64",
            "tuning": None if tuning is None else {"cfg": tuning[0], "ms": list(tuning[1])},
            "workload": args.workload, "sweeps": args.steps, "nrhs": nb,
            "ms_per_sweep": ms / args.steps, "GLUP/s": nb * n_free * args.steps / (ms * 1e-3) / 1e9}


def main():
    args = parse()
    if args.mode == "smoother":
        print(json.dumps(run_smoother(args)))
        return
    if args.mode == "serve":
        print(json.dumps(serve_run(args.serve_requests, max_batch_rhs=args.serve_batch_rhs)))
        return
    if args.mode == "variants":
        print(json.dumps(run_variants(args)))
        return
    if args.mode == "discretisation":
        print(json.dumps(run_discretisation(args)))
        return
    if args.mode == "batch":
        print(json.dumps(run_batch(args)))
        return
    if args.mode == "peaks":
        print(json.dumps(run_peaks(args)))
        return
    if args.mode == "traffic":
        print(json.dumps(run_traffic(args)))
        return
    if args.mode == "mixed":
        print(json.dumps(mixed_vs_f64("shell3840_N128", args.q, args.j)))
        return
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    rank, world, local = dist_init(args.gpus)
    log("start: %s" % args.workload)
    out = run_ours(args, rank, world, local)
    log("solve, smoother and e2e timed")
    if rank == 0 and world == 1:
        if args.precision == "f64" and not args.no_mixed_c3 and args.workload == "shell3840_N64":
            mp = sub_json(["--mode", "mixed", "--q", str(args.q), "--j", str(args.j)], 300)
            out["mixed_precision"] = mp
            out["speedup_over_f64_solve"] = mp.get("speedup_over_f64_solve")
            out["speedup_over_f64_solve_workload"] = mp.get("workload")
            log("mixed precision at N = 128 done")
        if args.serve_requests > 0:
            out["serving"] = sub_json(["--mode", "serve", "--serve-requests", str(args.serve_requests),
                                       "--serve-batch-rhs", str(args.serve_batch_rhs)], 300)
            log("serving done")
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.workload)
            log("cpu baseline done")
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
