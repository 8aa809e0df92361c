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
    "shell60_N16": (0, 1, 4, "60 macro cells (icosahedral shell, 1 layer), N=16, r in [0.55, 1]"),
}
HBM_MEASURED_GBS = 6794.8    # MEASURED_PEAKS.json: copy bandwidth on the GB300s
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (recipe's nominal figure: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)
LSQP_FLOPS = {1: 44, 2: 59, 3: 74}   # Table 4.2: 29 + 15 q flops per stencil-based update


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
    p.add_argument("--mode", choices=["solve", "smoother", "serve", "variants", "discretisation"], default="solve",
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
    p.add_argument("--serve-batch-rhs", type=int, default=16,
                   help="continuous batching of the serving stream: right-hand sides per merged solve (1 = off)")
    p.add_argument("--disc-max-nodes", type=float, default=25e6,
                   help="--mode discretisation: largest level (total nodes) of the study")
    p.add_argument("--disc-cells", type=str, default="60,480,3840,30720",
                   help="--mode discretisation: macro meshes (cell counts) of the study")
    p.add_argument("--disc-min-level", type=int, default=2,
                   help="--mode discretisation: first level L (N = 2^(L+2))")
    p.add_argument("--compare-f64", action="store_true",
                   help="with --precision mixed: also time one plain FP64 solve and report the speedup")
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

def traffic_record(kernel: str, workload: str):
    """ncu DRAM bytes per launch of `kernel` on `workload`, if recorded for the
    current kernel source (profiles/traffic.txt, JSON written from an ncu capture);
    None when absent or when the source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(f"{kernel}@{workload}")
    if not rec:
        return None
    src = open(os.path.join(ROOT, "paper_1608_06473_gb300", "csrc", rec["source"]), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != rec["sha256_16"]:
        return None
    return rec["dram_bytes_per_launch"]


def run_ours(args, rank, world, local):
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic

    torch.cuda.set_device(local)
    tang, layers, L, desc = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    s = hhg.Shell(0.55, 1.0, tang, layers, L, stream=stream)
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

    for _ in range(args.warmup):
        step(f, u)
    torch.cuda.synchronize()

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

    g_lsqp = sweep_glups(hhg.HHG_OP_LSQP, 3)
    g_ifem = sweep_glups(hhg.HHG_OP_IFEM, 1)
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
        ke = max(1, min(args.steps, 2))
        uhs = [torch.zeros(n_total, dtype=torch.float64).pin_memory() for _ in range(ke)]   # u0 = 0 per step
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_upd = 0
        for uh in uhs:
            rel, cycles = step(fh, uh)
            e_upd += updates(cycles)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": e_upd * world / te / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": 16 * n_total,
               "d2h_bytes_per_step": 8 * n_total, "steps": ke}

    # one smoother launch updates every cell-interior node of the finest level once
    N = 2 ** L
    n_cells = 20 * 4 ** tang * layers * 3
    units_per_launch = n_cells * (N - 1) * (N - 2) * (N - 3) // 6
    avg_launch_s = sm_ms * 1e-3 / max(sm_n, 1)
    flops = LSQP_FLOPS[args.q] * units_per_launch
    if args.precision == "f64":
        achieved = flops / avg_launch_s / 1e12
        roofline = {"kernel": "lsqp_node_kernel<%d,SMOOTH> (finest level; one sweep = 4 colour launches)" % args.q,
                    "bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_NOMINAL_TFLOPS,
                    "traffic": traffic_record("lsqp_node_smooth_f64", args.workload),
                    "peak_note": "FP64 nominal (recipe: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz)"}
    else:
        achieved = 12 * units_per_launch / avg_launch_s / 1e9
        cfg = hhg.hhg_tuning(s.handle, L)[0]
        kname = ("lsqp_stage32_smooth<%d> (finest level, one launch per sweep, planes staged in shared memory; "
                 "tuned configuration %d)" % (args.q, cfg)) if cfg >= 0 else \
            ("lsqp_node32_%skernel<%d,SMOOTH> (finest level, tuned: one launch per colour)"
             % ("x2_" if cfg == -2 else "", args.q))
        roofline = {"kernel": kname,
                    "bound": "hbm", "achieved": achieved, "peak": HBM_MEASURED_GBS, "unit": "GB/s",
                    "frac": achieved / HBM_MEASURED_GBS,
                    "traffic": traffic_record("lsqp_stage32_smooth", args.workload),
                    "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"}
    roofline.update({"launches": sm_n, "avg_launch_ms": avg_launch_s * 1e3,
                     "algorithmic_flops_per_launch": flops,
                     "algorithmic_bytes_per_launch": (24 if args.precision == "f64" else 12) * units_per_launch})
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
           "clocks": clk, "gpu_launches": launches, "roofline": roofline,
           "e2e": e2e,
           "smoother_glups": {"lsqp": g_lsqp, "ifem": g_ifem, "lsqp_over_ifem": g_lsqp / g_ifem},
           "vcycle_s_to_1e-8": ms * 1e-3 / args.steps, "cycles": cyc_list, "final_relres": max(rels),
           "breakdown": breakdown, "f64_solve": f64_solve,
           "smoother_tuning": ({str(l): hhg.hhg_tuning(s.handle, l)[0] for l in range(3, L + 1)}
                               if args.precision == "mixed" else None),
           "speedup_over_f64_solve": (f64_solve["s"] / (ms * 1e-3 / args.steps)) if f64_solve else None}
    s.close()
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


def cpu_baseline(workload, n_cells=6, sweeps=60):
    upd, sec = oracle_sample(workload, n_cells, sweeps)
    return {"value": upd / sec / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle LSQP multicolour GS, {sweeps} sweeps over the interior rows of {n_cells} seeded "
                      f"macro cells of {workload} (FP64 NumPy, one core; assembly and fit excluded)",
            "seconds": sec}


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
                             "sample": f"per step: {sweeps} oracle LSQP GS sweeps over {n_cells} seeded macro cells"},
            "e2e": {"value": v, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


SERVE_RADII = [0.35 + 0.05 * k for k in range(8)]   # inner radii of the request stream (8-point grid)
SERVE_LEVELS = [4, 5, 6, 7]                          # N = 16 .. 128 on the 60-macro shell


def serve_run(n_requests, rate_hz=200.0, seed=2024, max_inflight=4, warm=True, max_batch_rhs=16):
    """Poisson stream of shell solves through the library's request loop
    (hhg_server_*): levels 4-7 and inner radius (from an 8-point grid in
    [0.35, 0.7]) drawn uniformly, 1-8 right-hand sides uniform[-1, 1] each,
    mixed precision to relative residual 1e-8.  With warm=True every
    (radius, level) hierarchy is built once before the timed stream, so the
    stream measures the resident-hierarchy steady state.  max_batch_rhs > 1
    turns on continuous batching (queued requests of one key merged into one
    batched solve).  Returns latency percentiles and throughput from the
    library's own per-request stamps."""
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

    srv = hhg.Server(max_inflight=max_inflight, dtype=hhg.HHG_F32, rtol=1e-8, max_batch_rhs=max_batch_rhs)
    try:
        if warm:
            ts = [srv.submit(rhs(ri, L, 1), r_inner=ri, L=L) for ri in SERVE_RADII for L in SERVE_LEVELS]
            for t in ts:
                srv.wait(t)
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
    finally:
        srv.close()
    lat = np.array([i["t_end"] - i["t_submit"] for i in infos])
    span = max(i["t_end"] for i in infos) - min(i["t_submit"] for i in infos)
    n_rhs = sum(nr for _, _, nr in reqs)
    return {"requests": n_requests, "arrival_rate_hz": rate_hz, "max_inflight": max_inflight,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "throughput_req_s": n_requests / span,
            "throughput_rhs_s": n_rhs / span, "worst_relres": worst,
            "reused": int(sum(i["reused"] for i in infos)), "resident_hierarchies": stats["resident"],
            "max_batch_rhs": max_batch_rhs,
            "merged_requests": int(sum(i["batch_rhs"] > nr for i, (_, _, nr) in zip(infos, reqs))),
            "mean_batch_rhs": float(np.mean([i["batch_rhs"] for i in infos])),
            "resident_gb": stats["bytes"] / 1e9,
            "workload": "Poisson arrivals (mean %g req/s) of shell solves on the 60-macro icosahedral shell, "
                        "levels 4-7 (N=16..128) and r_inner in {0.35,0.40,...,0.70} drawn uniformly, 1-8 "
                        "right-hand sides uniform[-1,1]; mixed precision, V(3,3) to 1e-8; hierarchies "
                        "resident (built before the stream)" % rate_hz}


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


def run_smoother(args):
    """Finest-level smoother only: setup, fit, `warmup` sweeps, then `steps`
    sweeps timed with CUDA events on the launching stream."""
    import torch

    import paper_1608_06473_gb300 as hhg
    import synthetic
    tang, layers, L, desc = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    s = hhg.Shell(0.55, 1.0, tang, layers, L, stream=stream)
    n_total, n_free = s.num_nodes()
    opcode = hhg.HHG_OP_LSQP if args.op == "lsqp" else hhg.HHG_OP_IFEM
    if opcode == hhg.HHG_OP_LSQP:
        s.fit(args.q, args.j, stream=stream)
    dt = torch.float32 if args.precision == "mixed" else torch.float64
    dtype = hhg.HHG_F32 if args.precision == "mixed" else hhg.HHG_F64
    f = torch.from_numpy(synthetic.uniform(n_total, synthetic.SEED_F)).cuda().to(dt)
    u = torch.from_numpy(synthetic.uniform(n_total, synthetic.SEED_U)).cuda().to(dt)
    if args.smooth_cfg is not None and args.precision == "mixed":
        s.smooth(f, u.clone(), 1, op=opcode, dtype=dtype, stream=stream)   # allocates and tunes the FP32 buffers
        hhg.hhg_set_tuning(s.handle, L, args.smooth_cfg)
    s.smooth(f, u, args.warmup, op=opcode, dtype=dtype, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s.smooth(f, u, args.steps, op=opcode, dtype=dtype, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    tuning = hhg.hhg_tuning(s.handle, L) if args.precision == "mixed" else None
    s.close()
    return {"mode": "smoother", "op": args.op, "precision": "f32" if args.precision == "mixed" else "f64",
            "tuning": None if tuning is None else {"cfg": tuning[0], "ms": list(tuning[1])},
            "workload": args.workload, "sweeps": args.steps,
            "ms_per_sweep": ms / args.steps, "GLUP/s": n_free * args.steps / (ms * 1e-3) / 1e9}


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
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    rank, world, local = dist_init(args.gpus)
    out = run_ours(args, rank, world, local)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        out["serving"] = serve_run(args.serve_requests, max_batch_rhs=args.serve_batch_rhs)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
