"""Benchmark of the coupled flow + thermal lattice Boltzmann step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload evaporation|droplet|heated_wall] [--n SIDE] [--prec fp64|fp32]

A bench step is one coupled time step (flow and thermal populations, every part of the hot path)
over the whole grid. Default workload: 2048 x 2048 droplet evaporation (R = 320, dT = 0.1 T_c, the
Sec. IV A set-up scaled up), FP64 storage and arithmetic. Metric: coupled MLUPS (million lattice-node
updates of f and g per second). Each step is timed with CUDA events on the library's stream; a grid
whose working set is not well above L2 has L2 flushed (a 512 MiB write) before every timed step.
The line carries the binary64 step's ALU roofline against the FMA rate measured in the same run and
its HBM fraction, and, as variants, the double-word step on the same grid, the FP32 and FP16 fused
steps at 4096^2 and the 256-instance batch against the plain path.

Under torchrun (N > 1) each rank advances its own independent replica (weak scaling, no collective
on the data path); value = all ranks' node updates / the slowest rank's time.

--impl reference times the FP64 CPU oracle on the same workload, one oracle step per bench step, on
rank 0 only.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="evaporation",
                    choices=["evaporation", "droplet", "heated_wall", "batch", "serve"])
    ap.add_argument("--requests", type=int, default=300, help="served workload: number of requests")
    ap.add_argument("--rate", type=float, default=40.0, help="served workload: Poisson arrival rate (1/s)")
    ap.add_argument("--full-stream", action="store_true",
                    help="served workload: the full request distribution (sides 64-1024, 5k-50k steps) instead of the "
                         "bounded one (64-512, 1k-5k)")
    ap.add_argument("--instances", type=int, default=256, help="batched workload: number of instances")
    ap.add_argument("--variant", type=int, default=-1,
                    help="batched workload: step-kernel variant 0-5 instead of the autotuner's choice")
    ap.add_argument("--ctas", type=int, default=16, help="batched workload with --variant: CTAs per SM")
    ap.add_argument("--n", type=int, default=0,
                    help="grid side (0 = the workload's own size); batched workload: every instance of this side")
    ap.add_argument("--dT", type=float, default=0.1, help="superheat dT / T_c of the evaporation case")
    ap.add_argument("--prec", default="", choices=["", "fp64", "df64", "fp32", "fp16"])
    ap.add_argument("--path", default="auto", choices=["auto", "split", "fused"])
    ap.add_argument("--tile", type=int, default=-1,
                    help="fused tile: -1 = library default (4), 0 = 32x16, 1 = 32x8, 2 = 32x16 two nodes "
                         "per thread, 3 = 32x32 two per thread, 4 = 32x8 in persistent CTAs staging ahead")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variants of the evaporation line (DF64 on the same grid, FP32 and FP16 at 4096^2, "
                         "the 256-instance batch)")
    ap.add_argument("--no-side-run", action="store_true", help="served workload: no 4096^2 FP16 run alongside")
    return ap.parse_args(argv)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, ws, device):
    """Element-wise maximum of per-rank timings over all ranks of the process group (the slowest
    rank's time); the values themselves on a single rank."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def aggregate_mlups(ws, nodes, steps, seconds):
    """Whole-job throughput: each of ws ranks advances its own replica of `nodes` nodes by `steps`
    steps in `seconds` (the slowest rank's time)."""
    return ws * nodes * steps / seconds / 1e6


def make_case(args, Tc, rv, rl):
    from paper_1709_04400_gb300 import workloads

    if args.workload == "evaporation":
        n = args.n or 2048
        case, rho, T = workloads.droplet_evaporation(Tc, rv, rl, n=n, radius=40.0 * n / 256, dT_ratio=args.dT)
        prec = args.prec or "fp64"
    elif args.workload == "droplet":
        n = args.n or 128
        case, rho, T = workloads.droplet_periodic(Tc, rv, rl, n=n, radius=25.0 * n / 128)
        prec = args.prec or "fp64"
    else:
        case, rho, T = workloads.heated_wall(Tc, rv, rl)
        prec = args.prec or "fp32"
    return case, rho, T, prec


class ClockSampler:
    """nvidia-smi samples every 50 ms during the timed region; entering waits (at most 3 s) for the first
    sample, so that the sampler is running when the timed region starts."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_steps(job):
    """Worker: the FP64 oracle stepping one copy of the workload for budget_s seconds; (steps, seconds)."""
    case, rho, T, budget_s = job
    from oracle import model

    keys = set(model.OracleParams.__dataclass_fields__)
    p = model.OracleParams(**{k: v for k, v in case.items() if k in keys})
    s = model.init_state(p, rho, T)
    s = model.step(p, s)  # warm-up
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        s = model.step(p, s)
        n += 1
    return n, time.perf_counter() - t0


def cpu_baseline(case, rho, T, budget_s=12.0, all_budget_s=4.0, all_case=None):
    """The FP64 oracle as it stands, on this host, on the bench workload for a bounded time: one
    process with one thread, then one process per host core, each stepping its own copy (of all_case,
    a smaller grid of the same set-up, when given: a copy of a large grid per core would need tens of
    GB of host memory). The workers are spawned (never forked after CUDA is initialised), with the
    BLAS / OpenMP pools of numpy held to one thread so that the core counts are exact."""
    import multiprocessing as mp

    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    N = case["nx"] * case["ny"]
    with ctx.Pool(1) as pool:
        n, dt = pool.map(_oracle_steps, [(case, rho, T, budget_s)])[0]
    cores = os.cpu_count() or 1
    ac, ar, aT = all_case or (case, rho, T)
    Na = ac["nx"] * ac["ny"]
    with ctx.Pool(cores) as pool:
        runs = pool.map(_oracle_steps, [(ac, ar, aT, all_budget_s)] * cores)
    agg = sum(Na * k / t for k, t in runs) / 1e6
    return {"value": N * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{n} oracle steps of the {case['nx']}x{case['ny']} workload ({dt:.1f} s, numpy FP64, 1 thread)",
            "all_cores": {"value": agg, "unit": "MLUPS", "cores": cores, "workload": ac["name"],
                          "sample": f"{cores} processes, one thread each, each stepping its own copy of "
                                    f"{ac['name']} for {all_budget_s:.0f} s ({sum(k for k, _ in runs)} oracle steps in all)"}}


# Algorithmic HBM traffic per node and step of the fused kernel: read 9 f + 9 g, write 9 f* + 9 g*,
# read and write phi_prev (304 B in FP64, 152 B in FP32); FP16 deviation storage moves 2-byte
# populations plus the FP32 reference density and temperature (read and written) and FP32 phi: 96 B.
def fused_bytes_per_node(prec_bytes):
    if prec_bytes == 2:
        return 2 * 36 + 4 * 4 + 4 * 2
    return prec_bytes * (18 + 18 + 2)


# Algorithmic traffic of the split collide kernel per node: pull 9 f + 9 g, write 9 f* + 9 g*,
# read/write phi_prev, read the centre of 9 scratch planes (rho, T, 1/rho, vx, vy, Fx, Fy, Q, dp/dT);
# the neighbour reads of T, vx, vy (and rho) are served by L1/L2 and not counted.
def collide_bytes_per_node(prec_bytes):
    return prec_bytes * (18 + 18 + 2 + 9)


# Algorithmic FP64 operations of the split collide kernel per node (each add, subtract, multiply and
# divide counted once; an FMA counts as its multiply and its add), counted term by term from the
# kernel: flow collision 136 (moments 34, equilibria and forcing 29, relaxation of 6 moments 30,
# back-transform 41, momentum update 2); heat role 93 with unit thermal rates (gradients 41, source 14,
# thermal collision in closed form 38); general thermal rates take the full MRT collision, 78 more;
# lambda = rho c_V chi adds 20 for grad rho.
def collide_flops(lambda_mode, unit_heat_rates):
    return 229 + (20 if lambda_mode == "rho_cv_chi" else 0) + (0 if unit_heat_rates else 78)


# arithmetic type of each storage precision ("df64": double-word, pairs of binary32 with a 48-bit
# significand, on the FP32 pipes)
def _dtypes():
    from paper_1709_04400_gb300 import lbpc

    return {lbpc.FP64: "f64", lbpc.DF64: "df64 (f32 pair)", lbpc.FP32: "f32", lbpc.FP16DEV: "f32 (f16 storage)"}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels this bench
# reports, from one-pass ncu captures of the same commands, keyed by (kernel, workload, storage); for
# the batch's per-tile launches, the sum over the launches of one step. Each entry carries the hash of
# the kernel sources it was captured on (kernel_source_hash); when the sources differ from that hash
# the entry describes another build and the line reports null.
MEASURED_TRAFFIC = {
    # one-pass ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of the bench's own commands
    ("k_collide", "droplet_evaporation_2048_dT0.1Tc", "fp64"): (1_539_444_224, "51ee3432028044b0"),
    ("k_collide", "droplet_evaporation_2048_dT0.1Tc", "df64"): (1_640_148_224, "51ee3432028044b0"),
    ("k_fused", "droplet_evaporation_4096_dT0.1Tc", "fp32"): (2_502_832_640, "51ee3432028044b0"),
    ("k_fused", "droplet_evaporation_4096_dT0.1Tc", "fp16"): (1_576_405_248, "51ee3432028044b0"),
    ("k_batch_tiles", "batched_evaporation_256", "fp32"): (3_894_301_184, "51ee3432028044b0"),  # one step: 5 launches
}


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the library's CUDA sources and public header."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1709_04400_gb300", "csrc")
    files = sorted(os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h")))
    for f in files + [os.path.join(ROOT, "include", "lbpc.h")]:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload, storage):
    """DRAM bytes per launch of kernel on workload if they were captured on the current sources, else None."""
    e = MEASURED_TRAFFIC.get((kernel, workload, storage))
    if e is None or e[1] != kernel_source_hash():
        return None
    return e[0]


# Nominal HBM3e bandwidth of GB300 (7.9 TB/s): the second denominator of an HBM roofline fraction,
# beside the measured copy bandwidth.
NOMINAL_HBM_GBS = 7900.0


def _peak_hbm():
    """Measured copy bandwidth of the GB300s in GB/s (fallback 6800)."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def _step_times(sim, steps, warmup, flush=None):
    """Per-kernel device times in ms of `steps` steps after `warmup` untimed ones: every step timed with
    CUDA events on the library's stream (lbpc_step_timed). With a flush buffer, L2 is overwritten
    before every step."""
    import torch

    def one():
        if flush is not None:
            with torch.cuda.stream(sim.stream):
                flush.zero_()
        return sim.step_timed()

    for _ in range(warmup):
        one()
    per = {}
    for _ in range(steps):
        for k, v in one().items():
            per.setdefault(k, []).append(v)
    return per


def _needs_flush(nodes, bytes_per_node):
    """L2 (129 MB) is flushed between timed steps unless the step's working set is well above it."""
    return nodes * bytes_per_node < 4 * 129e6


def variant_line(lbpc, case, rho, T, prec, path, steps, warmup, peak_bw, bytes_per_node, flush, storage):
    """One storage precision of a workload, timed like the headline: MLUPS, per-kernel times and the
    HBM fraction of the whole step at its algorithmic bytes per node."""
    sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
    sim.set_path(path)
    sim.init(rho, T)
    fl = flush if _needs_flush(case["nx"] * case["ny"], bytes_per_node) else None
    per = _step_times(sim, steps, warmup, fl)
    sim.check()
    sim.close()
    N = case["nx"] * case["ny"]
    kms = {k: sum(v) / len(v) for k, v in per.items()}
    step_ms = sum(kms.values())
    gbs = bytes_per_node * N / (step_ms / 1e3) / 1e9
    top = max(kms, key=kms.get)
    return {"workload": case["name"], "value": N / (step_ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": step_ms,
            "kernel_ms": kms, "top_kernel": top, "top_kernel_traffic": measured_traffic(top, case["name"], storage),
            "hbm": {"bytes_per_node": bytes_per_node, "achieved": gbs, "peak": peak_bw, "unit": "GB/s",
                    "frac": gbs / peak_bw, "frac_of_nominal": gbs / NOMINAL_HBM_GBS, "of": "whole step"},
            "l2": "flushed before every timed step" if fl is not None else "working set larger than L2, no flush",
            "launches": len(per) * steps}


def batch_measure(lbpc, workloads, prec, instances, steps, warmup, variant=-1, ctas=16, n=0, dT=0.1, clk_index=None):
    """Batched workload: many uneven evaporation instances advanced together (lbpc_batch_step, graph
    replayed), against the plain path (each instance stepped on its own through lbpc_step)."""
    import torch

    p0 = lbpc.Params(nx=8, ny=8)
    Tc, _ = lbpc.eos_critical(p0)
    rv, rl, _ = lbpc.coexistence(p0, 0.86 * Tc)
    if n:  # every instance the evaporation case of side n (R = 0.2 n)
        one = workloads.droplet_evaporation(Tc, rv, rl, n=n, radius=0.2 * n, dT_ratio=dT)
        insts = [one] * instances
        wname = f"evaporation_{n}_x{instances}"
    else:
        insts = workloads.batched_evaporation(Tc, rv, rl, count=instances)
        wname = f"batched_evaporation_{len(insts)}"
    params = [lbpc.params_from_case(c, prec) for c, _, _ in insts]
    nodes = sum(p.nx * p.ny for p in params)
    arena = sum(lbpc.Batch.instance_bytes(p) for p in params) + (256 << 20)
    b = lbpc.Batch(prec, arena, max_instances=len(insts) + 8)
    for p, (c, r, t) in zip(params, insts):
        b.add(p, r, t)
    if variant >= 0:  # a fixed configuration (no tuner launches before the timed steps)
        b.set_config(variant, ctas)
        tuned = {"fixed": True, "variant": variant, "ctas_per_sm": ctas}
    else:
        tuned = b.autotune(steps_per_candidate=2)
    b.step(warmup)
    b.check()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(clk_index) if clk_index is not None else None
    if clk:
        clk.__enter__()
    torch.cuda.synchronize()
    ev0.record(b.stream)
    b.step(steps)
    ev1.record(b.stream)
    ev1.synchronize()
    if clk:
        clk.__exit__(None, None, None)
    b.check()
    batch_s = ev0.elapsed_time(ev1) / 1e3
    cfg = b.config()
    b.close()
    sims = []
    for p, (c, r, t) in zip(params, insts):
        sim = lbpc.Simulation(p)
        sim.init(r, t)
        sims.append(sim)
    for sim in sims:
        sim.step(warmup, sync=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for sim in sims:
        sim.step(steps, sync=False)
    e1.record()
    e1.synchronize()
    plain_s = e0.elapsed_time(e1) / 1e3
    for sim in sims:
        sim.check()
        sim.close()
    value = nodes * steps / batch_s / 1e6
    plain = nodes * steps / plain_s / 1e6
    peak_bw = _peak_hbm()
    # per-tile launches (0 CTAs per SM): ceil(instances / capacity) launches and the advance per step;
    # the work-list kernel: one launch and the advance
    per_tile = cfg["ctas_per_sm"] == 0
    kernel = "k_batch_tiles" if per_tile else "k_batch_step"
    launches_per_step = (-(-len(insts) // lbpc.Batch.per_tile_capacity(prec)) + 1) if per_tile else 2
    bpn = storage_bytes_per_node(prec, lbpc)
    achieved = bpn * nodes / (batch_s / steps) / 1e9
    prec_name = {lbpc.FP64: "fp64", lbpc.FP32: "fp32", lbpc.FP16DEV: "fp16"}[prec]
    return {
        "workload": wname, "instances": len(insts), "nodes": nodes, "storage": prec_name,
        "value": value, "unit": "MLUPS", "ms_per_step": batch_s * 1e3 / steps,
        "tile": [cfg["tile_x"], cfg["tile_y"]], "ctas_per_sm": cfg["ctas_per_sm"], "graph_chunk": cfg["graph_chunk"],
        "autotune": tuned,
        "plain_path": {"value": plain, "unit": "MLUPS", "ms_per_step": plain_s * 1e3 / steps,
                       "how": "each instance stepped alone through lbpc_step (fused kernel, one launch per step)"},
        "batched_over_plain": value / plain,
        "hbm": {"kernel": kernel, "bytes_per_node": bpn, "achieved": achieved, "peak": peak_bw,
                "unit": "GB/s", "frac": achieved / peak_bw, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "traffic": measured_traffic(kernel, wname, prec_name),
                "traffic_per": "step (every launch of the step)" if per_tile else "launch"},
        "l2": "working set of %.1f GB exceeds L2" % (nodes * bpn / 1e9),
        "launches": launches_per_step * steps, "clocks": clk.summary() if clk else None,
    }


def serve_measure(lbpc, serve, prec, requests, rate, side_lo, side_hi, steps_lo, steps_hi, clk_index=None):
    """A Poisson stream of mixed evaporation / heated-wall requests, admitted by an HBM budget and advanced
    together by continuous batching: p50 / p99 time-to-result and aggregate MLUPS."""
    reqs = serve.poisson_stream(requests, rate=rate, seed=170904400 + 4, side_lo=side_lo, side_hi=side_hi,
                                steps_lo=steps_lo, steps_hi=steps_hi)
    srv = serve.Server(prec=prec, hbm_budget_bytes=24 << 30)
    clk = ClockSampler(clk_index) if clk_index is not None else None
    if clk:
        clk.__enter__()
    srv.run(reqs)
    if clk:
        clk.__exit__(None, None, None)
    st = srv.stats()
    srv.close()
    return {"workload": f"served_stream_{requests}", "value": st["aggregate_mlups"], "unit": "MLUPS",
            "latency": {"p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"]},
            "rate_per_s": rate, "sides": [side_lo, side_hi], "steps": [steps_lo, steps_hi],
            "mix": "half evaporation, half heated wall", "served": st,
            "clocks": clk.summary() if clk else None}


def storage_bytes_per_node(prec, lbpc):
    """Algorithmic HBM bytes per node and step of the fused / batched step of a storage precision."""
    return fused_bytes_per_node({lbpc.FP64: 8, lbpc.DF64: 8, lbpc.FP32: 4, lbpc.FP16DEV: 2}[prec])


def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1709_04400_gb300 import build, lbpc, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()
    DTYPE = _dtypes()
    p0 = lbpc.Params(nx=8, ny=8)
    Tc, _ = lbpc.eos_critical(p0)
    rv, rl, _ = lbpc.coexistence(p0, 0.86 * Tc)
    case, rho, T, prec_name = make_case(args, Tc, rv, rl)
    prec = {"fp64": lbpc.FP64, "df64": lbpc.DF64, "fp32": lbpc.FP32, "fp16": lbpc.FP16DEV}[prec_name]
    params = lbpc.params_from_case(case, prec)
    N = case["nx"] * case["ny"]
    peak_bw = _peak_hbm()
    bw_src = "MEASURED_PEAKS.json hbm_gbs (burst copy)"
    pb = {lbpc.FP64: 8, lbpc.DF64: 8, lbpc.FP32: 4, lbpc.FP16DEV: 2}[prec]
    bpn = fused_bytes_per_node(pb)

    def barrier():
        if ws > 1:
            dist.barrier()

    path = {"auto": lbpc.PATH_AUTO, "split": lbpc.PATH_SPLIT, "fused": lbpc.PATH_FUSED}[args.path]
    sim = lbpc.Simulation(params)
    sim.set_path(path)
    if args.tile >= 0:
        sim.set_fused_tile(args.tile)
    sim.init(rho, T)
    flush_buf = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    flush = flush_buf if _needs_flush(N, bpn) else None

    def one_step():
        if flush is not None:
            with torch.cuda.stream(sim.stream):
                flush.zero_()
        return sim.step_timed()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    per_kernel = {}
    step_ms = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ks = one_step()
            step_ms.append(sum(ks.values()))
            for k, v in ks.items():
                per_kernel.setdefault(k, []).append(v)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    sim.check()
    dev_s = sum(step_ms) / 1e3
    dev_s, wall = max_over_ranks([dev_s, wall], ws, "cuda")
    value = aggregate_mlups(ws, N, args.steps, dev_s)
    nk = len(per_kernel)
    avg = {k: sum(v) / len(v) for k, v in per_kernel.items()}
    top = max(avg, key=avg.get)
    step_avg_ms = sum(avg.values())
    hbm_step = bpn * N / (step_avg_ms / 1e3) / 1e9
    hbm = {"bytes_per_node": bpn, "achieved": hbm_step, "peak": peak_bw, "unit": "GB/s", "frac": hbm_step / peak_bw,
           "frac_of_nominal": hbm_step / NOMINAL_HBM_GBS, "of": "whole step", "peak_source": bw_src}

    # dominant kernel and its roofline
    if prec == lbpc.FP64 and "k_collide" in avg:
        # the binary64 step is bound by the FP64 pipe: its denominator is the FMA rate of this GPU,
        # measured here by a probe kernel, with the clocks seen while it ran
        with ClockSampler(local) as pclk:
            fma64 = lbpc.fma_rate(lbpc.FP64, sim.stream) / 1e12
        fpn = collide_flops(case["lambda_mode"], all(v == 1.0 for v in case["s_g"][1:]))
        achieved = fpn * N / (avg["k_collide"] / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "k_collide", "achieved": achieved, "peak": fma64, "unit": "TFLOP/s",
                "frac": achieved / fma64, "traffic": measured_traffic("k_collide", case["name"], prec_name),
                "peak_source": "binary64 FMA rate measured in this run (lbpc_fma_rate: 8 independent FMA chains per "
                               "thread on every SM)", "probe_clocks": pclk.summary(),
                "flops_per_node": fpn, "top_kernel": top, "hbm": hbm}
    elif "k_fused" in avg:
        achieved = bpn * N / (avg["k_fused"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "k_fused", "achieved": achieved, "peak": peak_bw, "unit": "GB/s",
                "frac": achieved / peak_bw, "traffic": measured_traffic("k_fused", case["name"], prec_name),
                "peak_source": bw_src, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "bytes_per_node": bpn, "top_kernel": top, "hbm": hbm}
    else:
        cb = collide_bytes_per_node(pb)
        achieved = cb * N / (avg["k_collide"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "k_collide", "achieved": achieved, "peak": peak_bw, "unit": "GB/s",
                "frac": achieved / peak_bw, "traffic": measured_traffic("k_collide", case["name"], prec_name),
                "peak_source": bw_src, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "bytes_per_node": cb, "top_kernel": top, "hbm": hbm}

    e2e = None
    if not args.no_e2e:
        # end to end through the public API with pinned host buffers: H2D of the initial fields,
        # every step followed by a D2H read of the step's result (domain mass and heat), and the
        # final fields read back to the host
        h_rho = torch.from_numpy(np.ascontiguousarray(rho)).pin_memory().numpy()
        h_T = torch.from_numpy(np.ascontiguousarray(T)).pin_memory().numpy()
        h_sums = torch.zeros((args.steps, 2), dtype=torch.float64).pin_memory()
        sim2 = lbpc.Simulation(params)
        sim2.set_path(path)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2.init(h_rho, h_T)
        for k in range(args.steps):  # each step's (mass, heat) lands in pinned host memory, no wait per step
            sim2.step(1, sync=False)
            sim2.sums_async(h_sums[k])
        sim2.check()
        sim2.fields()
        torch.cuda.synchronize()
        barrier()
        te = time.perf_counter() - t0
        te = max_over_ranks([te], ws, "cuda")[0]
        sim2.close()
        h2d = 2 * N * 8
        d2h = args.steps * 16 + 4 * N * 8
        e2e = {"value": aggregate_mlups(ws, N, args.steps, te), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "lbpc_init from pinned host fields, per step lbpc_step_async(1) + lbpc_sums_async into "
                       "pinned host memory, lbpc_check and lbpc_fields to host at the end"}
    sim.close()

    # the other storage precisions, on rank 0 after the headline's timed region: the FP64-accurate
    # double-word step on the same workload, the binary32 and binary16-deviation fused steps on the
    # 4096^2 case, and the 256-instance batch against the plain path
    variants = None
    if rank == 0 and not args.no_variants and args.workload == "evaporation":
        variants = {}
        if prec == lbpc.FP64:
            variants["df64"] = variant_line(lbpc, case, rho, T, lbpc.DF64, path, args.steps, args.warmup, peak_bw,
                                            fused_bytes_per_node(8), flush_buf, "df64")
            variants["df64"]["dtype"] = "df64 (f32 pair, 48-bit significand)"
        n4 = 4096
        c4, r4, t4 = workloads.droplet_evaporation(Tc, rv, rl, n=n4, radius=40.0 * n4 / 256, dT_ratio=args.dT)
        for name, pv, sname in (("fp32_4096", lbpc.FP32, "fp32"), ("fp16_4096", lbpc.FP16DEV, "fp16")):
            variants[name] = variant_line(lbpc, c4, r4, t4, pv, lbpc.PATH_AUTO, args.steps, args.warmup, peak_bw,
                                          storage_bytes_per_node(pv, lbpc), flush_buf, sname)
            variants[name]["dtype"] = DTYPE[pv]
        del c4, r4, t4
        variants["batched_256"] = batch_measure(lbpc, workloads, lbpc.FP32, 256, args.steps, args.warmup,
                                                clk_index=local)
        # a bounded sample of the served stream (sides 64-512, 1k-5k steps, Poisson arrivals at 40 per
        # second), FP32: continuous batching of requests that arrive while others are on the GPU
        from paper_1709_04400_gb300 import serve

        variants["served_120"] = serve_measure(lbpc, serve, lbpc.FP32, 120, 40.0, 64, 512, 1000, 5000,
                                               clk_index=local)
    del flush_buf

    base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        small = None
        if N > 512 * 512:  # the all-cores leg steps one copy per core of the 256^2 case of the same set-up
            small = workloads.droplet_evaporation(Tc, rv, rl, n=256, radius=40.0, dT_ratio=args.dT)
        base = cpu_baseline(case, rho, T, all_case=small)

    if rank == 0:
        line = {
            "metric": "coupled flow+thermal MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[prec], "data": "synthetic",
            "config": {"workload": case["name"], "nx": case["nx"], "ny": case["ny"], "nodes": N,
                       "storage": prec_name, "parallelism": f"replicas{ws}", "path": args.path,
                       "fused_tile": args.tile if args.tile >= 0 else "library default (32x8, persistent, staged ahead)",
                       "l2": ("flushed before every timed step (512 MiB write)" if flush is not None else
                              "working set (%.2f GB) larger than L2, no flush" % (bpn * N / 1e9)) +
                             "; each step timed with CUDA events on the library's stream",
                       "wall_ms_per_step": wall * 1e3 / args.steps, "kernel_source_hash": kernel_source_hash()},
            "roofline": roof, "cpu_baseline": base, "e2e": e2e, "variants": variants,
            "gpu_launches": nk * args.steps,
            "kernel_ms": avg,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_batch(args):
    """Batched workload alone: the line of batch_measure."""
    import torch

    from paper_1709_04400_gb300 import build, lbpc, workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    prec_name = args.prec or "fp32"
    prec = {"fp64": lbpc.FP64, "fp32": lbpc.FP32, "fp16": lbpc.FP16DEV}[prec_name]
    m = batch_measure(lbpc, workloads, prec, args.instances, args.steps, args.warmup, args.variant, args.ctas,
                      args.n, args.dT, clk_index=local)
    line = {
        "metric": "batched coupled flow+thermal MLUPS (aggregate)", "value": m["value"], "unit": "MLUPS",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == lbpc.FP64 else "f32", "data": "synthetic",
        "config": {"workload": m["workload"], "instances": m["instances"], "nodes": m["nodes"],
                   "storage": prec_name, "tile": m["tile"], "ctas_per_sm": m["ctas_per_sm"],
                   "graph_chunk": m["graph_chunk"], "autotune": m["autotune"], "l2": m["l2"]},
        "plain_path": m["plain_path"], "batched_over_plain": m["batched_over_plain"],
        "roofline": dict(m["hbm"], bound="hbm"),
        "gpu_launches": m["launches"], "clocks": m["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args):
    """Served stream: Poisson arrivals of mixed evaporation / heated-wall requests, admitted by the
    arena budget, advanced together by continuous batching; p50/p99 time-to-result and aggregate
    MLUPS. A bounded sample of the 2000-request stream (smaller sides and step counts)."""
    import torch

    from paper_1709_04400_gb300 import build, lbpc, serve

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    prec = {"": lbpc.FP32, "fp32": lbpc.FP32, "fp16": lbpc.FP16DEV, "fp64": lbpc.FP64}[args.prec]
    if args.full_stream:  # the full request distribution: sides 64-1024, 5k-50k steps
        lo_hi = dict(side_lo=64, side_hi=1024, steps_lo=5000, steps_hi=50000)
    else:
        lo_hi = dict(side_lo=64, side_hi=512, steps_lo=1000, steps_hi=5000)
    reqs = serve.poisson_stream(args.requests, rate=args.rate, seed=170904400 + 4, **lo_hi)
    srv = serve.Server(prec=prec, hbm_budget_bytes=24 << 30)

    # the stream runs alongside one 4096 x 4096 FP16-deviation evaporation run on its own CUDA stream,
    # stepped by a host thread (the library calls release the GIL), whose throughput measures the
    # roofline under co-scheduling; its standalone rate is measured first for comparison
    side = None
    if not args.no_side_run:
        import threading

        from paper_1709_04400_gb300 import workloads

        p0 = lbpc.Params(nx=8, ny=8)
        Tc, _ = lbpc.eos_critical(p0)
        rv, rl, _ = lbpc.coexistence(p0, 0.86 * Tc)
        n4 = 4096
        c4, r4, t4 = workloads.droplet_evaporation(Tc, rv, rl, n=n4, radius=0.2 * n4, dT_ratio=0.1)
        s4 = torch.cuda.Stream()
        big = lbpc.Simulation(lbpc.params_from_case(c4, lbpc.FP16DEV), stream=s4)
        big.init(r4, t4)
        big.step(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s4)
        big.step(50)
        e1.record(s4)
        e1.synchronize()
        alone_glups = n4 * n4 * 50 / e0.elapsed_time(e1) / 1e6
        stop, done, err = threading.Event(), [0], []

        def side_loop():
            e0.record(s4)
            try:
                while not stop.is_set():
                    big.step(20)
                    done[0] += 20
            except lbpc.LbpcError as e:
                err.append(str(e))
            e1.record(s4)
            s4.synchronize()

        th = threading.Thread(target=side_loop)
        th.start()
    with ClockSampler(local) as clk:
        srv.run(reqs)
    st = srv.stats()
    srv.close()
    if not args.no_side_run:
        stop.set()
        th.join()
        big.close()
        glups = n4 * n4 * done[0] / e0.elapsed_time(e1) / 1e6
        side = {"workload": f"droplet_evaporation_{n4}_fp16dev", "steps": done[0], "glups_alongside": glups,
                "glups_alone": alone_glups, "bytes_per_node": 96,
                "hbm_frac_alongside": glups * 1e9 * 96 / 1e9 / _peak_hbm(), "hbm_frac_alone":
                alone_glups * 1e9 * 96 / 1e9 / _peak_hbm(), "error": err[0] if err else None}
    if rank == 0:
        line = {"metric": "served coupled flow+thermal MLUPS (aggregate)", "value": st["aggregate_mlups"],
                "unit": "MLUPS", "n_gpus": 1, "steps": None, "warmup": 0, "ms_per_step": None,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == lbpc.FP64 else "f32", "data": "synthetic",
                "config": {"workload": f"served_stream_{args.requests}", "rate_per_s": args.rate,
                           "sides": [lo_hi["side_lo"], lo_hi["side_hi"]], "steps": [lo_hi["steps_lo"], lo_hi["steps_hi"]],
                           "mix": "half evaporation, half heated wall",
                           "storage": args.prec or "fp32", "budget_gb": 24},
                "latency": {"p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"]},
                "served": st, "side_run": side, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import eos, model

    a, b, R, om = 3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344
    Tc = eos.critical_temperature(a, b, R)
    rv, rl, _ = eos.maxwell_coexistence(0.86 * Tc, a, b, R, om)
    case, rho, T, prec_name = make_case(args, Tc, rv, rl)
    keys = set(model.OracleParams.__dataclass_fields__)
    p = model.OracleParams(**{k: v for k, v in case.items() if k in keys})
    s = model.init_state(p, rho, T)
    for _ in range(args.warmup):
        s = model.step(p, s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = model.step(p, s)
    dt = time.perf_counter() - t0
    N = case["nx"] * case["ny"]
    v = N * args.steps / dt / 1e6
    sample = f"{args.steps} oracle steps of {case['name']} ({dt:.1f} s, numpy FP64, 1 thread)"
    line = {"impl": "reference", "metric": "coupled flow+thermal MLUPS", "value": v, "unit": "MLUPS",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case["name"], "nx": case["nx"], "ny": case["ny"], "nodes": N,
                       "storage": "fp64", "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    a = parse()
    if a.warmup < 3:
        a.warmup = 3
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "serve":
        run_serve(a)
    else:
        run_native(a)
