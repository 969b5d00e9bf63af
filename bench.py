"""Benchmark: energy+gradient evaluations per second of Lamarckian-GA
docking on the batched workload `lga_n32`: 20 runs x 150 genotypes of a
32-atom, 8-torsion ligand against a 64^3 grid with 8+2 maps; 27 generations,
every individual locally searched with 300 ADADELTA evaluations.

One step = one whole dock() call: initial population scoring, 27 x (GA
generation + one fused local-search launch over all 3000 individuals + run
best/evaluation accounting), FP64 rescoring of the 20 run bests:
20 * 150 * (1 + 27 * 300) = 24.3M energy+gradient evaluations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl adgb|reference]
                  [--variant shfl|mma_tf32x2|mma_bf16x3]

Prints ONE JSON line (rank 0).  `value`: device time (CUDA events on the
launching stream; receptor and ligand resident; L2 flushed between steps,
flush not timed).  `e2e`: the same metric through the host C calls a
docking job makes (upload_ligand_torsion_tree, dock with host outputs,
release_ligand).  The roofline line is for the local-search kernel (98-99%
of the GPU time), measured from standalone launches of the same shape.
`--impl reference` times the FP64 CPU oracle's docking on a bounded sample.
Multi-GPU: `--gpus N` (N > 1) re-runs the command as N ranks of one node
(torch.distributed.run, 127.0.0.1) unless it already runs under a launcher;
every rank docks its own replica (weak scaling, no data-path collective),
the slowest rank's time gives the job rate.  `--dry-run` checks that launch
path with a host loop only.
"""
from __future__ import annotations

import argparse
import hashlib
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

WORKLOAD = "lga_n32"
ITERS = 300
RUNS, POP, GENS = 20, 150, 27
EVALS_PER_DOCK = RUNS * POP * (1 + GENS * ITERS)
# kernel launches of one dock(): state init, initial population, its scoring
# and accounting, then GA + local search + accounting per generation, rescoring
LAUNCHES_PER_DOCK = 4 + 3 * GENS + 1
# Algorithmic work per energy+gradient evaluation, counted from the method
# (what any implementation must compute; FMA = 2 flops), FP32 arithmetic and
# special-function (MUFU) operations kept apart:
#   grid terms      110 flops per atom (trilinear value and gradient of three
#                   maps, 24 gathers of 4 bytes)
#   pair terms      40 flops + 3 MUFU per pair: 1 reciprocal square root and
#                   2 exponentials (the dielectric's and the desolvation's)
#   pose            20 flops per moving atom of each torsion + 30 per atom
#   gene gradient   12 flops per moving atom of each torsion
#   reduction       8 adds per thread of a pose (the 8-wide reduce-and-broadcast)
#   ADADELTA        15 flops + 2 square roots per gene
# The roofline of the local-search kernel is the binding one of the FP32 pipe
# and the MUFU pipe: each fraction is its operations / its peak, the pipes
# working in parallel.
FLOP_GRID, FLOP_PAIR, FLOP_POSE_MOV, FLOP_POSE_ATOM = 110, 40, 20, 30
FLOP_GGRAD_MOV, FLOP_RED_THREAD, FLOP_GENE = 12, 8, 15
RSQ_PAIR, EX2_PAIR, SQRT_GENE = 1, 2, 2
SM_COUNT, FP32_LANES, SM_MHZ_MAX = 152, 128, 2070.0
# special-function results an SM completes a clock, by operation (from the
# ALU probe on GB300: ex2 10.0 T/s and rsqrt 5.0 T/s at 2070 MHz over 152 SMs)
MUFU_EX2_PER_SM_CLK, MUFU_RSQ_PER_SM_CLK = 32, 16


def eval_work(lig, threads_per_pose=32):
    """(FP32 flops, reciprocal-square-root-class MUFU ops, ex2 MUFU ops) per
    energy+gradient evaluation of `lig`."""
    N, T = lig["n_atoms"], lig["n_tors"]
    moving = int(lig["mov_off"][-1]) if T else 0     # sum of moving-set sizes
    P = len(lig["pairs"])
    G = 6 + T
    flops = (FLOP_GRID * N + FLOP_PAIR * P + FLOP_POSE_MOV * moving + FLOP_POSE_ATOM * N
             + FLOP_GGRAD_MOV * moving + FLOP_RED_THREAD * threads_per_pose + FLOP_GENE * G)
    return float(flops), float(RSQ_PAIR * P + SQRT_GENE * G), float(EX2_PAIR * P)


def alu_roofline(lig, evals_per_s, probe=None, sm_mhz=SM_MHZ_MAX):
    """FP32 and MUFU roofline fractions of a kernel doing `evals_per_s`
    evaluations of `lig`: against peaks derived from the unit counts and the
    clock, and against the measured ALU probe when given."""
    fl, rsq, ex2 = eval_work(lig)
    clk = sm_mhz * 1e6
    fp32_peak = SM_COUNT * FP32_LANES * 2 * clk / 1e12               # TFLOP/s
    rsq_peak = SM_COUNT * MUFU_RSQ_PER_SM_CLK * clk                  # ops/s
    ex2_peak = SM_COUNT * MUFU_EX2_PER_SM_CLK * clk
    fp32 = evals_per_s * fl / 1e12
    frac_fp32 = fp32 / fp32_peak
    frac_mufu = evals_per_s * (rsq / rsq_peak + ex2 / ex2_peak)
    out = {"bound": "alu", "achieved": fp32, "peak": fp32_peak, "unit": "TFLOP/s",
           "frac": max(frac_fp32, frac_mufu), "frac_fp32": frac_fp32, "frac_mufu": frac_mufu,
           "fp32_flops_per_eval": fl, "mufu_rsqrt_per_eval": rsq, "mufu_ex2_per_eval": ex2,
           "peak_basis": "derived: FP32 152 SMs x 128 lanes x 2 flops x %.0f MHz; MUFU 152 SMs "
                         "x (16 rsqrt-class, 32 ex2) a clock" % sm_mhz}
    if probe:
        out["frac_fp32_of_measured_ffma"] = fp32 / probe["ffma_tflops"]
        out["frac_mufu_of_measured"] = evals_per_s * (rsq / (probe["rsqrt_gops"] * 1e9)
                                                      + ex2 / (probe["ex2_gops"] * 1e9))
        out["measured_probe"] = probe
    return out


def alu_probe(ctx, torch, waves=8, threads=256, reps=2000):
    """Measured ALU peaks over the whole GPU: FP32 FMA TFLOP/s, packed FP32x2
    FMA TFLOP/s, ex2.approx and rsqrt.approx Gop/s (alu_bench_dev)."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    nb = props.multi_processor_count * waves
    out = torch.empty(nb * threads, device="cuda")
    res = {"sms": props.multi_processor_count}
    for kind, name in ((0, "ffma"), (1, "ex2"), (2, "rsqrt"), (3, "ffma2")):
        ctx.alu_bench_dev(kind, nb, threads, 10, out)
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.alu_bench_dev(kind, nb, threads, reps, out)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        rate = nb * threads * reps * 128.0 / (min(ms) / 1e3)
        if kind == 0:
            res["ffma_tflops"] = 2 * rate / 1e12
        elif kind == 3:
            res["ffma2_tflops"] = 4 * rate / 1e12
        else:
            res[name + "_gops"] = rate / 1e9
    return res


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(dist, t, device):
    """The slowest rank's time, on every rank (t itself without a process group)."""
    if not dist:
        return t
    import torch
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(world, units_per_rank, t_max):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units, timed by the slowest rank."""
    return world * units_per_rank / t_max


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index):
        self.index, self.rows, self.p = index, [], None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0])]
        util = [num(r[7]) for r in self.rows if len(r) > 7]
        loaded = [s for s, u in zip(sm, util) if u and u > 50] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 3 + i and r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": num(self.rows[0][1]), "samples": len(self.rows),
                "reasons": reasons}


def profile_traffic(kernel_sha):
    """DRAM bytes per launch of the local-search kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_ls_kernel_lga_n32.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        item = line.strip().lstrip("-* ")
        if ":" in item and item.startswith(("traffic_bytes_per_launch", "kernel_source_sha1")):
            k, v = item.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha1") != kernel_sha:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def kernel_sha():
    h = hashlib.sha1()
    for f in ("eval.cu", "reduce.cuh", "tcgen05.cuh", "adgb_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2410_10447_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def oracle_dock_sample(w, n_runs, gens, nthreads, seed):
    """FP64 oracle docking of n_runs runs x 150 genotypes for `gens`
    generations (a bounded sample of the benchmark's dock); returns
    (evaluations, seconds)."""
    import oracle
    prm = oracle.dock_params(n_runs=n_runs, pop=POP, max_gens=gens, ls_iters=ITERS,
                             ls_rate=1.0, seed=seed)
    t = time.perf_counter()
    _, _, ev = oracle.dock(w["receptor"], w["ligand"], prm, nthreads=nthreads)
    return int(ev.sum()), time.perf_counter() - t


def cpu_model():
    """The host CPU's model name (lscpu), or the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def reference_arm(args, rank, world):
    """FP64 CPU oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    w = synth.workload(WORKLOAD, n_poses=1)
    cores = os.cpu_count() or 1
    for i in range(args.warmup):
        oracle_dock_sample(w, args.ref_runs, 1, cores, 1000 + i)
    ev = t = 0
    for i in range(args.steps):
        e_i, t_i = oracle_dock_sample(w, args.ref_runs, 1, cores, 2000 + i)
        ev += e_i
        t += t_i
    v = ev / t
    sample = ("%d runs x %d genotypes x 1 generation (%d evaluations) per step, of the "
              "20 x 150 x 27-generation dock" % (args.ref_runs, POP, ev // args.steps))
    line = {"metric": "energy+gradient evals/s", "value": v, "unit": "evals/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD + ": 20 runs x 150 genotypes, 32 atoms, 8 torsions, "
                       "64^3 x (8+2) maps, 27 generations x 300 ADADELTA evaluations",
                       "sample": sample},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def launch_ranks(n):
    """Re-runs this command as n ranks of one node (torch.distributed.run,
    rendezvous on 127.0.0.1) and returns their exit status; rank 0 prints
    the line."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", str(n), "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.run(cmd).returncode


def dry_run(args, rank, world):
    """The N-rank host path without device work: every rank times a short
    host loop, the slowest rank's time gives the job rate, rank 0 prints."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist.barrier()
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        units += int(np.arange(20000).sum() > 0)
    t = max_over_ranks(dist, time.perf_counter() - t0, "cpu" if not torch.cuda.is_available()
                       else "cuda")
    if dist:
        dist.barrier()
    if rank == 0:
        print(json.dumps({"metric": "dry run (host loop iterations/s)", "dry_run": True,
                          "value": job_rate(world, units, t), "unit": "iterations/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak"}), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="adgb", choices=["adgb", "reference"])
    ap.add_argument("--variant", default="shfl")
    ap.add_argument("--ref-runs", type=int, default=16)
    ap.add_argument("--cpu-runs", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-variants", action="store_true")
    ap.add_argument("--dry-run", action="store_true",
                    help="rank set-up, barrier and max-over-ranks timing of a tiny host loop "
                         "only (no GPU work; gloo without CUDA): checks the launch path")
    args = ap.parse_args()
    rank, local_rank, world = dist_env()
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        sys.exit(launch_ranks(args.gpus))
    if args.dry_run:
        dry_run(args, rank, world)
        return
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import paper_2410_10447_gb300 as pkg
    import synth

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    pkg.load(build=(world == 1))
    variant = pkg.VARIANTS[args.variant]
    w = synth.workload(WORKLOAD)
    lig = w["ligand"]
    n, G = RUNS * POP, 6 + lig["n_tors"]
    ctx = pkg.Context(local_rank)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(lig)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    best_g = torch.empty(RUNS, G, device="cuda")
    best_e = torch.empty(RUNS, dtype=torch.float64, device="cuda")
    evals = torch.empty(RUNS, dtype=torch.int64, device="cuda")

    def params(i):
        # a distinct seed for every step and rank: distinct initial populations
        return pkg.adgb.dock_params(n_runs=RUNS, pop=POP, max_gens=GENS, max_evals=2_500_000,
                                    ls_iters=ITERS, ls_rate=1.0, reduce_variant=variant,
                                    seed=1_000_003 * (rank + 1) + i)

    def step(i):
        flush.fill_(i & 255)                       # evict L2 (256 MiB > 129 MB)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx.dock_dev(rid, lid, params(i), best_g, best_e, evals)
        ev1.record(stream)
        return ev0, ev1

    evs = []
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)                           # let the sampler start
        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            evs.append(step(args.warmup + i))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    dev_ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = sum(dev_ms) / 1e3
    assert int(evals.sum()) == EVALS_PER_DOCK, int(evals.sum())
    assert torch.isfinite(best_e).all()
    t_dev = max_over_ranks(dist, t_dev, "cuda")
    evals_rank = args.steps * EVALS_PER_DOCK
    value = job_rate(world, evals_rank, t_dev)

    # end to end through the host C calls of one docking job per step
    lig_bytes = sum(np.asarray(lig[k]).nbytes for k in ("type", "charge", "xyz", "tors_bond",
                                                           "mov_off", "mov_atoms", "pairs"))
    for i in range(2):
        l2 = ctx.upload_ligand_torsion_tree(lig)
        ctx.dock(rid, l2, params(10_000 + i))
        ctx.release_ligand(l2)
    if dist:
        dist.barrier()
    e2e_ms = []
    for i in range(args.steps):
        t1 = time.perf_counter()
        l2 = ctx.upload_ligand_torsion_tree(lig)
        _, be_h, ev_h = ctx.dock(rid, l2, params(args.warmup + i))
        ctx.release_ligand(l2)
        e2e_ms.append(1e3 * (time.perf_counter() - t1))
    t_e2e = sum(e2e_ms) / 1e3
    t_e2e = max_over_ranks(dist, t_e2e, "cuda")
    e2e = job_rate(world, evals_rank, t_e2e)

    # the local-search kernel alone, same launch shape as inside dock()
    g0 = torch.from_numpy(synth.make_poses(7, n, w["receptor"], lig["n_tors"])).cuda()
    gls = torch.empty_like(g0)
    bls = torch.empty(n, device="cuda")
    ls_ms = []
    for i in range(6):
        gls.copy_(g0)
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.local_search_dev(rid, lid, gls, bls, ITERS, variant=variant)
        b.record(stream)
        torch.cuda.synchronize()
        ls_ms.append(a.elapsed_time(b))
    ls_ms = ls_ms[1:]
    extra = {}
    if args.compare_variants:
        for name, vv in pkg.VARIANTS.items():
            ms = []
            for i in range(3):
                gls.copy_(g0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.local_search_dev(rid, lid, gls, bls, ITERS, variant=vv)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            extra[name] = n * ITERS / (min(ms) / 1e3)
    # measured FP32 FMA and special-function throughput (after the timed region)
    probe = alu_probe(ctx, torch)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    launch_s = statistics.mean(ls_ms) / 1e3
    clocks = clk.summary()
    roof = alu_roofline(lig, n * ITERS / launch_s, probe)
    roof["traffic"] = profile_traffic(kernel_sha())
    roof["kernel"] = "eval_kernel (local search, 3000 genotypes x 300 evaluations)"
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        ev_c, t_c = oracle_dock_sample(w, args.cpu_runs, 1, cores, 77)
        ev_1, t_1 = oracle_dock_sample(w, 1, 1, 1, 78)
        cpu = {"value": ev_c / t_c, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle dock of %d runs x %d genotypes x 1 generation (%d "
                         "evaluations), OpenMP over runs" % (args.cpu_runs, POP, ev_c),
               "single_thread": {"value": ev_1 / t_1, "sample": "1 run x %d genotypes x 1 "
                                 "generation (%d evaluations), one thread" % (POP, ev_1)},
               "cpu_model": cpu_model()}
    q = lambda v, p: float(np.percentile(v, p))
    line = {
        "metric": "energy+gradient evals/s", "value": value, "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + ": dock of 20 runs x 150 genotypes, 32-atom 8-torsion "
                   "%d-pair ligand, 64^3 x (8+2) maps, 27 generations x 300 ADADELTA "
                   "evaluations, FP64 rescoring" % len(lig["pairs"]),
                   "evals_per_step": EVALS_PER_DOCK, "reduce_variant": args.variant,
                   "l2": "flushed between steps (256 MiB write), flush not timed",
                   "dock_latency_ms": {"p50": q(dev_ms, 50), "p99": q(dev_ms, 99)},
                   "e2e_dock_latency_ms": {"p50": q(e2e_ms, 50), "p99": q(e2e_ms, 99)},
                   "poses_per_s": world * args.steps * RUNS * POP * GENS / t_dev,
                   "ls_kernel_evals_per_s": n * ITERS / launch_s,
                   "wall_s_timed_region": wall},
        "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": int(lig_bytes),
                "d2h_bytes_per_step": RUNS * (G * 4 + 8 + 8)},
        "gpu_launches": args.steps * LAUNCHES_PER_DOCK,
        "roofline": roof,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if extra:
        line["variants_ls_evals_per_s"] = extra
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
