"""Benchmark: energy+gradient evaluations per second of the ADADELTA local
search on the batched-LGA workload (20 runs x 150 genotypes of a 32-atom,
8-torsion ligand on a 64^3 grid with 10 maps, 300 ADADELTA steps each).

One step = one local-search pass of the whole population: 3000 genotypes x
300 energy+gradient evaluations = 900,000 evaluations, one kernel launch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl adgb|reference]
                  [--variant shfl|mma_tf32x2|mma_bf16x3]

Prints ONE JSON line (rank 0).  `value` is device-timed (CUDA events on
the launching stream, inputs resident in HBM, L2 flushed between steps and
excluded); `e2e` is the same metric through the host-buffer C call
`local_search` (host->device genes, device->host genes and energies inside
the timed region).  `--impl reference` times the FP64 CPU oracle instead.
Multi-GPU (torchrun) runs one independent replica per rank (weak scaling).
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
# Algorithmic ALU work per energy+gradient evaluation, counted from the
# method (FMA = 2 flops; one MUFU op = 16 flop-equivalents, the FP32 pipe
# being 8x wider than the special-function pipe):
#   per atom  : pose transform 20 + 20 per enclosing torsion, grid term 80
#   per pair  : 50 FP32 flops + 5 MUFU ops (rsqrt, 2 exp, 2 rcp)
#   per gene  : ADADELTA 15;  per moving atom of a torsion 12 (torsion gradient)
FLOP_ATOM, FLOP_ATOM_TORS, FLOP_GRID, FLOP_PAIR, MUFU_PAIR, MUFU_EQ = 20, 20, 80, 50, 5, 16
FLOP_GENE, FLOP_MOVING = 15, 12
SM_COUNT, FP32_LANES = 152, 128


def eval_flops(lig) -> float:
    N, T = lig["n_atoms"], lig["n_tors"]
    moving = int(lig["mov_off"][-1]) if T else 0     # sum of moving-set sizes
    P = len(lig["pairs"])
    return (N * (FLOP_ATOM + FLOP_GRID) + moving * (FLOP_ATOM_TORS + FLOP_MOVING)
            + P * (FLOP_PAIR + MUFU_PAIR * MUFU_EQ) + (6 + T) * FLOP_GENE)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


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
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_source_sha1")):
            k, v = line.split(":", 1)
            vals[k.strip().strip("-* ")] = v.strip().strip("`")
    if vals.get("kernel_source_sha1") != kernel_sha:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def kernel_sha():
    h = hashlib.sha1()
    for f in ("eval.cu", "reduce.cuh", "adgb_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2410_10447_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def run_oracle_sample(w, n_geno, nthreads):
    import oracle
    t = time.perf_counter()
    oracle.local_search_batch(w["receptor"], w["ligand"], w["genes"][:n_geno], ITERS,
                              nthreads=nthreads)
    return time.perf_counter() - t


def reference_arm(args, rank, world):
    """FP64 CPU oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    w = synth.workload(WORKLOAD)
    cores = os.cpu_count() or 1
    n_geno = args.ref_genotypes
    for _ in range(args.warmup):
        run_oracle_sample(w, n_geno, cores)
    t = sum(run_oracle_sample(w, n_geno, cores) for _ in range(args.steps))
    evals = args.steps * n_geno * ITERS
    v = evals / t
    line = {"metric": "energy+gradient evals/s", "value": v, "unit": "evals/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD + ": 20 runs x 150 genotypes, 32 atoms, 8 torsions, "
                       "64^3 x 10 maps, 300 ADADELTA steps", "sample_genotypes": n_geno},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": "%d genotypes x %d steps per step (of 3000 x 300)" % (n_geno, ITERS)},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="adgb", choices=["adgb", "reference"])
    ap.add_argument("--variant", default="shfl")
    ap.add_argument("--ref-genotypes", type=int, default=400)
    ap.add_argument("--cpu-genotypes", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-variants", action="store_true")
    args = ap.parse_args()
    rank, local_rank, world = dist_env()
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
    pkg.load(build=(rank == 0 and world == 1))
    variant = pkg.VARIANTS[args.variant]
    w = synth.workload(WORKLOAD)
    lig = w["ligand"]
    n, G = w["genes"].shape
    ctx = pkg.Context(local_rank)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(lig)
    # a distinct seeded population for every step
    pops = [synth.make_poses(synth.generate.BASE_SEED + 1000 * (rank + 1) + s, n, w["receptor"],
                             lig["n_tors"]) for s in range(args.warmup + args.steps)]
    pops_dev = [torch.from_numpy(p).cuda() for p in pops]
    genes = torch.empty_like(pops_dev[0])
    best = torch.empty(n, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(i, var):
        genes.copy_(pops_dev[i])
        flush.fill_(i & 255)                       # evict L2 (256 MiB > 129 MB)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx.local_search_dev(rid, lid, genes, best, ITERS, variant=var)
        ev1.record(stream)
        return ev0, ev1

    evs = []
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)                       # let the sampler start
        for i in range(args.warmup):
            step(i, variant)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            evs.append(step(args.warmup + i, variant))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    dev_ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = sum(dev_ms) / 1e3
    assert torch.isfinite(best).all()
    if dist:
        tt = torch.tensor([t_dev], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev = float(tt.item())
    evals_rank = args.steps * n * ITERS
    value = world * evals_rank / t_dev

    # end to end through the host-buffer C call (pinned host memory)
    pin_g = [torch.from_numpy(p).pin_memory() for p in pops]
    pin_e = torch.empty(n, dtype=torch.float32).pin_memory()
    for i in range(2):
        ctx.local_search_host_ptr(rid, lid, pin_g[i].data_ptr(), n, ITERS, pin_e.data_ptr(),
                                  variant=variant)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        ctx.local_search_host_ptr(rid, lid, pin_g[args.warmup + i].data_ptr(), n, ITERS,
                                  pin_e.data_ptr(), variant=variant)
    t_e2e = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    e2e = world * evals_rank / t_e2e

    extra = {}
    if args.compare_variants:
        for name, vv in pkg.VARIANTS.items():
            ms = []
            for i in range(3):
                a, b = step(i, vv)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            extra[name] = n * ITERS / (min(ms) / 1e3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # roofline of the local-search kernel (one launch per step)
    fl = eval_flops(lig)
    launch_s = t_dev / args.steps
    achieved = n * ITERS * fl / launch_s / 1e12
    clocks = clk.summary()
    peak = SM_COUNT * FP32_LANES * 2 * 2070e6 / 1e12
    traffic = profile_traffic(kernel_sha())
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        t = run_oracle_sample(w, args.cpu_genotypes, cores)
        cpu = {"value": args.cpu_genotypes * ITERS / t, "unit": "evals/s", "cores": cores,
               "kind": "oracle",
               "sample": "%d of the 3000 genotypes x %d ADADELTA steps, FP64, OpenMP" % (args.cpu_genotypes, ITERS)}
    line = {
        "metric": "energy+gradient evals/s", "value": value, "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + ": 20 runs x 150 genotypes of a 32-atom, 8-torsion, "
                   "%d-pair ligand, 64^3 grid x 10 maps, 300 ADADELTA steps" % len(lig["pairs"]),
                   "genotypes_per_gpu": n, "ls_iters": ITERS, "reduce_variant": args.variant,
                   "l2": "flushed between steps (256 MiB write), flush not timed",
                   "poses_per_s": world * args.steps * n / t_dev,
                   "wall_s_timed_region": wall},
        "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": n * G * 4,
                "d2h_bytes_per_step": n * G * 4 + n * 4},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "flops_per_eval": fl, "peak_basis": "FP32 FMA pipe, 152 SMs x 128 lanes x 2 x 2070 MHz"},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if extra:
        line["variants_evals_per_s"] = extra
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
