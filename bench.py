"""Benchmark: energy+gradient evaluations per second of Lamarckian-GA
docking on the batched workload `lga_n32`: 20 runs x 150 genotypes of a
32-atom, 8-torsion ligand against a 64^3 grid with 8+2 maps; 27 generations,
every individual locally searched with 300 ADADELTA evaluations.

One step = one whole dock() call: initial population scoring, 27 x (GA
generation + one fused local-search launch over all 3000 individuals + run
best/evaluation accounting), FP64 rescoring of the 20 run bests:
20 * 150 * (1 + 27 * 300) = 24.3M energy+gradient evaluations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl adgb|reference]
                  [--variant shfl|mma_tf32x2|mma_bf16x3|tcgen05] [--no-extras]

Prints ONE JSON line (rank 0).  `value`: device time (CUDA events on the
launching stream; receptor and ligand resident; L2 flushed between steps,
flush not timed).  `e2e`: the same metric through the host C calls a
docking job makes (upload_ligand_torsion_tree, dock with host outputs,
release_ligand).  The roofline line is for the local-search kernel (98-99%
of the GPU time), measured from standalone launches of the same shape.

After the timed region (rank 0, unless --no-extras) the line also carries:
  variants_ls_evals_per_s   the dock's local-search launch with each
                            reduction variant, two genotypes a warp (the
                            default) and one genotype a warp (the plain form)
  batch_uneven_512          one persistent graph-replayed launch of 512
                            ligands (autotuned, shuffle, tcgen05) vs the
                            plain form ligand by ligand
  serving                   10 serving-mix jobs served together vs docked one
                            after another; a Poisson stream at half the
                            saturation rate: time-to-result p50 / p99
  tensor_core_vs_plain_shfl the tensor-core forms over the plain FP32
                            warp-shuffle form on the same inputs
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
GRID_BYTES_ATOM = 96   # type map 32 B + e map 32 B + d map 32 B of the atom's cell
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


def l2_probe(ctx, torch, mb=64, waves=8, threads=256):
    """Measured L2 read bandwidth over the whole GPU (l2_bench_dev) on a
    buffer of `mb` MB that stays resident in L2: streaming (16-byte coalesced
    reads) and the scoring kernels' 96-byte cell gathers, GB/s."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    nb = props.multi_processor_count * waves
    buf = torch.ones(mb * (1 << 20) // 4, device="cuda")
    out = torch.empty(nb * threads, device="cuda")
    res = {"buffer_mb": mb}
    for kind, name, reps, per in ((0, "stream", 2000, 16), (1, "gather96", 400, 96)):
        ctx.l2_bench_dev(kind, buf, nb, threads, 20, out)
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.l2_bench_dev(kind, buf, nb, threads, reps, out)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name + "_gbs"] = nb * threads * reps * per / (min(ms) / 1e3) / 1e9
    return res


def grid_roofline(lig, evals_per_s, l2):
    """The grid gathers' L2 roofline: their algorithmic bytes (96 a ligand
    atom and evaluation) at the local search's rate, against the measured L2
    streaming and gather bandwidths."""
    gbs = evals_per_s * lig["n_atoms"] * GRID_BYTES_ATOM / 1e9
    return {"bound": "l2", "achieved": gbs, "peak": l2["stream_gbs"], "unit": "GB/s",
            "frac": gbs / l2["stream_gbs"], "frac_of_gather_probe": gbs / l2["gather96_gbs"],
            "bytes_per_eval": lig["n_atoms"] * GRID_BYTES_ATOM,
            "peak_basis": "measured: l2_bench_dev streaming reads of a %d MB L2-resident "
                          "buffer (gathers of 96 B: %.0f GB/s)" % (l2["buffer_mb"], l2["gather96_gbs"])}


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
    """Digest of the sources the profiled kernel (eval_pair_kernel) is built from."""
    h = hashlib.sha1()
    for f in ("eval_pair.cu", "reduce.cuh", "tcgen05.cuh", "adgb_internal.cuh"):
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


def time_launch(torch, fn, reps=3, flush=None):
    """Best CUDA-event time (ms) of fn() over `reps` runs after one warm-up,
    L2 flushed before each when a flush buffer is given."""
    ms = []
    for r in range(reps + 1):
        if flush is not None:
            flush.fill_(r & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return min(ms[1:])


def ls_variants(pkg, torch, w, rid_of, flush):
    """The local-search launch of the dock (3000 genotypes x 300 evaluations)
    with each reduction variant, in both kernel forms: two genotypes a warp
    (the library's default for this ligand) and one genotype a warp (the
    plain warp-shuffle form of the method)."""
    import synth
    n = RUNS * POP
    g0 = torch.from_numpy(synth.make_poses(7, n, w["receptor"], w["ligand"]["n_tors"])).cuda()
    g = torch.empty_like(g0)
    best = torch.empty(n, device="cuda")
    out = {}
    for gpw, key in ((0, "two_genotypes_a_warp"), (1, "one_genotype_a_warp")):
        ctx = pkg.Context(torch.cuda.current_device(), genotypes_per_warp=gpw)
        rid = ctx.upload_receptor_grids(w["receptor"])
        lid = ctx.upload_ligand_torsion_tree(w["ligand"])
        row = {}
        for name, v in pkg.VARIANTS.items():
            def run():
                g.copy_(g0)
                ctx.local_search_dev(rid, lid, g, best, ITERS, variant=v)
            row[name] = n * ITERS / (time_launch(torch, run, 3, flush) / 1e3)
        out[key] = row
        ctx.close()
    return out


def batch_phase(pkg, torch, flush, iters=300, poses=64):
    """uneven_512 (512 ligands of 10-128 atoms and 0-32 torsions, 64
    genotypes each, 300 evaluations, 72^3 grid): one graph-replayed
    persistent launch (autotuned shape; then with the tcgen05 reduction
    forced) against the plain form, one single-ligand shuffle launch per
    ligand with one genotype a warp."""
    import numpy as np
    import synth
    wb = synth.WORKLOADS["uneven_512"]
    rec = synth.make_receptor(synth.generate.BASE_SEED + wb["index"], wb["grid"], wb["n_type_maps"])
    ligs = synth.make_uneven_batch(synth.generate.BASE_SEED + wb["index"], wb["n_ligands"],
                                   wb["atoms"], wb["tors"], wb["n_types"])
    genes = [synth.make_poses(7000 + i, poses, rec, L["n_tors"]) for i, L in enumerate(ligs)]
    packed = np.zeros((len(ligs) * poses, pkg.adgb.MAX_GENES), np.float32)
    for i, gg in enumerate(genes):
        packed[i * poses:(i + 1) * poses, :gg.shape[1]] = gg
    dev = torch.cuda.current_device()
    ctx = pkg.Context(dev)
    rid = ctx.upload_receptor_grids(rec)
    lids = [ctx.upload_ligand_torsion_tree(L) for L in ligs]
    g0 = torch.from_numpy(packed).cuda()
    g = torch.empty_like(g0)
    e = torch.empty(g0.shape[0], device="cuda")
    bid = ctx.batch_create([rid] * len(ligs), lids, [poses] * len(ligs))
    tuned = ctx.batch_autotune(bid, g0, iters=15)
    evals = len(ligs) * poses * iters
    res = {"workload": "uneven_512: 512 ligands (10-128 atoms, 0-32 torsions) x 64 genotypes x "
                       "%d ADADELTA evaluations, 72^3 x (10+2) maps" % iters, "autotuned": tuned}
    for name, v in (("batched_autotuned", -1), ("batched_shfl", 0), ("batched_tcgen05", 3)):
        def run():
            g.copy_(g0)
            ctx.batch_local_search_dev(bid, g, e, iters, variant=v)
        res[name + "_evals_per_s"] = evals / (time_launch(torch, run, 3, flush) / 1e3)
    ctx.batch_release(bid)
    ctx.close()
    plain = pkg.Context(dev, genotypes_per_warp=1)
    rid = plain.upload_receptor_grids(rec)
    lids = [plain.upload_ligand_torsion_tree(L) for L in ligs]
    gs = [torch.from_numpy(x).cuda() for x in genes]
    gs0 = [x.clone() for x in gs]
    es = [torch.empty(poses, device="cuda") for _ in genes]

    def run_plain():
        for i in range(len(ligs)):
            gs[i].copy_(gs0[i])
            plain.local_search_dev(rid, lids[i], gs[i], es[i], iters, variant=0)
    res["plain_shfl_ligand_by_ligand_evals_per_s"] = evals / (time_launch(torch, run_plain, 1, flush) / 1e3)
    plain.close()
    base = res["plain_shfl_ligand_by_ligand_evals_per_s"]
    res["batched_tcgen05_vs_plain_shfl"] = res["batched_tcgen05_evals_per_s"] / base
    res["batched_autotuned_vs_plain_shfl"] = res["batched_autotuned_evals_per_s"] / base
    return res


def serving_phase(pkg, burst=10, window=30.0, pool_n=24, seed=1):
    """The serving workload's jobs (ligands of 10-256 atoms and 0-40 torsions
    against one of four resident receptors, 48^3-96^3 grids with 10+2 maps;
    10 runs x 150 genotypes and 2.5e6 evaluations a run): a burst of `burst`
    jobs served together (the saturation throughput) against the same jobs
    docked one after another with dock(), then a Poisson stream at half the
    saturation rate for `window` seconds (time-to-result p50 / p99)."""
    import numpy as np
    import synth
    ws = synth.WORKLOADS["serving"]
    rng = np.random.default_rng(seed)
    recs = [synth.make_receptor(synth.generate.BASE_SEED + ws["index"] + 10 * k, n, ws["n_type_maps"])
            for k, n in enumerate(ws["grids"])]
    pool = []
    for k in range(pool_n):
        na = int(rng.integers(ws["atoms"][0], ws["atoms"][1] + 1))
        nt = int(rng.integers(ws["tors"][0], ws["tors"][1] + 1))
        pool.append(synth.make_ligand(90000 + k, na, ws["n_type_maps"], nt))
    ctx = pkg.Context(0)
    rids = [ctx.upload_receptor_grids(r) for r in recs]
    runs, pop, evals_run, iters = 10, 150, 2_500_000, 300
    gens = evals_run // (pop * iters) + 2

    def prm(k, variant=-1):
        return pkg.adgb.dock_params(n_runs=runs, pop=pop, max_gens=gens, max_evals=evals_run,
                                    ls_iters=iters, seed=seed * 1_000_000 + k, reduce_variant=variant)
    choice = rng.integers(0, pool_n, burst)
    recv = rng.integers(0, len(rids), burst)
    out = {"job": "10 runs x 150 genotypes, 2.5e6 evaluations a run, ligands of 10-256 atoms "
                  "and 0-40 torsions, receptors 48^3-96^3 x (10+2) maps", "burst_jobs": burst}

    # warm-up: every burst job's kernels (both reduction forms) launched once
    # (one generation each), so that no timed phase pays first-launch loading
    for k in range(burst):
        lid = ctx.upload_ligand_torsion_tree(pool[int(choice[k])])
        for v in (0, 3):
            wp = pkg.adgb.dock_params(n_runs=runs, pop=pop, max_gens=1, ls_iters=iters,
                                      seed=k, reduce_variant=v)
            ctx.dock(rids[recv[k]], lid, wp)
        ctx.release_ligand(lid)

    def served(variant):
        srv = pkg.Server(ctx, reduce_variant=variant)
        t0 = time.perf_counter()
        ids = [srv.submit(rids[recv[k]], pool[choice[k]], prm(k, variant)) for k in range(burst)]
        infos = [srv.wait(j, -1) for j in ids]
        wall = time.perf_counter() - t0
        srv.stop()
        assert all(i["status"] == 0 for i in infos)
        return wall, sum(i["evals"] for i in infos)
    wall_s, ev_s = served(-1)
    wall_tc, ev_tc = served(3)
    # the same jobs one after another: each arrives with its ligand (upload,
    # which builds the pair schedule as dock_submit does), is docked, released
    t_ser, ev_ser = 0.0, 0
    for k in range(burst):
        t1 = time.perf_counter()
        lid = ctx.upload_ligand_torsion_tree(pool[int(choice[k])])
        _, _, ev = ctx.dock(rids[recv[k]], lid, prm(k, 0))
        ctx.release_ligand(lid)
        t_ser += time.perf_counter() - t1
        ev_ser += int(ev.sum())
    sat = burst / wall_s
    out.update(served_evals_per_s=ev_s / wall_s, served_tcgen05_evals_per_s=ev_tc / wall_tc,
               serial_dock_shfl_evals_per_s=ev_ser / t_ser,
               served_vs_serial=(ev_s / wall_s) / (ev_ser / t_ser),
               served_tcgen05_vs_serial_shfl=(ev_tc / wall_tc) / (ev_ser / t_ser),
               saturation_jobs_per_s=sat)
    # Poisson arrivals at half the saturation rate
    rate = 0.5 * sat
    n_jobs = int(rng.poisson(rate * window))
    arrivals = np.sort(rng.uniform(0.0, window, n_jobs))
    ch = rng.integers(0, pool_n, n_jobs)
    rv = rng.integers(0, len(rids), n_jobs)
    srv = pkg.Server(ctx)
    t0 = time.perf_counter()
    ids = []
    for k in range(n_jobs):
        d = arrivals[k] - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        ids.append(srv.submit(rids[rv[k]], pool[ch[k]], prm(1000 + k)))
    infos = [srv.wait(j, -1) for j in ids]
    srv.stop()
    lat = np.array([i["finish_s"] - i["submit_s"] for i in infos if i["status"] == 0])
    out.update(poisson_rate_jobs_per_s=rate, poisson_window_s=window, poisson_jobs=n_jobs,
               serve_p50_ms=1e3 * float(np.percentile(lat, 50)) if len(lat) else None,
               serve_p99_ms=1e3 * float(np.percentile(lat, 99)) if len(lat) else None)
    ctx.close()
    return out


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
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the reduction-variant, uneven-batch and serving phases")
    ap.add_argument("--serve-window", type=float, default=30.0)
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
    if not args.no_extras and rank == 0:
        extra["variants_ls_evals_per_s"] = ls_variants(pkg, torch, w, rid, flush)
        extra["batch_uneven_512"] = batch_phase(pkg, torch, flush)
        extra["serving"] = serving_phase(pkg, window=args.serve_window)
    # measured FP32 FMA and special-function throughput (after the timed region)
    probe = alu_probe(ctx, torch)
    l2bw = l2_probe(ctx, torch)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    launch_s = statistics.mean(ls_ms) / 1e3
    clocks = clk.summary()
    roof = alu_roofline(lig, n * ITERS / launch_s, probe)
    roof["traffic"] = profile_traffic(kernel_sha())
    roof["kernel"] = ("eval_pair_kernel (local search, two genotypes a warp, 3000 genotypes x 300 "
                      "evaluations)")
    roof_grid = grid_roofline(lig, n * ITERS / launch_s, l2bw)
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
        "roofline_grid_l2": roof_grid,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if extra:
        v = extra["variants_ls_evals_per_s"]
        plain = v["one_genotype_a_warp"]["shfl"]
        extra["tensor_core_vs_plain_shfl"] = {
            "ls_two_genotypes_a_warp_tcgen05": v["two_genotypes_a_warp"]["tcgen05"] / plain,
            "ls_two_genotypes_a_warp_shfl": v["two_genotypes_a_warp"]["shfl"] / plain,
            "batched_tcgen05": extra["batch_uneven_512"]["batched_tcgen05_vs_plain_shfl"],
            "served_tcgen05": extra["serving"]["served_tcgen05_vs_serial_shfl"]}
        line.update(extra)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
