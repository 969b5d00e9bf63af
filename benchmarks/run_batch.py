"""Uneven batch benchmark: many ligands of different sizes, each with its own
genotypes, locally searched by one persistent multi-ligand launch replayed
from a CUDA graph, against the same work done ligand by ligand.

    python -m benchmarks.run_batch [--ligands 512] [--poses 64]
        [--iters 300] [--reps 3] [--no-autotune] [--no-serial] [--variant V]
        [--shape THREADS:POSES]

Workload uneven_512: ligands with atom counts uniform in [10, 128] and
torsions uniform in [0, 32] (10 atom types), 64 genotypes each, 300 ADADELTA
evaluations, one shared 72^3 grid with 10 + 2 maps.  --variant forces the
batch's reduction (REDUCE_*) over the autotuner's pick; the ligand-by-ligand
comparison always uses the shuffle reduction.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import numpy as np
    import torch

    import paper_2410_10447_gb300 as P
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--ligands", type=int, default=512)
    ap.add_argument("--poses", type=int, default=64)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-serial", action="store_true")
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--shape", default="", help="THREADS:POSES instead of autotuning")
    ap.add_argument("--pair-rounds", type=int, default=0, help="adgb_options.pair_rounds")
    a = ap.parse_args(argv)
    P.load(build=True)
    w = synth.WORKLOADS["uneven_512"]
    t0 = time.time()
    rec = synth.make_receptor(synth.generate.BASE_SEED + w["index"], w["grid"], w["n_type_maps"])
    ligs = synth.make_uneven_batch(synth.generate.BASE_SEED + w["index"], a.ligands, w["atoms"],
                                   w["tors"], w["n_types"])
    t_gen = time.time() - t0
    if a.shape:
        tpp, ppb = (int(x) for x in a.shape.split(":"))
        ctx = P.Context(0, threads_per_pose=tpp, poses_per_block=ppb, pair_rounds=a.pair_rounds)
        a.no_autotune = True
    else:
        ctx = P.Context(0, pair_rounds=a.pair_rounds)
    rid = ctx.upload_receptor_grids(rec)
    lids = [ctx.upload_ligand_torsion_tree(L) for L in ligs]
    genes = [synth.make_poses(7000 + i, a.poses, rec, L["n_tors"]) for i, L in enumerate(ligs)]
    packed = np.zeros((a.ligands * a.poses, P.adgb.MAX_GENES), np.float32)
    for i, g in enumerate(genes):
        packed[i * a.poses:(i + 1) * a.poses, :g.shape[1]] = g
    g0 = torch.from_numpy(packed).cuda()
    bid = ctx.batch_create([rid] * a.ligands, lids, [a.poses] * a.ligands)
    tuned = None
    if not a.no_autotune:
        tuned = ctx.batch_autotune(bid, g0, iters=max(5, a.iters // 20))
    g = torch.empty_like(g0)
    e = torch.empty(g0.shape[0], device="cuda")
    ms = []
    for r in range(a.reps + 1):
        g.copy_(g0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        ctx.batch_local_search_dev(bid, g, e, a.iters, variant=a.variant)
        ev1.record()
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    t_batch = min(ms[1:])
    evals = a.ligands * a.poses * a.iters
    out = dict(workload="uneven_512", ligands=a.ligands, poses_per_ligand=a.poses, iters=a.iters,
               atoms_mean=float(np.mean([L["n_atoms"] for L in ligs])),
               pairs_mean=float(np.mean([len(L["pairs"]) for L in ligs])),
               batch_ms=t_batch, batch_evals_per_s=evals / t_batch * 1e3, autotuned=tuned,
               variant=a.variant, shape=a.shape or None, pair_rounds=a.pair_rounds,
               first_call_ms_incl_capture=ms[0], generate_s=t_gen)
    if not a.no_serial:
        # the same work as one single-ligand launch per ligand, back to back
        gs = [torch.from_numpy(x).cuda() for x in genes]
        es = [torch.empty(a.poses, device="cuda") for _ in genes]
        sms = []
        for r in range(2):
            for i in range(a.ligands):
                gs[i].copy_(torch.from_numpy(genes[i]))
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for i in range(a.ligands):
                ctx.local_search_dev(rid, lids[i], gs[i], es[i], a.iters, variant=P.REDUCE_SHFL)
            ev1.record()
            torch.cuda.synchronize()
            sms.append(ev0.elapsed_time(ev1))
        out.update(serial_ms=min(sms), serial_evals_per_s=evals / min(sms) * 1e3,
                   batch_speedup=min(sms) / t_batch)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
