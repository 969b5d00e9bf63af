"""Times local-search launches on a named synthetic workload.

    python -m benchmarks.run_ls [--workload lga_n32] [--iters 300]
        [--n 0] [--cfgs 32:4,64:2] [--variants 0,1,2] [--reps 3] [--method adadelta|sw]
        [--gpw 0,1]

For every launch shape "threads_per_pose:poses_per_block" and reduction
variant it runs one warm-up launch and `reps` timed launches (CUDA events)
and prints the best time and evaluations/s.  --gpw lists the
genotypes_per_warp options to run (0: two genotypes a warp where the ligand
qualifies, the default; 1: one).  Used for launch-shape sweeps
and as the target of ncu captures (one launch per repetition).  With
--method sw the launches are Solis-Wets searches of at most `iters`
evaluations (energy only) and the rate counts the evaluations spent.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import paper_2410_10447_gb300 as P
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lga_n32")
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--n", type=int, default=0, help="genotypes (0 = the workload's own)")
    ap.add_argument("--cfgs", default="32:4")
    ap.add_argument("--variants", default="0")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--method", default="adadelta", choices=["adadelta", "sw"])
    ap.add_argument("--gpw", default="0")
    a = ap.parse_args(argv)
    P.load(build=True)
    w = synth.workload(a.workload, n_poses=a.n or None)
    g0 = torch.from_numpy(w["genes"]).cuda()
    n = g0.shape[0]
    res = {}
    for cfg, gpw in [(c, int(x)) for c in a.cfgs.split(",") for x in a.gpw.split(",")]:
        tpp, ppb = map(int, cfg.split(":"))
        ctx = P.Context(0, threads_per_pose=tpp, poses_per_block=ppb, genotypes_per_warp=gpw)
        rid = ctx.upload_receptor_grids(w["receptor"])
        lid = ctx.upload_ligand_torsion_tree(w["ligand"])
        for v in map(int, a.variants.split(",")):
            best = torch.empty(n, device="cuda")
            g = torch.empty_like(g0)
            ms = []
            evc = torch.empty(n, dtype=torch.int32, device="cuda")
            swp = P.adgb.sw_params(max_evals=a.iters, reduce_variant=v)
            for _ in range(a.reps + 1):
                g.copy_(g0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                if a.method == "sw":
                    ctx.local_search_sw_dev(rid, lid, g, best, swp, evals=evc)
                else:
                    ctx.local_search_dev(rid, lid, g, best, a.iters, variant=v)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = min(ms[1:]) if a.reps else ms[0]
            evals = int(evc.sum()) if a.method == "sw" else n * a.iters
            key = "%s:%d:%d:v%d:g%d" % (a.method, tpp, ppb, v, gpw)
            res[key] = dict(ms=t, evals=evals, evals_per_s=evals / t * 1e3,
                            median_best=float(best.median()))
            print("%s %s tpp=%d ppb=%d variant=%d gpw=%d: %.3f ms  %.1f M evals/s  median best %.3f"
                  % (a.workload, a.method, tpp, ppb, v, gpw, t, evals / t / 1e3,
                     float(best.median())), flush=True)
        ctx.close()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
