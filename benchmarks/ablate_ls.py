"""Share of each step of the two-genotypes-a-warp local search (ligands of at
most 32 atoms): times ls_ablation_dev launches with one step left out at
compile time and reports each step's share as the time saved.

    python -m benchmarks.ablate_ls [--workload lga_n32] [--iters 300] [--variants 0,3] [--n 0]

The launches are the local-search launch of the workload (its genotypes, one
launch of `iters` evaluations each), best of `reps` after one warm-up; the
outputs of a launch with steps left out are not energies.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

STEPS = {0: "whole evaluation", 1: "pair rounds", 2: "grid terms",
         12: "reduce-and-broadcast + torsion moving-set sums", 8: "torsion moving-set sums (shuffle)",
         16: "torsion-tree walk", 32: "gene-gradient formulas", 64: "sines and cosines",
         3: "pair rounds + grid terms", 128: "pair-term arithmetic (exchanges kept)",
         256: "pair-round shuffles (arithmetic kept)",
         512: "one tcgen05 MMA a block instead of one a warp (design, not a step)"}


def main(argv=None):
    import torch

    import paper_2410_10447_gb300 as P
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lga_n32")
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--variants", default="0,3")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--n", type=int, default=0,
                    help="genotypes (0 = the workload's own); few genotypes (1-2 warps an SM) "
                         "give each step's share of one warp's dependency chain")
    a = ap.parse_args(argv)
    P.load(build=True)
    w = synth.workload(a.workload, n_poses=a.n or None)
    g0 = torch.from_numpy(w["genes"]).cuda()
    n = g0.shape[0]
    ctx = P.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    best = torch.empty(n, device="cuda")
    g = torch.empty_like(g0)
    res = {}
    for v in map(int, a.variants.split(",")):
        row = {}
        for mask, name in STEPS.items():
            if (mask == 8 and v == 3) or (mask == 512 and v != 3):
                continue   # tensor-core form: moving-set sums in its MMA; 512 is its design
            ms = []
            for _ in range(a.reps + 1):
                g.copy_(g0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.ls_ablation_dev(rid, lid, g, best, a.iters, v, mask)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            row[mask] = min(ms[1:])
        base = row[0]
        out = {STEPS[m]: {"ms": t, "share": (base - t) / base if m else 1.0} for m, t in row.items()}
        res["variant%d" % v] = out
        print("%s variant %d: whole %.3f ms" % (a.workload, v, base))
        for m, t in row.items():
            if m == 512:
                print("  design: %-48s %.3f ms  (%+.1f%% time)" % (STEPS[m], t, 100 * (t - base) / base))
            elif m:
                print("  without %-48s %.3f ms  share %5.1f%%" % (STEPS[m], t, 100 * (base - t) / base))
    ctx.close()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
