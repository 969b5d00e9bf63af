"""Docking time with and without early stopping (convergence detection).

    python -m benchmarks.run_dock [--workload lga_n32] [--runs 20]
        [--pop 150] [--gens 100] [--every 5] [--top 15] [--tol 0.15] [--reps 3]

Docks the workload's ligand (runs x pop, up to `gens` generations of 300
ADADELTA evaluations) once with the early-stopping test off and once with it
on, and prints one JSON line: wall time per dock (CUDA events), evaluations,
the distribution of generations the runs took, and the best energies.
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
    import numpy as np
    import torch

    import paper_2410_10447_gb300 as P
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lga_n32")
    ap.add_argument("--runs", type=int, default=20)
    ap.add_argument("--pop", type=int, default=150)
    ap.add_argument("--gens", type=int, default=100)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--every", type=int, default=5)
    ap.add_argument("--top", type=int, default=15)
    ap.add_argument("--tol", type=float, default=0.15)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    P.load(build=True)
    w = synth.workload(a.workload)
    ctx = P.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    G = 6 + w["ligand"]["n_tors"]
    out = {"workload": a.workload, "runs": a.runs, "pop": a.pop, "max_gens": a.gens,
           "ls_iters": a.iters, "test": {"every": a.every, "top": a.top, "tol": a.tol}}
    for name, every in (("off", 0), ("on", a.every)):
        prm = P.adgb.dock_params(n_runs=a.runs, pop=a.pop, max_gens=a.gens, ls_iters=a.iters,
                                 max_evals=10 ** 12, conv_every=every, conv_top=a.top,
                                 conv_tol=a.tol)
        bg = torch.empty(a.runs, G, device="cuda")
        be = torch.empty(a.runs, dtype=torch.float64, device="cuda")
        ev = torch.empty(a.runs, dtype=torch.int64, device="cuda")
        ms = []
        for _ in range(a.reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.dock_dev(rid, lid, prm, bg, be, ev)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        evals = ev.cpu().numpy()
        gens = (evals - a.pop) // (a.pop * a.iters)
        energies = be.cpu().numpy()
        out[name] = {"ms_per_dock": min(ms[1:]), "evals": int(evals.sum()),
                     "evals_per_s": float(evals.sum() / (min(ms[1:]) / 1e3)),
                     "generations": {"min": int(gens.min()), "median": float(np.median(gens)),
                                     "max": int(gens.max()), "hist": np.bincount(gens).tolist()},
                     "best_energy": {"min": float(energies.min()),
                                     "median": float(np.median(energies))}}
        print(name, json.dumps(out[name]), flush=True)
    out["speedup"] = out["off"]["ms_per_dock"] / out["on"]["ms_per_dock"]
    print(json.dumps(out), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
