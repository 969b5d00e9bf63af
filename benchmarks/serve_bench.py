"""Serving benchmark: an open-loop Poisson stream of docking jobs into the
continuous-batching server.

    python -m benchmarks.serve_bench [--rate 200] [--duration 60]
        [--runs 10] [--pop 150] [--evals-per-run 2.5e6] [--ls-iters 300]
        [--pool 48] [--max-active 0] [--seed 1] [--variant -1] [--serial] [--burst N]

Jobs: ligands of 10-256 atoms and 0-40 torsions (a seeded pool, sampled
uniformly), each against one of four resident receptors (48^3, 64^3, 80^3,
96^3 grids at 0.375 A, 10 + 2 maps).  Prints one JSON line: offered and
completed jobs, evaluations/s over the busy period, and the p50/p99 of
time-to-result (submission to results ready) and of queueing delay.
--burst N: instead of the stream, N jobs submitted at once (the saturation
measurement).  --variant: the server's reduction (REDUCE_*; -1 = the context's default,
the shuffle form).  --serial: afterwards the same jobs are docked one after
another through the plain dock() call with the shuffle reduction, and the
line adds their wall time, evaluations/s and the served/serial ratio of
evaluations/s over wall time.
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

    import paper_2410_10447_gb300 as P
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--runs", type=int, default=10)
    ap.add_argument("--pop", type=int, default=150)
    ap.add_argument("--evals-per-run", type=float, default=2.5e6)
    ap.add_argument("--ls-iters", type=int, default=300)
    ap.add_argument("--pool", type=int, default=48)
    ap.add_argument("--max-active", type=int, default=0)
    ap.add_argument("--grids", default="48,64,80,96")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--serial", action="store_true")
    ap.add_argument("--burst", type=int, default=0)
    a = ap.parse_args(argv)
    P.load(build=True)
    w = synth.WORKLOADS["serving"]
    rng = np.random.default_rng(a.seed)
    grids = [int(x) for x in a.grids.split(",")]
    recs = [synth.make_receptor(synth.generate.BASE_SEED + w["index"] + 10 * k, n, w["n_type_maps"])
            for k, n in enumerate(grids)]
    pool = []
    for k in range(a.pool):
        na = int(rng.integers(w["atoms"][0], w["atoms"][1] + 1))
        nt = int(rng.integers(w["tors"][0], w["tors"][1] + 1))
        pool.append(synth.make_ligand(90000 + k, na, w["n_type_maps"], nt))
    ctx = P.Context(0)
    rids = [ctx.upload_receptor_grids(r) for r in recs]
    srv = P.Server(ctx, max_active_jobs=a.max_active, reduce_variant=a.variant)
    # arrival times and job choices, all seeded
    n_jobs = a.burst if a.burst else rng.poisson(a.rate * a.duration)
    arrivals = np.zeros(n_jobs) if a.burst else np.sort(rng.uniform(0.0, a.duration, n_jobs))
    choice = rng.integers(0, a.pool, n_jobs)
    recv = rng.integers(0, len(rids), n_jobs)
    gens = int(a.evals_per_run // (a.pop * a.ls_iters)) + 2
    # warm-up: every job's kernels launched once (one generation each, both the
    # served and the serial reduction forms), so that neither the stream nor the
    # serial pass pays first-launch loading
    for c in sorted(set(int(x) for x in choice)):
        lid = ctx.upload_ligand_torsion_tree(pool[c])
        for v in sorted({a.variant if a.variant >= 0 else P.REDUCE_SHFL, P.REDUCE_SHFL}):
            wp = P.adgb.dock_params(n_runs=a.runs, pop=a.pop, max_gens=1, ls_iters=a.ls_iters,
                                    seed=c, reduce_variant=v)
            ctx.dock(rids[0], lid, wp)
        ctx.release_ligand(lid)
    jobs = []
    t0 = time.perf_counter()
    for k in range(n_jobs):
        delay = arrivals[k] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        prm = P.adgb.dock_params(n_runs=a.runs, pop=a.pop, max_gens=gens,
                                 max_evals=int(a.evals_per_run), ls_iters=a.ls_iters,
                                 seed=a.seed * 1_000_000 + k)
        jobs.append(srv.submit(rids[recv[k]], pool[choice[k]], prm))
    t_submitted = time.perf_counter() - t0
    infos = [srv.wait(j, -1) for j in jobs]
    t_end = time.perf_counter() - t0
    st = srv.stats()
    srv.stop()
    done = [i for i in infos if i["status"] == 0]
    lat = np.array([i["finish_s"] - i["submit_s"] for i in done])
    queue = np.array([i["start_s"] - i["submit_s"] for i in done])
    evals = sum(i["evals"] for i in done)
    q = lambda v, p: float(np.percentile(v, p)) if len(v) else None
    serial = None
    if a.serial:
        # the same jobs, one plain dock() call after another (shuffle reduction)
        lig_ids, t_serial, ev_serial = {}, 0.0, 0
        for k in range(n_jobs):
            c = int(choice[k])
            if c not in lig_ids:
                lig_ids[c] = ctx.upload_ligand_torsion_tree(pool[c])
            prm = P.adgb.dock_params(n_runs=a.runs, pop=a.pop, max_gens=gens,
                                     max_evals=int(a.evals_per_run), ls_iters=a.ls_iters,
                                     seed=a.seed * 1_000_000 + k, reduce_variant=P.REDUCE_SHFL)
            t1 = time.perf_counter()
            _, _, ev = ctx.dock(rids[recv[k]], lig_ids[c], prm)
            t_serial += time.perf_counter() - t1
            ev_serial += int(ev.sum())
        serial = dict(wall_s=t_serial, evals=ev_serial, evals_per_s=ev_serial / t_serial,
                      variant="shfl",
                      served_over_serial=(evals / t_end) / (ev_serial / t_serial))
    print(json.dumps(dict(
        variant=a.variant, serial=serial,
        rate_hz=a.rate, duration_s=a.duration, offered_jobs=int(n_jobs), completed_jobs=len(done),
        runs=a.runs, pop=a.pop, evals_per_run=a.evals_per_run, ls_iters=a.ls_iters,
        evals_total=int(evals), wall_s=t_end, submit_window_s=t_submitted,
        evals_per_s=evals / max(st["busy_s"], 1e-9), jobs_per_s=len(done) / t_end,
        gpu_busy_s=st["busy_s"], ticks=st["ticks"],
        latency_s={"p50": q(lat, 50), "p99": q(lat, 99), "max": q(lat, 100)},
        queue_s={"p50": q(queue, 50), "p99": q(queue, 99)})), flush=True)


if __name__ == "__main__":
    main()
