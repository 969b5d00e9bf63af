"""Reduction micro-benchmark (the test kernel of Sec. 5.2): every thread of a
block holds one four-element vector and the block computes the sum that every
thread receives.  Times each variant for block sizes 64..1024 and reports the
speed-up over the per-component shuffle + shared-atomic reduction profiled in
Sec. 3.

    python -m benchmarks.reduce_bench [--reps 1000] [--waves 4]
    python -m benchmarks.reduce_bench --alu

--alu instead measures the arithmetic units the scoring kernels are bound by:
FP32 fused multiply-add throughput (TFLOP/s) and special-function-unit
throughput (ex2.approx, rsqrt.approx; operations/s).
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

    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=1000, help="reductions per launch")
    ap.add_argument("--waves", type=int, default=4, help="blocks = 152 x waves")
    ap.add_argument("--threads", default="64,128,256,512,1024")
    ap.add_argument("--alu", action="store_true")
    a = ap.parse_args(argv)
    P.load(build=True)
    ctx = P.Context(0)
    if a.alu:
        import bench
        print(json.dumps(bench.alu_probe(ctx, torch)), flush=True)
        return
    names = {"paper_reducefs": P.REDUCE4_PAPER_FS, "paper_half": P.REDUCE4_PAPER_HALF,
             "shfl": 0, "mma_tf32x2": 1, "mma_bf16x3": 2,
             "tcgen05_tf32x2": P.REDUCE4_TCGEN05_TF32X2}
    res = {}
    for th in map(int, a.threads.split(",")):
        nb = 152 * a.waves
        x = torch.randn(nb * th * 4, device="cuda")
        xd = x.double().view(nb, th, 4)
        exact = xd.sum(dim=1)
        mag = xd.abs().sum(dim=1)
        row, err = {}, {}
        for name, v in names.items():
            if name == "tcgen05_tf32x2" and th % 64:
                continue
            out = ctx.reduce4_bench_dev(v, x, th, reps=1)
            got = out.view(nb, th, 4)[:, 0, :].double()
            err[name] = float(((got - exact).abs() / mag).max())
            ctx.reduce4_bench_dev(v, x, th, reps=a.reps, out=out)
            ms = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.reduce4_bench_dev(v, x, th, reps=a.reps, out=out)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            row[name] = min(ms) * 1e3 / a.reps   # microseconds per block-wide reduction wave
        base = row["paper_reducefs"]
        res[th] = {k: {"us_per_reduction": v, "speedup_vs_reducefs": base / v,
                       "max_err_over_sum_abs": err[k]} for k, v in row.items()}
        print(th, {k: round(base / v, 2) for k, v in row.items()}, flush=True)
    print(json.dumps({"blocks": 152 * a.waves, "reps": a.reps, "results": res}), flush=True)


if __name__ == "__main__":
    main()
