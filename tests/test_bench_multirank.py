"""The N > 1 host path of bench.py on CPU: two gloo ranks, each timing its
own replica (weak scaling), agree on the slowest rank's time; the job rate
is world x per-rank units / that time; only rank 0 runs the reference arm."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = bench.dist_env()
    t = bench.max_over_ranks(dist, 1.5 + rank, "cpu")      # rank r took 1.5 + r seconds
    rate = bench.job_rate(w, 1000, t)
    buf = io.StringIO()

    class A:
        steps, warmup, ref_runs = 1, 0, 1
    if r != 0:
        with contextlib.redirect_stdout(buf):
            bench.reference_arm(A, r, w)                   # other ranks do no work
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, lr, w, t, rate, buf.getvalue()))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, local_rank, world, t, rate, printed) in enumerate(res):
        assert (rank, local_rank, world) == (r, r, 2)
        assert t == pytest.approx(2.5)
        assert rate == pytest.approx(2 * 1000 / 2.5)
        assert printed == ""


def test_bench_gpus_2_launches_two_ranks():
    """`bench.py --gpus 2` re-runs itself as two ranks (torch.distributed.run
    on 127.0.0.1; gloo without CUDA) and reports n_gpus = the ranks run."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                          "--dry-run", "--steps", "2"], capture_output=True, text=True,
                         timeout=240, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    rec = json.loads(lines[0])
    assert rec["n_gpus"] == 2 and rec["dry_run"] is True
