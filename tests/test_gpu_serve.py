"""GPU tests of the continuous-batching server: a job returns the same bits
alone and in a mix of other jobs (other ligands, receptors and sizes), the
same bits as dock() (ADADELTA and Solis-Wets jobs), and admission,
rejection, cancellation and waiting behave as documented.  Failures are
made on the host (cancelled or oversized jobs); nothing faults the GPU."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    return T


@pytest.fixture(scope="module")
def pkg(torch):
    import paper_2410_10447_gb300 as P
    P.load(build=True)
    return P


@pytest.fixture(scope="module")
def world():
    recs = [synth.make_receptor(synth.generate.BASE_SEED + 3 + k, n, 10) for k, n in enumerate((32, 40))]
    ligs = [synth.make_ligand(500 + k, na, 10, nt) for k, (na, nt) in
            enumerate([(16, 4), (40, 10), (90, 20), (12, 0)])]
    return recs, ligs


def params(pkg, seed, runs=3, pop=24, gens=3, iters=20, **kw):
    return pkg.adgb.dock_params(n_runs=runs, pop=pop, max_gens=gens, ls_iters=iters, seed=seed, **kw)


def test_job_same_alone_and_in_mix(pkg, torch, world):
    recs, ligs = world
    ctx = pkg.Context(0)
    rids = [ctx.upload_receptor_grids(r) for r in recs]
    srv = pkg.Server(ctx)
    a = srv.submit(rids[0], ligs[0], params(pkg, 41))
    assert srv.wait(a, 60000)["status"] == 0
    ga, ea, va = srv.result(a)
    b = srv.submit(rids[1], ligs[1], params(pkg, 42, runs=2, pop=30, gens=4))
    a2 = srv.submit(rids[0], ligs[0], params(pkg, 41))
    c = srv.submit(rids[1], ligs[2], params(pkg, 43, runs=1, pop=40, gens=2))
    d = srv.submit(rids[0], ligs[3], params(pkg, 44, runs=4, pop=16, gens=5, iters=15))
    for j in (b, a2, c, d):
        info = srv.wait(j, 120000)
        assert info is not None and info["status"] == 0, info
    g2, e2, v2 = srv.result(a2)
    assert np.array_equal(ga, g2) and np.array_equal(ea, e2) and np.array_equal(va, v2)
    # the mixed jobs, run alone afterwards, also reproduce their results
    gc, ec, _ = srv.result(c)
    c2 = srv.submit(rids[1], ligs[2], params(pkg, 43, runs=1, pop=40, gens=2))
    srv.wait(c2, 120000)
    gc2, ec2, _ = srv.result(c2)
    assert np.array_equal(gc, gc2) and np.array_equal(ec, ec2)
    st = srv.stats()
    assert st["ticks"] > 0 and st["queued"] == 0 and st["active"] == 0
    srv.stop()
    ctx.close()


@pytest.mark.parametrize("conv", [None, (1, 5, 1e6), (2, 5, 0.5)])
def test_job_equals_dock_call(pkg, torch, world, conv):
    """A served job gives what dock() gives, also with early stopping (runs
    that stop early stop at the same generation)."""
    recs, ligs = world
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(recs[0])
    lid = ctx.upload_ligand_torsion_tree(ligs[0])
    prm = params(pkg, 7, runs=3, pop=20, gens=6 if conv else 3, iters=25)
    if conv:
        prm.conv_every, prm.conv_top, prm.conv_tol = conv
    gd, ed, vd = ctx.dock(rid, lid, prm)
    srv = pkg.Server(ctx)
    j = srv.submit(rid, ligs[0], prm)
    info = srv.wait(j, 60000)
    assert info["status"] == 0
    if conv and conv[2] > 1e5:
        assert info["generations"] == 1      # every run converged at the first test
    gs, es, vs = srv.result(j)
    # the same kernels, launch shape and launch order as dock(): the same bits
    assert np.array_equal(vd, vs)
    assert np.array_equal(gs, gd[:, :gs.shape[1]])
    assert np.array_equal(es, ed)
    srv.stop()
    ctx.close()


@pytest.mark.parametrize("variant", [0, 3])
def test_solis_wets_job_equals_dock_call(pkg, torch, world, variant):
    """Jobs whose local search is Solis-Wets (ls_method 1) are served too, with
    dock()'s bits; mixed with ADADELTA jobs of other ligands."""
    recs, ligs = world
    ctx = pkg.Context(0)
    rids = [ctx.upload_receptor_grids(r) for r in recs]
    lid = ctx.upload_ligand_torsion_tree(ligs[1])
    prm = params(pkg, 17, runs=3, pop=20, gens=3, iters=30, ls_method=1, reduce_variant=variant)
    gd, ed, vd = ctx.dock(rids[1], lid, prm)
    srv = pkg.Server(ctx)
    other = srv.submit(rids[0], ligs[0], params(pkg, 18, reduce_variant=variant))
    j = srv.submit(rids[1], ligs[1], prm)
    assert srv.wait(j, 60000)["status"] == 0 and srv.wait(other, 60000)["status"] == 0
    gs, es, vs = srv.result(j)
    assert np.array_equal(vd, vs) and np.array_equal(es, ed)
    assert np.array_equal(gs, gd[:, :gs.shape[1]])
    assert vs.sum() > 0
    srv.stop()
    ctx.device_status()   # no tensor-core completion wait gave up
    ctx.close()


def test_admission_rejection_cancel_timeout(pkg, torch, world):
    recs, ligs = world
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(recs[0])
    prm = params(pkg, 9, runs=2, pop=16, gens=2, iters=10)
    # the device bytes of one such job, seen while it runs
    srv = pkg.Server(ctx)
    probe = srv.submit(rid, ligs[0], params(pkg, 9, runs=2, pop=16, gens=100000, iters=10))
    job_bytes = 0
    for _ in range(2000):
        st = srv.stats()
        if st["active"] == 1:
            job_bytes = st["device_bytes_in_use"]
            break
    srv.cancel(probe)
    assert srv.wait(probe, 60000)["status"] == -7 and job_bytes > 0
    srv.stop()
    # a budget that holds one such job at a time: jobs run one after another
    srv = pkg.Server(ctx, mem_budget_bytes=int(1.5 * job_bytes))
    ids = [srv.submit(rid, ligs[0], params(pkg, 100 + k, runs=2, pop=16, gens=2, iters=10)) for k in range(3)]
    infos = [srv.wait(j, 60000) for j in ids]
    assert all(i["status"] == 0 for i in infos)
    for x, y in zip(infos, infos[1:]):
        assert y["start_s"] >= x["finish_s"] - 1e-9
    # a job that can never fit is rejected at submission
    with pytest.raises(pkg.AdgbError) as ei:
        srv.submit(rid, ligs[0], params(pkg, 1, runs=50, pop=1000, gens=1, iters=2))
    assert ei.value.code == -6
    # a bad ligand is refused on the calling thread
    bad = dict(ligs[0])
    bad["n_atoms"] = 300
    with pytest.raises(pkg.AdgbError) as ei:
        srv.submit(rid, bad, prm)
    assert ei.value.code == -1
    srv.stop()
    # cancellation of a running and a queued job; a short wait times out
    srv = pkg.Server(ctx, max_active_jobs=1)
    long_prm = params(pkg, 5, runs=8, pop=100, gens=2000, iters=300)
    j1 = srv.submit(rid, ligs[0], long_prm)
    j2 = srv.submit(rid, ligs[0], long_prm)
    assert srv.wait(j1, 1) is None
    srv.cancel(j2)
    srv.cancel(j1)
    i1, i2 = srv.wait(j1, 60000), srv.wait(j2, 60000)
    assert i1["status"] == -7 and i2["status"] == -7
    with pytest.raises(pkg.AdgbError):
        srv.result(j1)
    srv.forget(j1)
    with pytest.raises(pkg.AdgbError):
        srv.poll(j1)
    srv.stop()
    ctx.close()
