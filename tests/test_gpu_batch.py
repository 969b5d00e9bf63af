"""GPU tests of uneven batches: one persistent multi-ligand local-search
launch (graph-captured) over ligands of different sizes, checked against
the single-ligand path and the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
MAXG = 46


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
def setup():
    rec = synth.make_receptor(synth.generate.BASE_SEED + 2, 48, 10)
    ligs = synth.make_uneven_batch(11, 9, atoms=(10, 128), tors=(0, 32), n_types=10)
    ligs.append(synth.make_ligand(77, 256, 10, 40, chain_bias=0.7))   # one large ligand
    n_poses = [5, 9, 1, 12, 3, 8, 7, 2, 10, 6]
    genes = [synth.make_poses(100 + i, n, rec, L["n_tors"]) for i, (L, n) in enumerate(zip(ligs, n_poses))]
    return rec, ligs, n_poses, genes


def pack(genes):
    rows = sum(g.shape[0] for g in genes)
    out = np.zeros((rows, MAXG), np.float32)
    r = 0
    for g in genes:
        out[r:r + g.shape[0], :g.shape[1]] = g
        r += g.shape[0]
    return out


def test_batch_scores_match_single_ligand_calls(pkg, torch, setup):
    rec, ligs, n_poses, genes = setup
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(rec)
    lids = [ctx.upload_ligand_torsion_tree(L) for L in ligs]
    bid = ctx.batch_create([rid] * len(ligs), lids, n_poses)
    g = torch.from_numpy(pack(genes)).cuda()
    e = torch.empty(g.shape[0], device="cuda")
    ctx.batch_local_search_dev(bid, g, e, 1)          # one evaluation = scoring
    got = e.cpu().numpy()
    r = 0
    for i, L in enumerate(ligs):
        e_ref, _ = ctx.score_poses(rid, lids[i], genes[i], with_grad=False)
        assert np.allclose(got[r:r + n_poses[i]], e_ref, rtol=1e-5, atol=1e-4), i
        # genes are untouched by a one-evaluation search
        assert np.array_equal(g.cpu().numpy()[r:r + n_poses[i], :genes[i].shape[1]], genes[i])
        r += n_poses[i]
    ctx.close()


@pytest.mark.parametrize("autotune, variant, tpp", [(False, -1, 0), (True, -1, 0), (False, 3, 0),
                                                   (False, -1, 128), (False, 3, 128)])
def test_batch_local_search_returns_its_best(pkg, torch, setup, autotune, variant, tpp):
    """tpp 128: the 256-atom ligand takes the block form of the matching
    rounds inside the multi-ligand kernel (two atoms a thread)."""
    rec, ligs, n_poses, genes = setup
    ctx = pkg.Context(0, threads_per_pose=tpp, poses_per_block=128 // tpp) if tpp else pkg.Context(0)
    rid = ctx.upload_receptor_grids(rec)
    lids = [ctx.upload_ligand_torsion_tree(L) for L in ligs]
    bid = ctx.batch_create([rid] * len(ligs), lids, n_poses)
    g0 = torch.from_numpy(pack(genes)).cuda()
    if autotune:
        cfg = ctx.batch_autotune(bid, g0, iters=5)
        assert cfg["threads_per_pose"] in (32, 64, 128) and 1 <= cfg["poses_per_block"] <= 8
        assert np.array_equal(g0.cpu().numpy(), pack(genes))      # autotune leaves genes alone
    g = g0.clone()
    e = torch.empty(g.shape[0], device="cuda")
    ctx.batch_local_search_dev(bid, g, e, 40, variant=variant)        # captured
    g2 = g0.clone()
    e2 = torch.empty_like(e)
    ctx.batch_local_search_dev(bid, g2, e2, 40, variant=variant)      # other buffers: captured again
    g2.copy_(g0)
    ctx.batch_local_search_dev(bid, g2, e2, 40, variant=variant)      # same buffers: graph replayed
    assert np.array_equal(e.cpu().numpy(), e2.cpu().numpy())
    assert np.array_equal(g.cpu().numpy(), g2.cpu().numpy())
    be = e.cpu().numpy()
    gb = g.cpu().numpy()
    r = 0
    for i, L in enumerate(ligs):
        R, OL = oracle.Receptor(rec), oracle.Ligand(L)
        G = 6 + L["n_tors"]
        for k in range(n_poses[i]):
            e_ref = oracle.score(R, OL, gb[r + k, :G])[0]
            assert abs(be[r + k] - e_ref) <= max(1e-4 * abs(e_ref), 1e-3), (i, k, be[r + k], e_ref)
            e0 = oracle.score(R, OL, genes[i][k])[0]
            assert be[r + k] <= e0 + max(1e-4 * abs(e0), 1e-3)
        r += n_poses[i]
    ctx.batch_release(bid)
    ctx.close()


def test_uneven_512_full_size_sampled(pkg, torch):
    """The uneven workload at its full size in the launch configuration
    run_batch times (512 ligands of 10-128 atoms x 64 genotypes x 300
    evaluations, one autotuned, graph-replayed persistent launch): sampled
    genotypes' returned energies equal the FP64 oracle's energy of the
    returned genotypes, and are no higher than their start energies."""
    w = synth.WORKLOADS["uneven_512"]
    rec = synth.make_receptor(synth.generate.BASE_SEED + w["index"], w["grid"], w["n_type_maps"])
    ligs = synth.make_uneven_batch(synth.generate.BASE_SEED + w["index"], 512, w["atoms"], w["tors"],
                                   w["n_types"])
    poses = 64
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(rec)
    lids = [ctx.upload_ligand_torsion_tree(L) for L in ligs]
    genes = [synth.make_poses(7000 + i, poses, rec, L["n_tors"]) for i, L in enumerate(ligs)]
    g0 = torch.from_numpy(pack(genes)).cuda()
    bid = ctx.batch_create([rid] * len(ligs), lids, [poses] * len(ligs))
    ctx.batch_autotune(bid, g0, iters=15)
    g = g0.clone()
    e = torch.empty(g0.shape[0], device="cuda")
    ctx.batch_local_search_dev(bid, g, e, 300)
    be, gb = e.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.isfinite(be))
    rng = np.random.default_rng(0)
    R = oracle.Receptor(rec)
    for i in sorted(rng.choice(len(ligs), 12, replace=False)):
        L = oracle.Ligand(ligs[i])
        G = 6 + ligs[i]["n_tors"]
        for k in rng.choice(poses, 2, replace=False):
            row = i * poses + k
            e_ref = oracle.score(R, L, gb[row, :G])[0]
            assert abs(be[row] - e_ref) <= max(1e-4 * abs(e_ref), 1e-3), (i, k, be[row], e_ref)
            e0 = oracle.score(R, L, genes[i][k])[0]
            assert be[row] <= e0 + max(1e-4 * abs(e0), 1e-3)
    ctx.batch_release(bid)
    ctx.close()
