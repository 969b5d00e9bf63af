"""GPU tests of the two-genotypes-a-warp kernels (ligands of at most 32
atoms, every FP32 operation packed across the two genotypes; the tcgen05
variant computes the reduce-and-broadcast and the torsions' moving-set sums
in one tensor-core product with the ligand's 0/1 mask matrix).

  - a genotype's results do not depend on the genotype sharing its warp, nor
    on running alone (odd counts): bit-identical energies, gradients, best
    genotypes and ADADELTA state under re-pairing;
  - both kernels (two genotypes a warp, and one) match the FP64 oracle within
    the stated tolerances (energy max(1e-4 |E|, 1e-3 kcal/mol), gene gradient
    1e-3 / 2e-3 (split-precision variants) of max(|g|_inf, 1));
  - the persistent multi-ligand form (batches, serving) gives the same bits
    as the single-ligand calls;
  - per-genotype iteration counts that differ inside a warp (the LGA's local
    searches with ls_rate < 1) leave the GA's accounting and results as with
    one genotype a warp.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

E_REL, E_ABS = 1e-4, 1e-3
G_TOL = {0: 1e-3, 1: 2e-3, 2: 2e-3, 3: 2e-3}
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
def cfg1():
    return synth.workload("lga_n32", n_poses=37)


def near_face(rec, x, tol=1e-4):
    u = (np.asarray(x, np.float64) - np.asarray(rec["origin"], np.float64)) / rec["spacing"]
    return bool(np.any(np.abs(u - np.round(u)) * rec["spacing"] < tol))


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_pairing_leaves_each_genotype_unchanged(pkg, torch, cfg1, variant):
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    genes = cfg1["genes"][:9]
    perm = np.array([4, 0, 8, 2, 6, 1, 3, 5, 7])        # every genotype gets another partner
    e1, g1 = ctx.score_poses(rid, lid, genes, variant=variant)
    e2, g2 = ctx.score_poses(rid, lid, genes[perm], variant=variant)
    assert np.array_equal(e1[perm], e2) and np.array_equal(g1[perm], g2)
    e3, g3 = ctx.score_poses(rid, lid, genes[4:5], variant=variant)   # alone in its warp
    assert np.array_equal(e3, e1[4:5]) and np.array_equal(g3, g1[4:5])
    b1, gb1, st1 = ctx.local_search(rid, lid, genes.copy(), 40, variant=variant, want_state=True)
    b2, gb2, st2 = ctx.local_search(rid, lid, genes[perm].copy(), 40, variant=variant,
                                    want_state=True)
    assert np.array_equal(b1[perm], b2) and np.array_equal(gb1[perm], gb2)
    assert np.array_equal(st1[perm], st2)
    b3, gb3, _ = ctx.local_search(rid, lid, genes[8:9].copy(), 40, variant=variant)
    assert np.array_equal(b3, b1[8:9]) and np.array_equal(gb3, gb1[8:9])
    ctx.close()


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("gpw", [0, 1])
def test_both_kernels_match_oracle(pkg, torch, cfg1, variant, gpw):
    ctx = pkg.Context(0, genotypes_per_warp=gpw)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    genes = cfg1["genes"]
    e, g = ctx.score_poses(rid, lid, genes, variant=variant)
    R, L = oracle.Receptor(cfg1["receptor"]), oracle.Ligand(cfg1["ligand"])
    compared = 0
    for p in range(genes.shape[0]):
        er, gr, x, _ = oracle.score(R, L, genes[p])
        assert abs(e[p] - er) <= max(E_REL * abs(er), E_ABS), (p, e[p], er)
        if near_face(cfg1["receptor"], x):
            continue
        err = np.max(np.abs(g[p] - gr)) / max(np.max(np.abs(gr)), 1.0)
        assert err <= G_TOL[variant], (p, err)
        compared += 1
    assert compared >= genes.shape[0] // 2
    # the searches return energies of the genotypes they return
    best, gb, _ = ctx.local_search(rid, lid, genes.copy(), 60, variant=variant)
    for p in range(0, genes.shape[0], 4):
        er = oracle.score(R, L, gb[p])[0]
        assert abs(best[p] - er) <= max(E_REL * abs(er), E_ABS), (p, best[p], er)
    ctx.close()


@pytest.mark.parametrize("variant", [0, 3])
def test_paired_batch_equals_single_ligand_calls(pkg, torch, variant):
    rec = synth.make_receptor(synth.generate.BASE_SEED + 5, 48, 10)
    ligs = synth.make_uneven_batch(21, 6, atoms=(10, 32), tors=(0, 20), n_types=10)
    n_poses = [7, 4, 1, 9, 2, 6]
    genes = [synth.make_poses(300 + i, n, rec, L["n_tors"]) for i, (L, n) in enumerate(zip(ligs, n_poses))]
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(rec)
    lids = [ctx.upload_ligand_torsion_tree(L) for L in ligs]
    bid = ctx.batch_create([rid] * len(ligs), lids, n_poses)
    rows = sum(n_poses)
    packed = np.zeros((rows, MAXG), np.float32)
    r = 0
    for gg in genes:
        packed[r:r + gg.shape[0], :gg.shape[1]] = gg
        r += gg.shape[0]
    g = torch.from_numpy(packed).cuda()
    e = torch.empty(rows, device="cuda")
    ctx.batch_local_search_dev(bid, g, e, 30, variant=variant)
    be, gb = e.cpu().numpy(), g.cpu().numpy()
    r = 0
    for i in range(len(ligs)):
        b1, g1, _ = ctx.local_search(rid, lids[i], genes[i].copy(), 30, variant=variant)
        assert np.array_equal(be[r:r + n_poses[i]], b1), i
        assert np.array_equal(gb[r:r + n_poses[i], :g1.shape[1]], g1), i
        r += n_poses[i]
    ctx.batch_release(bid)
    ctx.close()


def test_mixed_iteration_counts_in_a_warp(pkg, torch):
    """ls_rate 0.5: about half the individuals are scored once, the others
    searched; a warp often holds one of each.  The GA's decisions and
    evaluation counts equal those of one genotype a warp, and the run bests
    agree within the energy tolerance (the two kernels round differently)."""
    w = synth.workload("plain_n16", n_poses=4)
    res = []
    for gpw in (0, 1):
        ctx = pkg.Context(0, genotypes_per_warp=gpw)
        rid = ctx.upload_receptor_grids(w["receptor"])
        lid = ctx.upload_ligand_torsion_tree(w["ligand"])
        prm = pkg.adgb.dock_params(n_runs=4, pop=30, max_gens=1, ls_iters=6, ls_rate=0.5, seed=99)
        res.append(ctx.dock(rid, lid, prm))
        ctx.close()
    (g0, e0, v0), (g1, e1, v1) = res
    assert np.array_equal(v0, v1)
    assert np.all(np.abs(e0 - e1) <= np.maximum(E_REL * np.abs(e1), E_ABS)), (e0, e1)


def test_tcgen05_wait_give_up_is_reported(pkg, torch, cfg1):
    """The failure path of the tensor-core waits, without a GPU fault: the
    test form of the tcgen05 kernel issues nothing to the tensor core, so
    every warp's first completion wait gives up after a short bounded wait.
    The give-up is reported once (device_status for the asynchronous call,
    the next synchronous call otherwise), and the context keeps working with
    the same bits as before."""
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    genes = cfg1["genes"][:12]
    e0, g0 = ctx.score_poses(rid, lid, genes, variant=3)
    ctx.device_status()                                  # nothing to report
    g = torch.from_numpy(genes.copy()).cuda()
    best = torch.empty(genes.shape[0], device="cuda")
    ctx.ls_ablation_dev(rid, lid, g, best, 5, 3, 1024)
    with pytest.raises(pkg.adgb.AdgbError) as ei:
        ctx.device_status()
    assert ei.value.code == -4
    ctx.device_status()                                  # reported once
    ctx.ls_ablation_dev(rid, lid, g, best, 5, 3, 1024)
    torch.cuda.synchronize()                             # (the call ran on torch's stream)
    with pytest.raises(pkg.adgb.AdgbError) as ei:        # the next synchronous call reports it
        ctx.score_poses(rid, lid, genes, variant=3)
    assert ei.value.code == -4
    e1, g1 = ctx.score_poses(rid, lid, genes, variant=3)
    assert np.array_equal(e0, e1) and np.array_equal(g0, g1)
    ctx.close()


def test_block_mma_design_equals_warp_mma(pkg, torch, cfg1):
    """The other tensor-core design (one tcgen05 MMA a block over both warps'
    partials, measurement form 512 of ls_ablation_dev) computes every column
    of D as one MMA a warp does: the searched genotypes and energies are the
    same bits; it refuses launches whose last block is not full."""
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    genes = cfg1["genes"][:36]                 # 9 blocks of 4 genotypes
    out = []
    for mask in (0, 512):
        g = torch.from_numpy(genes.copy()).cuda()
        best = torch.empty(genes.shape[0], device="cuda")
        ctx.ls_ablation_dev(rid, lid, g, best, 25, 3, mask)
        torch.cuda.synchronize()
        out.append((g.cpu().numpy(), best.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    g = torch.from_numpy(cfg1["genes"][:37].copy()).cuda()
    best = torch.empty(37, device="cuda")
    with pytest.raises(pkg.adgb.AdgbError):
        ctx.ls_ablation_dev(rid, lid, g, best, 25, 3, 512)
    ctx.device_status()
    ctx.close()
