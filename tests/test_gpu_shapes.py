"""Ligand shapes across the kernels' internal boundaries, each against the
FP64 oracle: atom counts just below and above one warp (32), two warps (64),
four warps (128) and the maximum (256); torsion counts 0 and the maximum
(40); pair lists below and above one force-buffer chunk (1024 pairs); both
pair paths (matching rounds, warp or block form, and force buffer).  For
every shape: scores with each reduction variant, a short ADADELTA search
that must return its best, and the Solis-Wets start energy.
Tolerances: energy max(1e-4 |E|, 1e-3 kcal/mol); gene gradient 1e-3 (FP32
shuffle) or 2e-3 (split-precision variants) of max(|g|_inf, 1), on poses
whose atoms are at least 1e-4 A from grid-cell faces."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SHAPES = [(2, 0), (31, 6), (32, 8), (33, 8), (63, 12), (64, 16), (65, 16), (127, 30),
          (128, 32), (129, 32), (200, 0), (256, 40)]
TOL = {0: 1e-3, 1: 2e-3, 2: 2e-3, 3: 2e-3}


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
def rec():
    return synth.make_receptor(synth.generate.BASE_SEED + 77, 48, 8)


def near_face(r, x, tol=1e-4):
    u = (np.asarray(x, np.float64) - np.asarray(r["origin"], np.float64)) / r["spacing"]
    return bool(np.any(np.abs(u - np.round(u)) * r["spacing"] < tol))


@pytest.mark.parametrize("pair_rounds", [0, 1])
@pytest.mark.parametrize("n_atoms, n_tors", SHAPES)
def test_shape_parity(pkg, torch, rec, n_atoms, n_tors, pair_rounds):
    lig = synth.make_ligand(31_000 + n_atoms, n_atoms, 8, n_tors)
    genes = synth.make_poses(32_000 + n_atoms, 6, rec, n_tors)
    R, L = oracle.Receptor(rec), oracle.Ligand(lig)
    refs = [oracle.score(R, L, g) for g in genes]
    ctx = pkg.Context(0, pair_rounds=pair_rounds)
    rid = ctx.upload_receptor_grids(rec)
    lid = ctx.upload_ligand_torsion_tree(lig)
    for v in (0, 1, 2, 3):
        e, g = ctx.score_poses(rid, lid, genes, variant=v)
        for p, (er, gr, x, _) in enumerate(refs):
            assert abs(e[p] - er) <= max(1e-4 * abs(er), 1e-3), (n_atoms, v, p, e[p], er)
            if not near_face(rec, x):
                scale = max(np.max(np.abs(gr)), 1.0)
                assert np.max(np.abs(g[p] - gr)) <= TOL[v] * scale, (n_atoms, v, p)
    best, gb, _ = ctx.local_search(rid, lid, genes.copy(), 10)
    for p in range(len(genes)):
        e_ref = oracle.score(R, L, gb[p])[0]
        assert abs(best[p] - e_ref) <= max(1e-4 * abs(e_ref), 1e-3), (n_atoms, p, best[p], e_ref)
        assert best[p] <= refs[p][0] + max(1e-4 * abs(refs[p][0]), 1e-3)
    e1, g1, ev, _ = ctx.local_search_sw(rid, lid, genes, pkg.adgb.sw_params(max_evals=1))
    assert np.all(ev == 1) and np.array_equal(g1, genes)
    for p, (er, _, _, _) in enumerate(refs):
        assert abs(e1[p] - er) <= max(1e-4 * abs(er), 1e-3)
    ctx.close()
