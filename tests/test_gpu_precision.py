"""Error of every energy and gradient component against the FP64 oracle, for
each reduction variant, on the benchmark ligand (lga_n32) and the 256-atom
stress ligand; the table is printed (run with -s) and the stated tolerances
are asserted: energy max(1e-4 |E|, 1e-3 kcal/mol), gene gradient 1e-3 (FP32
shuffle) or 2e-3 (split-precision MMA / tcgen05) of max(|g|_inf, 1).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-3, 1: 2e-3, 2: 2e-3, 3: 2e-3}
NAMES = {0: "shfl", 1: "mma_tf32x2", 2: "mma_bf16x3", 3: "tcgen05"}


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


def near_face(rec, x, tol=1e-4):
    u = (np.asarray(x, np.float64) - np.asarray(rec["origin"], np.float64)) / rec["spacing"]
    return bool(np.any(np.abs(u - np.round(u)) * rec["spacing"] < tol))


@pytest.mark.parametrize("name, n", [("lga_n32", 96), ("stress_n256", 12)])
def test_component_errors(pkg, torch, name, n):
    w = synth.workload(name, n_poses=n)
    R, L = oracle.Receptor(w["receptor"]), oracle.Ligand(w["ligand"])
    refs = []
    for p in range(n):
        e, g, x, _ = oracle.score(R, L, w["genes"][p])
        refs.append((e, g, near_face(w["receptor"], x)))
    G = 6 + w["ligand"]["n_tors"]
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    rows = []
    for v in (0, 1, 2, 3):
        e, g = ctx.score_poses(rid, lid, w["genes"], variant=v)
        e_rel, e_abs, gt, gr, gtor = [], [], [], [], []
        for p, (er, gref, face) in enumerate(refs):
            e_abs.append(abs(e[p] - er))
            e_rel.append(abs(e[p] - er) / max(abs(er), 1e-12))
            assert abs(e[p] - er) <= max(1e-4 * abs(er), 1e-3), (name, v, p, e[p], er)
            if face:
                continue
            scale = max(np.max(np.abs(gref)), 1.0)
            d = np.abs(g[p].astype(np.float64) - gref) / scale
            gt.append(d[:3].max())
            gr.append(d[3:6].max())
            if G > 6:
                gtor.append(d[6:].max())
            assert d.max() <= TOL[v], (name, v, p, d.max())
        rows.append((NAMES[v], np.median(e_rel), np.max(e_rel), np.max(e_abs), np.max(gt),
                     np.max(gr), np.max(gtor) if gtor else 0.0))
    print("\n%s (%d poses): variant | energy rel. median / max | energy abs. max | "
          "grad max/scale: translation, rotation, torsion" % (name, n))
    for r in rows:
        print("  %-11s %.2e / %.2e | %.2e kcal/mol | %.2e %.2e %.2e" % r)
    # FP64 rescoring on the GPU
    gd = torch.from_numpy(w["genes"]).cuda()
    ed = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.rescore_fp64_dev(rid, lid, gd, ed)
    d64 = np.array([abs(ed[p].item() - refs[p][0]) / max(abs(refs[p][0]), 1.0) for p in range(n)])
    print("  fp64 rescoring: max rel. error %.2e" % d64.max())
    assert d64.max() <= 1e-9
    ctx.close()
