"""Error of every energy and gradient component against the FP64 oracle, for
each reduction variant, on the benchmark ligand (lga_n32) and the 256-atom
stress ligand; the table is printed (run with -s) and the stated tolerances
are asserted: energy max(1e-4 |E|, 1e-3 kcal/mol); each gene-gradient
component within 1e-3 (FP32 shuffle) or 2e-3 (split-precision MMA /
tcgen05) of its value where the value is above the floor 16 u A_j / tol
(u = 2^-24, A_j the component's magnitude from oracle.score_magnitude: the
chain rule over the absolute values of every contribution plus their
sensitivity to rounding the coordinates), else within 16 u A_j; and the
vector max-norm bound tol * max(|g|_inf, 1).  16 u: a few roundings per
contribution on its way through the kernels (the measured worst is about
4 u A_j on these workloads).  Printed per
gene group: the worst relative error of the components above the floor,
the share of components above it, and the worst error in units of u A_j.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-3, 1: 2e-3, 2: 2e-3, 3: 2e-3}
U32, C_U = 2.0 ** -24, 16.0
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
        m, pm = oracle.score_magnitude(R, L, w["genes"][p], with_positions=True)
        refs.append((e, g, near_face(w["receptor"], x), m + pm))
    G = 6 + w["ligand"]["n_tors"]
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    rows, rows_c, failures = [], [], []
    for v in (0, 1, 2, 3):
        e, g = ctx.score_poses(rid, lid, w["genes"], variant=v)
        e_rel, e_abs, gt, gr, gtor = [], [], [], [], []
        groups = {"translation": slice(0, 3), "rotation": slice(3, 6), "torsion": slice(6, G)}
        comp = {k: ([], [], []) for k in groups}   # rel. errors above the floor, well mask, err/(u A)
        for p, (er, gref, face, mag) in enumerate(refs):
            e_abs.append(abs(e[p] - er))
            e_rel.append(abs(e[p] - er) / max(abs(er), 1e-12))
            assert abs(e[p] - er) <= max(1e-4 * abs(er), 1e-3), (name, v, p, e[p], er)
            if face:
                continue
            scale = max(np.max(np.abs(gref)), 1.0)
            err = np.abs(g[p].astype(np.float64) - gref)
            d = err / scale
            gt.append(d[:3].max())
            gr.append(d[3:6].max())
            if G > 6:
                gtor.append(d[6:].max())
            assert d.max() <= TOL[v], (name, v, p, d.max())
            b_rel, b_abs = TOL[v] * np.abs(gref), C_U * U32 * mag
            bad = np.nonzero(err > np.maximum(b_rel, b_abs))[0]
            failures.extend((NAMES[v], p, int(j), float(err[j]), float(gref[j]),
                             float(err[j] / (U32 * mag[j]))) for j in bad)
            well = b_rel >= b_abs
            for k, sl in groups.items():
                comp[k][0].extend((err[sl] / np.maximum(np.abs(gref[sl]), 1e-300))[well[sl]])
                comp[k][1].extend(well[sl])
                comp[k][2].extend(err[sl] / np.maximum(U32 * mag[sl], 1e-300))
        rows.append((NAMES[v], np.median(e_rel), np.max(e_rel), np.max(e_abs), np.max(gt),
                     np.max(gr), np.max(gtor) if gtor else 0.0))
        crow = []
        for k in groups:
            rel, wl, ua = comp[k]
            crow.append("%s %.1e (%d%% above floor, max %.1f u A)"
                        % (k, max(rel) if rel else 0.0, 100 * np.mean(wl) if wl else 0,
                           max(ua) if ua else 0.0))
        rows_c.append((NAMES[v], "; ".join(crow)))
    print("\n%s (%d poses): variant | energy rel. median / max | energy abs. max | "
          "grad max/scale: translation, rotation, torsion" % (name, n))
    for r in rows:
        print("  %-11s %.2e / %.2e | %.2e kcal/mol | %.2e %.2e %.2e" % r)
    print("  per component, worst relative error above the floor 16 u A_j / tol:")
    for r in rows_c:
        print("  %-11s %s" % r)
    for f in failures[:20]:
        print("  FAIL variant %s pose %d gene %d: |dg| %.3e, g %.3e, %.1f u A" % f)
    assert not failures, failures[:5]
    # FP64 rescoring on the GPU
    gd = torch.from_numpy(w["genes"]).cuda()
    ed = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.rescore_fp64_dev(rid, lid, gd, ed)
    d64 = np.array([abs(ed[p].item() - refs[p][0]) / max(abs(refs[p][0]), 1.0) for p in range(n)])
    print("  fp64 rescoring: max rel. error %.2e" % d64.max())
    assert d64.max() <= 1e-9
    ctx.close()
