"""GPU Solis-Wets local search (energy only) through the C ABI against the
FP64 oracle.

A whole search is a chain of accept/reject decisions on FP32 energies, so
like the ADADELTA search it is compared step by step from the GPU's own
state (teacher forcing), where decisions whose two energies lie within the
FP32 energy tolerance of each other are ambiguous and skipped, and by
invariants and statistics for whole searches.  Tolerances: energies
|dE| <= max(1e-4 |E|, 1e-3 kcal/mol); genes after a step 1e-5 (the deviates
come from the same Philox words; FP32 vs FP64 Box-Muller and additions).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

E_REL, E_ABS = 1e-4, 1e-3


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
    return synth.workload("lga_n32", n_poses=48)


def etol(e):
    return max(E_REL * abs(e), E_ABS)


def wrap(v):
    v = np.array(v, np.float64)
    v[6:] = (v[6:] + np.pi) % (2 * np.pi) - np.pi
    return v


def ang_diff(a, b):
    return (a - b + np.pi) % (2 * np.pi) - np.pi


def test_sw_start_energy_matches_oracle(pkg, torch, cfg1):
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    p = pkg.adgb.sw_params(max_evals=1)
    e, g, ev, _ = ctx.local_search_sw(rid, lid, cfg1["genes"], p)
    assert np.all(ev == 1) and np.array_equal(g, cfg1["genes"])
    R, L = oracle.Receptor(cfg1["receptor"]), oracle.Ligand(cfg1["ligand"])
    for k in range(len(e)):
        ref = oracle.score(R, L, cfg1["genes"][k])[0]
        assert abs(e[k] - ref) <= etol(ref), (k, e[k], ref)
    ctx.close()


@pytest.mark.parametrize("variant", [0, 3])
def test_sw_teacher_forced_steps(pkg, torch, cfg1, variant):
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    R, L = oracle.Receptor(cfg1["receptor"]), oracle.Ligand(cfg1["ligand"])
    G = 6 + cfg1["ligand"]["n_tors"]
    kw = dict(seed=77, max_succ=2, max_fail=2, angle_scale=0.5, reduce_variant=variant)
    n = cfg1["genes"].shape[0]
    checked = 0
    for t in (1, 9, 40):
        _, _, _, st = ctx.local_search_sw(rid, lid, cfg1["genes"], pkg.adgb.sw_params(max_evals=t, **kw),
                                          want_state=True)
        for evals in (1, 2):
            p1 = pkg.adgb.sw_params(max_evals=evals, flags=pkg.LS_RESUME, **kw)
            e1, g1, ev1, s1 = ctx.local_search_sw(rid, lid, st[:, :G], p1, state=st)
            po = oracle.sw_params(max_evals=evals, seed=77, max_succ=2, max_fail=2, angle_scale=0.5)
            for k in range(n):
                s = st[k].astype(np.float64)
                x, b, rho, ex, step = s[:G], s[G:2 * G], s[2 * G], s[2 * G + 3], int(s[2 * G + 4])
                if rho < 0.01:
                    continue
                z = np.array([oracle.sw_normal(77, k, step, 0, j) for j in range(G)])
                d = b + rho * np.where(np.arange(G) < 3, 1.0, 0.5) * z
                ep = oracle.score(R, L, wrap(x + d))[0]
                em = oracle.score(R, L, wrap(x - d))[0]
                if abs(ep - ex) <= 2 * etol(ex) or (evals == 2 and abs(em - ex) <= 2 * etol(ex)):
                    continue                               # the decision is within FP32 noise
                if evals == 2 and ep < ex:
                    continue                               # a success leaves one evaluation for the next step
                e_r, g_r, ev_r, s_r = oracle.sw_search(R, L, x, po, genotype=k, state=s)
                assert ev1[k] == ev_r
                assert abs(e1[k] - e_r) <= etol(e_r), (t, evals, k, e1[k], e_r)
                dx = g1[k].astype(np.float64) - g_r
                dx[6:] = ang_diff(g1[k, 6:].astype(np.float64), g_r[6:])
                assert np.max(np.abs(dx)) <= 1e-5, (t, evals, k, dx)
                assert np.allclose(s1[k, G:2 * G], s_r[G:2 * G], atol=1e-5)
                assert np.array_equal(s1[k, 2 * G:2 * G + 3].astype(np.float64), s_r[2 * G:2 * G + 3])
                assert s1[k, 2 * G + 4] == s_r[2 * G + 4]
                checked += 1
    assert checked >= n
    ctx.close()


def test_sw_whole_searches(pkg, torch, cfg1):
    """Invariants of whole searches, determinism, and the best-energy
    distribution against the oracle's own searches (Sec. 5.1 compares
    distributions the same way)."""
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    R, L = oracle.Receptor(cfg1["receptor"]), oracle.Ligand(cfg1["ligand"])
    G = 6 + cfg1["ligand"]["n_tors"]
    p = pkg.adgb.sw_params(max_evals=300, seed=5)
    g0 = cfg1["genes"]
    e, g, ev, st = ctx.local_search_sw(rid, lid, g0, p, want_state=True)
    e_b, g_b, ev_b, _ = ctx.local_search_sw(rid, lid, g0, p)
    assert np.array_equal(e, e_b) and np.array_equal(g, g_b) and np.array_equal(ev, ev_b)
    assert np.all(ev <= 300) and np.all(ev >= 1)
    assert np.all((ev == 300) | (st[:, 2 * G] < 0.01))
    refs = []
    for k in range(len(e)):
        start = oracle.score(R, L, g0[k])[0]
        assert e[k] <= start + etol(start)
        at = oracle.score(R, L, g[k])[0]
        assert abs(e[k] - at) <= etol(at), (k, e[k], at)
        refs.append(oracle.sw_search(R, L, g0[k], oracle.sw_params(max_evals=300, seed=5),
                                     genotype=k)[0])
    q_gpu, q_ref = np.quantile(e, [0.1, 0.5]), np.quantile(refs, [0.1, 0.5])
    assert np.all(np.abs(q_gpu - q_ref) <= 0.15 * np.abs(q_ref) + 1.0), (q_gpu, q_ref)
    # device call on torch buffers gives the host call's results
    gd = torch.from_numpy(g0.copy()).cuda()
    ed = torch.empty(len(e), device="cuda")
    evd = torch.empty(len(e), dtype=torch.int32, device="cuda")
    ctx.local_search_sw_dev(rid, lid, gd, ed, p, evals=evd)
    assert np.array_equal(ed.cpu().numpy(), e) and np.array_equal(gd.cpu().numpy(), g)
    # zero genotypes; bad parameters
    e0, _, _, _ = ctx.local_search_sw(rid, lid, np.zeros((0, G), np.float32), p)
    assert e0.shape == (0,)
    for bad in (dict(max_evals=0), dict(rho0=0.0), dict(max_succ=0), dict(angle_scale=-1.0),
                dict(call=70000)):
        with pytest.raises(pkg.AdgbError):
            ctx.local_search_sw(rid, lid, g0[:2], pkg.adgb.sw_params(**bad))
    ctx.close()
