"""GPU parity of the Lamarckian GA path (dock) against the FP64 oracle.

The GA rules and the Philox4x32-10 stream are implemented independently in
the oracle and the CUDA library; with the same seed and the same inputs
their decisions (tournaments, cut points, mutations, local-search choices)
coincide exactly, and gene values agree to float32 rounding.  Whole docking
runs diverge chaotically (FP32 vs FP64 local searches), so they are checked
through invariants and the FP64 rescoring of their results.
"""
import numpy as np
import pytest

import oracle
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
def w():
    return synth.workload("plain_n16", n_poses=8)


def f32(x):
    return float(np.float32(x))


def oracle_params(gp):
    """the oracle's parameter block holding the float32 values the GPU uses"""
    return oracle.dock_params(n_runs=gp.n_runs, pop=gp.pop, max_gens=gp.max_gens,
                              max_evals=gp.max_evals, ls_iters=gp.ls_iters,
                              ls_rate=f32(gp.ls_rate), rho=f32(gp.rho), eps=f32(gp.eps),
                              p_cross=f32(gp.p_cross), p_mut=f32(gp.p_mut),
                              mut_trans=f32(gp.mut_trans), mut_angle=f32(gp.mut_angle),
                              seed=gp.seed, conv_every=gp.conv_every, conv_top=gp.conv_top,
                              conv_tol=f32(gp.conv_tol), ls_method=gp.ls_method,
                              sw_rho0=f32(gp.sw_rho0), sw_rho_min=f32(gp.sw_rho_min),
                              sw_max_succ=gp.sw_max_succ, sw_max_fail=gp.sw_max_fail,
                              sw_angle_scale=f32(gp.sw_angle_scale))


def ang(a, b):
    return (a - b + np.pi) % (2 * np.pi) - np.pi


def test_philox_device_known_answer_vectors(pkg, torch, philox_kat):
    """The device generator (philox.cuh) gives the published Philox4x32-10
    known-answer words (Salmon et al., SC'11; tests/golden) and the oracle's
    words on 4096 seeded random counters and keys, bit for bit."""
    kat = philox_kat
    rng = np.random.default_rng(2410)
    rand = rng.integers(0, 1 << 32, size=(4096, 6), dtype=np.uint64)
    inp = np.array([c + k for c, k, _ in kat] + rand.tolist(), np.uint64).astype(np.uint32)
    ctx = pkg.Context(0)
    dev_in = torch.from_numpy(inp.view(np.int32)).cuda()
    dev_out = torch.empty(inp.shape[0], 4, dtype=torch.int32, device="cuda")
    ctx.philox4x32_10_dev(dev_in, dev_out)
    got = dev_out.cpu().numpy().view(np.uint32)
    for i, (_, _, want) in enumerate(kat):
        assert got[i].tolist() == want
    for i in range(len(kat), inp.shape[0]):
        want = oracle.philox(inp[i, :4].tolist(), inp[i, 4:].tolist())
        assert got[i].tolist() == list(want), i
    ctx.philox4x32_10_dev(dev_in[:0], dev_out[:0])      # n = 0 is a no-op


def test_initial_population_matches_oracle(pkg, torch, w):
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    T = w["ligand"]["n_tors"]
    runs, pop = 3, 50
    g = torch.empty(runs * pop, 6 + T, device="cuda")
    ctx.ga_init_population_dev(rid, lid, 77, runs, pop, g)
    got = g.cpu().numpy().astype(np.float64)
    for r in range(runs):
        for k in range(pop):
            ref = oracle.init_individual(w["receptor"], T, 77, r, k)
            row = got[r * pop + k]
            assert np.max(np.abs(row[:3] - ref[:3])) < 2e-5
            assert np.max(np.abs(ang(row[3:], ref[3:]))) < 2e-6, (r, k, row, ref)
    ctx.close()


@pytest.mark.parametrize("p_cross, p_mut, ls_rate", [(0.8, 0.02, 1.0), (0.5, 0.3, 0.4), (1.0, 0.0, 0.0)])
def test_ga_generation_matches_oracle(pkg, torch, w, p_cross, p_mut, ls_rate):
    ctx = pkg.Context(0)
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    G = 6 + w["ligand"]["n_tors"]
    runs, pop = 4, 37
    rng = np.random.default_rng(3)
    genes = rng.normal(size=(runs * pop, G)).astype(np.float32)
    energy = (rng.normal(size=runs * pop) * 20).astype(np.float32)
    energy[5] = energy[9]          # a tie: lower index wins
    gp = pkg.adgb.dock_params(n_runs=runs, pop=pop, p_cross=p_cross, p_mut=p_mut,
                              ls_rate=ls_rate, ls_iters=17, seed=991)
    gi = torch.from_numpy(genes).cuda()
    ei = torch.from_numpy(energy).cuda()
    go = torch.empty_like(gi)
    it = torch.empty(runs * pop, dtype=torch.int32, device="cuda")
    for gen in (1, 2, 25):
        ctx.ga_generation_dev(lid, gp, gen, gi, ei, go, it)
        got = go.cpu().numpy().astype(np.float64)
        its = it.cpu().numpy()
        op = oracle_params(gp)
        for r in range(runs):
            ref, fl = oracle.ga_generation(genes[r * pop:(r + 1) * pop], energy[r * pop:(r + 1) * pop],
                                           op, r, gen)
            assert np.array_equal(its[r * pop:(r + 1) * pop], np.where(fl == 1, 17, 1))
            d = got[r * pop:(r + 1) * pop] - ref
            d[:, 6:] = ang(got[r * pop:(r + 1) * pop, 6:], ref[:, 6:])
            assert np.max(np.abs(d)) < 1e-5, (gen, r, np.max(np.abs(d)))
    ctx.close()


def test_fp64_rescoring_matches_oracle(pkg, torch):
    for name in ("plain_n16", "lga_n32", "stress_n256"):
        wk = synth.workload(name, n_poses=24)
        ctx = pkg.Context(0)
        rid = ctx.upload_receptor_grids(wk["receptor"])
        lid = ctx.upload_ligand_torsion_tree(wk["ligand"])
        g = torch.from_numpy(wk["genes"]).cuda()
        e = torch.empty(g.shape[0], dtype=torch.float64, device="cuda")
        ctx.rescore_fp64_dev(rid, lid, g, e)
        got = e.cpu().numpy()
        R, L = oracle.Receptor(wk["receptor"]), oracle.Ligand(wk["ligand"])
        for p in range(g.shape[0]):
            ref = oracle.score(R, L, wk["genes"][p])[0]
            assert abs(got[p] - ref) <= 1e-9 * max(abs(ref), 1.0), (name, p, got[p], ref)
        ctx.close()


@pytest.mark.parametrize("variant", [-1, 3])
def test_dock_results_and_accounting(pkg, torch, w, variant):
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    runs, pop, gens, it = 3, 24, 4, 30
    gp = pkg.adgb.dock_params(n_runs=runs, pop=pop, max_gens=gens, ls_iters=it, ls_rate=1.0, seed=5,
                              reduce_variant=variant)
    bg, be, ev = ctx.dock(rid, lid, gp)
    assert np.all(ev == pop + gens * pop * it)
    R, L = oracle.Receptor(w["receptor"]), oracle.Ligand(w["ligand"])
    T = w["ligand"]["n_tors"]
    for r in range(runs):
        ref = oracle.score(R, L, bg[r])[0]               # FP64 rescoring of the result
        assert abs(be[r] - ref) <= 1e-9 * max(abs(ref), 1.0)
        init = min(oracle.score(R, L, oracle.init_individual(w["receptor"], T, 5, r, k))[0]
                   for k in range(pop))
        assert be[r] <= init + 1e-3 * max(abs(init), 1.0)
    # deterministic for a fixed seed
    bg2, be2, ev2 = ctx.dock(rid, lid, gp)
    assert np.array_equal(bg, bg2) and np.array_equal(be, be2) and np.array_equal(ev, ev2)
    # the evaluation budget stops the runs after the generation that reaches it
    gp2 = pkg.adgb.dock_params(n_runs=2, pop=pop, max_gens=10, max_evals=100, ls_iters=it,
                               ls_rate=1.0, seed=5)
    _, _, ev3 = ctx.dock(rid, lid, gp2)
    assert np.all(ev3 == pop + pop * it)
    ctx.close()


def test_dock_matches_oracle_statistically(pkg, torch, w):
    """Best energies of GPU and oracle docking of the same runs (same seed,
    same initial populations) come from the same distribution (Sec. 5.1
    compares best-energy distributions the same way)."""
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    gp = pkg.adgb.dock_params(n_runs=8, pop=20, max_gens=3, ls_iters=40, ls_rate=1.0, seed=31)
    _, be, _ = ctx.dock(rid, lid, gp)
    _, be_ref, _ = oracle.dock(w["receptor"], w["ligand"], oracle_params(gp))
    med, med_ref = np.median(be), np.median(be_ref)
    assert abs(med - med_ref) <= 0.15 * abs(med_ref) + 1.0, (be, be_ref)
    ctx.close()


# ----------------------------------------------------------- early stopping
def _conv_cases(rng, pop, top, tol):
    """Energies of runs whose `top` lowest lie just inside, just outside and
    far from the tolerance, with ties, shuffles and non-finite values."""
    runs = []
    for scale in (0.5, 0.999, 1.001, 2.0, 0.0):
        e = rng.normal(-20.0, 2.0, pop)
        base = rng.normal(0.0, 1.0, top)
        base = (base - base.mean()) / base.std() if scale else np.zeros(top)
        e[:top] = -40.0 + base * tol * scale
        runs.append(rng.permutation(e))
    e = rng.normal(-20.0, 2.0, pop)
    e[:top + 3] = -30.0                      # ties across the cut
    runs.append(e)
    e = rng.normal(-20.0, 0.01, pop)
    e[5] = np.nan                            # a NaN among the lowest
    runs.append(e)
    e = rng.normal(-20.0, 0.01, pop)
    e[7] = np.inf                            # an unevaluated individual above the top
    runs.append(e)
    runs += [rng.normal(-20.0, s, pop) for s in (1e-3, 1e-2, 0.05, 0.1, 0.3)]
    return np.array(runs, np.float32)


@pytest.mark.parametrize("pop, top, tol", [(150, 15, 0.15), (64, 2, 0.05), (1024, 300, 1.0)])
def test_converged_flags_match_oracle(pkg, torch, pop, top, tol):
    ctx = pkg.Context(0)
    rng = np.random.default_rng(pop + top)
    e = _conv_cases(rng, pop, top, tol)
    runs = e.shape[0]
    gp = pkg.adgb.dock_params(n_runs=runs, pop=pop, conv_top=top, conv_tol=tol)
    flags = torch.empty(runs, dtype=torch.int32, device="cuda")
    ctx.ga_converged_dev(gp, torch.from_numpy(e.reshape(-1)).cuda(), flags)
    got = flags.cpu().numpy()
    ref = np.array([oracle.converged(e[r].astype(np.float64), top, f32(tol)) for r in range(runs)])
    assert np.array_equal(got, ref.astype(np.int32)), (got, ref)
    assert got[0] == 1 and got[3] == 0 and got[4] == 1 and got[6] == 0
    ctx.close()


def test_dock_early_stopping(pkg, torch, w):
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    runs, pop, gens, it = 4, 24, 12, 20
    base = dict(n_runs=runs, pop=pop, max_gens=gens, ls_iters=it, ls_rate=1.0, seed=9)
    full = pop + gens * pop * it
    # always converged: every run stops at the first test (generation 3)
    _, _, ev = ctx.dock(rid, lid, pkg.adgb.dock_params(conv_every=3, conv_top=6, conv_tol=1e6, **base))
    assert np.all(ev == pop + 3 * pop * it)
    # never converged: the full schedule, identical to early stopping off
    off = ctx.dock(rid, lid, pkg.adgb.dock_params(**base))
    never = ctx.dock(rid, lid, pkg.adgb.dock_params(conv_every=3, conv_top=6, conv_tol=1e-12, **base))
    assert np.all(never[2] == full)
    for a, b in zip(off, never):
        assert np.array_equal(a, b)
    # a tolerance in between: runs stop at test generations, deterministically,
    # and keep the best they found before stopping
    gp = pkg.adgb.dock_params(conv_every=2, conv_top=6, conv_tol=0.5, **base)
    bg, be, ev = ctx.dock(rid, lid, gp)
    stop_gen = (ev - pop) // (pop * it)
    assert np.all((ev - pop) % (pop * it) == 0)
    assert np.all((stop_gen % 2 == 0) | (stop_gen == gens)) and np.all(stop_gen >= 2)
    bg2, be2, ev2 = ctx.dock(rid, lid, gp)
    assert np.array_equal(bg, bg2) and np.array_equal(be, be2) and np.array_equal(ev, ev2)
    R, L = oracle.Receptor(w["receptor"]), oracle.Ligand(w["ligand"])
    for r in range(runs):
        assert abs(be[r] - oracle.score(R, L, bg[r])[0]) <= 1e-9 * max(abs(be[r]), 1.0)
    # bad parameters are refused
    with pytest.raises(pkg.AdgbError):
        ctx.dock(rid, lid, pkg.adgb.dock_params(conv_every=2, conv_top=1, **base))
    with pytest.raises(pkg.AdgbError):
        ctx.dock(rid, lid, pkg.adgb.dock_params(conv_every=2, conv_top=6, conv_tol=0.0, **base))
    ctx.close()


# ------------------------------------------------- Solis-Wets inside the LGA
def test_dock_with_solis_wets(pkg, torch, w):
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    runs, pop, gens, it = 4, 20, 4, 40
    gp = pkg.adgb.dock_params(n_runs=runs, pop=pop, max_gens=gens, ls_iters=it, ls_rate=1.0, seed=13,
                              ls_method=1, sw_angle_scale=0.5, sw_rho_min=0.3)
    bg, be, ev = ctx.dock(rid, lid, gp)
    # evaluations actually spent: a search stops before its budget once rho < rho_min
    assert np.all(ev >= pop + gens * pop) and np.all(ev <= pop + gens * pop * it)
    assert np.any(ev < pop + gens * pop * it)
    bg2, be2, ev2 = ctx.dock(rid, lid, gp)
    assert np.array_equal(bg, bg2) and np.array_equal(be, be2) and np.array_equal(ev, ev2)
    R, L = oracle.Receptor(w["receptor"]), oracle.Ligand(w["ligand"])
    T = w["ligand"]["n_tors"]
    for r in range(runs):
        assert abs(be[r] - oracle.score(R, L, bg[r])[0]) <= 1e-9 * max(abs(be[r]), 1.0)
        init = min(oracle.score(R, L, oracle.init_individual(w["receptor"], T, 13, r, k))[0]
                   for k in range(pop))
        assert be[r] <= init + 1e-3 * max(abs(init), 1.0)
    # the oracle's LGA with the same Solis-Wets searches: same distribution of results
    gp8 = pkg.adgb.dock_params(n_runs=8, pop=16, max_gens=3, ls_iters=40, ls_rate=1.0, seed=21,
                               ls_method=1, sw_angle_scale=0.5, sw_rho_min=0.3)
    _, be_g, ev_g = ctx.dock(rid, lid, gp8)
    _, be_o, ev_o = oracle.dock(w["receptor"], w["ligand"], oracle_params(gp8))
    assert abs(np.median(be_g) - np.median(be_o)) <= 0.15 * abs(np.median(be_o)) + 1.0, (be_g, be_o)
    assert abs(np.mean(ev_g) - np.mean(ev_o)) <= 0.25 * np.mean(ev_o)
    # the serving loop runs Solis-Wets jobs as dock() does
    srv = pkg.Server(ctx)
    j = srv.submit(rid, w["ligand"], gp)
    assert srv.wait(j, 60000)["status"] == 0
    gs, es, vs = srv.result(j)
    assert np.array_equal(es, be) and np.array_equal(vs, ev) and np.array_equal(gs, bg)
    srv.stop()
    ctx.close()


def test_dock_edge_sizes(pkg, torch, w):
    """Largest population (1024), no generations, one-individual-budget runs."""
    ctx = pkg.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    R, L = oracle.Receptor(w["receptor"]), oracle.Ligand(w["ligand"])
    T = w["ligand"]["n_tors"]
    # pop 1024, one generation of 2-evaluation searches
    bg, be, ev = ctx.dock(rid, lid, pkg.adgb.dock_params(n_runs=2, pop=1024, max_gens=1, ls_iters=2,
                                                         ls_rate=1.0, seed=3))
    assert np.all(ev == 1024 + 1024 * 2)
    for r in range(2):
        assert abs(be[r] - oracle.score(R, L, bg[r])[0]) <= 1e-9 * max(abs(be[r]), 1.0)
    # no generation: the best of the initial population, each scored once
    bg, be, ev = ctx.dock(rid, lid, pkg.adgb.dock_params(n_runs=3, pop=8, max_gens=0, seed=4))
    assert np.all(ev == 8)
    for r in range(3):
        init = [oracle.score(R, L, oracle.init_individual(w["receptor"], T, 4, r, k))[0]
                for k in range(8)]
        assert abs(be[r] - min(init)) <= max(1e-4 * abs(min(init)), 1e-3)
    # bad population sizes are refused
    for pop in (1, 1025):
        with pytest.raises(pkg.AdgbError):
            ctx.dock(rid, lid, pkg.adgb.dock_params(n_runs=1, pop=pop, max_gens=1, seed=1))
    ctx.close()
