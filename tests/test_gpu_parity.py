"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs.

Tolerances (written out per check):
  coordinates          max |dx| <= 1e-5 A
  energy (FP32 path)   |dE| <= max(1e-4 |E|, 1e-3 kcal/mol)
  gene gradient        per component: |dg_j| <= 1e-3 |g_j| where |g_j| is above
                       the floor F_j = 16 u A_j / 1e-3, else |dg_j| <= 16 u A_j
                       (u = 2^-24; A_j = oracle.score_magnitude with positions:
                       the chain rule over the absolute values of all
                       contributions, plus their sensitivity to rounding the
                       coordinates, so that 16 u A_j bounds the rounding error
                       of an FP32 evaluation and |g_j| < F_j means cancellation
                       has left fewer than three correct digits to test); and
                       the vector max-norm max_j |dg_j| <= 1e-3 * max(max_j |g_j|, 1)
  split-precision MMA reductions: the same gradient bounds at 2e-3.
Trilinear interpolation is only C0: gradients are compared on poses whose
atoms all lie at least 1e-4 A from every grid-cell face.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

E_REL, E_ABS, G_REL, G_REL_MMA, X_ABS = 1e-4, 1e-3, 1e-3, 2e-3, 1e-5
VARIANT_TOL = {0: G_REL, 1: G_REL_MMA, 2: G_REL_MMA, 3: G_REL_MMA}
U32, C_U = 2.0 ** -24, 16.0


def component_check(g_gpu, g_ref, mag, tol):
    """Per-component gradient bound; returns (relative errors of the components
    above the floor, mask of those components)."""
    err = np.abs(np.asarray(g_gpu, np.float64) - g_ref)
    b_rel, b_abs = tol * np.abs(g_ref), C_U * U32 * mag
    bad = err > np.maximum(b_rel, b_abs)
    assert not bad.any(), (np.nonzero(bad), err[bad], g_ref[bad], mag[bad])
    well = b_rel >= b_abs
    return np.where(well, err / np.maximum(np.abs(g_ref), 1e-300), 0.0), well


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


def make_ctx(pkg, **kw):
    return pkg.Context(0, **kw)


@pytest.fixture(scope="module")
def cfg0():
    return synth.workload("plain_n16", n_poses=64)


@pytest.fixture(scope="module")
def cfg1():
    return synth.workload("lga_n32", n_poses=96)


def near_face(rec, x, tol=1e-4):
    u = (np.asarray(x, np.float64) - np.asarray(rec["origin"], np.float64)) / rec["spacing"]
    return bool(np.any(np.abs(u - np.round(u)) * rec["spacing"] < tol))


def ang_diff(a, b):
    return (a - b + np.pi) % (2 * np.pi) - np.pi


def oracle_scores(w, genes):
    R, L = oracle.Receptor(w["receptor"]), oracle.Ligand(w["ligand"])
    out = [oracle.score(R, L, g) for g in np.asarray(genes, np.float64)]
    return out


def check_scores(w, genes, e_gpu, g_gpu, g_tol):
    refs = oracle_scores(w, genes)
    R, L = oracle.Receptor(w["receptor"]), oracle.Ligand(w["ligand"])
    worst_e = worst_g = 0.0
    compared = n_comp = n_well = 0
    for p, (e, g, x, _) in enumerate(refs):
        assert abs(e_gpu[p] - e) <= max(E_REL * abs(e), E_ABS), (p, float(e_gpu[p]), e)
        worst_e = max(worst_e, abs(e_gpu[p] - e) / max(abs(e), 1e-12))
        if g_gpu is None or near_face(w["receptor"], x):
            continue
        err = np.max(np.abs(g_gpu[p] - g)) / max(np.max(np.abs(g)), 1.0)
        assert err <= g_tol, (p, err, g_gpu[p], g)
        m, pm = oracle.score_magnitude(R, L, genes[p], with_positions=True)
        rel, well = component_check(g_gpu[p], g, m + pm, g_tol)
        worst_g = max(worst_g, float(rel.max()))
        n_comp += well.size
        n_well += int(well.sum())
        compared += 1
    assert compared >= len(refs) // 2
    assert g_gpu is None or n_well >= n_comp // 10   # a share of components is tested relatively
    return worst_e, worst_g


# ------------------------------------------------------------- coordinates
@pytest.mark.parametrize("name", ["plain_n16", "lga_n32", "stress_n256"])
def test_pose_coords_parity(pkg, torch, name):
    w = synth.workload(name, n_poses=24)
    ctx = make_ctx(pkg)
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    N = w["ligand"]["n_atoms"]
    genes = torch.from_numpy(w["genes"]).cuda()
    xyz = torch.empty(genes.shape[0], N, 3, device="cuda")
    ctx.pose_coords_dev(lid, genes, xyz)
    got = xyz.cpu().numpy()
    L = oracle.Ligand(w["ligand"])
    for p in range(genes.shape[0]):
        ref = oracle.pose_coords(L, w["genes"][p])
        assert np.max(np.abs(got[p] - ref)) <= X_ABS, (p, np.max(np.abs(got[p] - ref)))
    # host-pointer entry point gives the same numbers
    host = ctx.pose_coords(lid, w["genes"], N)
    assert np.array_equal(host, got)
    ctx.close()


def test_zero_pose_is_exact_on_gpu(pkg, torch, cfg1):
    ctx = make_ctx(pkg)
    lig = cfg1["ligand"]
    lid = ctx.upload_ligand_torsion_tree(lig)
    G = 6 + lig["n_tors"]
    g = np.zeros((3, G), np.float32)
    g[1, :3] = (1.25, -3.5, 0.75)
    g[2, 3:5] = (0.7, 1.9)  # axis only, zero angle
    x = ctx.pose_coords(lid, g, lig["n_atoms"])
    ref = lig["xyz"].astype(np.float32)
    assert np.array_equal(x[0], ref)
    assert np.array_equal(x[1], (ref.astype(np.float64) + g[1, :3].astype(np.float64)).astype(np.float32))
    assert np.array_equal(x[2], ref)
    ctx.close()


# ----------------------------------------------------------------- scoring
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("tpp", [32, 64, 128])
def test_score_parity_cfg0(pkg, torch, cfg0, variant, tpp):
    ctx = make_ctx(pkg, threads_per_pose=tpp)
    rid = ctx.upload_receptor_grids(cfg0["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg0["ligand"])
    genes = torch.from_numpy(cfg0["genes"]).cuda()
    n, G = genes.shape
    e = torch.empty(n, device="cuda")
    g = torch.empty(n, G, device="cuda")
    ctx.score_poses_dev(rid, lid, genes, e, g, variant=variant)
    check_scores(cfg0, cfg0["genes"], e.cpu().numpy(), g.cpu().numpy(), VARIANT_TOL[variant])
    ctx.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_score_parity_cfg1(pkg, torch, cfg1, variant):
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    e, g = ctx.score_poses(rid, lid, cfg1["genes"], variant=variant)
    check_scores(cfg1, cfg1["genes"], e, g, VARIANT_TOL[variant])
    ctx.close()


def test_score_parity_stress_n256_sampled(pkg, torch):
    # the 256-atom / 40-torsion / ~30k-pair ligand on the 128^3 x 16-map
    # grid; 256 poses scored on the GPU, 12 of them checked against the oracle
    w = synth.workload("stress_n256", n_poses=256)
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    e, g = ctx.score_poses(rid, lid, w["genes"])
    idx = np.linspace(0, 255, 12).astype(int)
    check_scores(w, w["genes"][idx], e[idx], g[idx], G_REL)
    ctx.close()


def test_score_edge_cases(pkg, torch, cfg0):
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(cfg0["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg0["ligand"])
    # empty batch
    e, g = ctx.score_poses(rid, lid, np.zeros((0, 10), np.float32))
    assert e.shape == (0,)
    # poses far outside the grid: the clamp + quadratic wall
    G = 6 + cfg0["ligand"]["n_tors"]
    out = cfg0["genes"][:8].copy()
    out[:, 0] += 40.0
    out[:4, 1] -= 25.0
    e, g = ctx.score_poses(rid, lid, out)
    check_scores(cfg0, out, e, g, G_REL)
    # a one-atom ligand with no torsion and no pair
    one = dict(cfg0["ligand"])
    one.update(n_atoms=1, n_tors=0, type=one["type"][:1], charge=one["charge"][:1],
               xyz=np.zeros((1, 3), np.float32), tors_bond=np.zeros((0, 2), np.int32),
               mov_off=np.zeros(1, np.int32), mov_atoms=np.zeros(0, np.int32),
               pairs=np.zeros((0, 2), np.int32))
    lid1 = ctx.upload_ligand_torsion_tree(one)
    w1 = dict(cfg0, ligand=one)
    gs = cfg0["genes"][:16, :6].copy()
    e, g = ctx.score_poses(rid, lid1, gs)
    check_scores(w1, gs, e, g, G_REL)
    # a ligand type without a receptor map is refused
    bad = dict(cfg0["ligand"])
    bad["type"] = bad["type"].copy()
    bad["type"][0] = cfg0["receptor"]["n_type_maps"]
    bad["n_types"] = int(cfg0["receptor"]["n_type_maps"]) + 1
    for k in ("R", "eps", "vol", "solpar"):
        bad[k] = np.concatenate([bad[k], bad[k][:1]])
    bad["hb_role"] = np.concatenate([bad["hb_role"], [0]]).astype(np.int32)
    lidb = ctx.upload_ligand_torsion_tree(bad)
    with pytest.raises(pkg.AdgbError):
        ctx.score_poses(rid, lidb, cfg0["genes"][:2])
    ctx.close()


def test_host_and_device_calls_agree(pkg, torch, cfg1):
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    e_h, g_h = ctx.score_poses(rid, lid, cfg1["genes"])
    genes = torch.from_numpy(cfg1["genes"]).cuda()
    e_d = torch.empty(genes.shape[0], device="cuda")
    g_d = torch.empty_like(genes)
    ctx.score_poses_dev(rid, lid, genes, e_d, g_d)
    assert np.array_equal(e_h, e_d.cpu().numpy())
    assert np.array_equal(g_h, g_d.cpu().numpy())
    ctx.close()


# ------------------------------------------------------------ local search
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_local_search_teacher_forced_step(pkg, torch, cfg1, variant):
    """One ADADELTA step from the GPU's own state at step t equals the
    oracle's step from that same state (the trajectory itself is chaotic).

    Bounds follow from the gradient bound tol_g = G_REL * max(|g|_inf, 1):
    the step d(g) = -A g / sqrt(B + (1-rho) g^2), A = sqrt(E[d^2] + eps),
    B = rho E[g^2] + eps, has |d'(g)| <= A / sqrt(B), so
    |d_gpu - d_ref| <= A / sqrt(B) * tol_g; E[g^2] and E[d^2] follow from
    their update formulas the same way."""
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(cfg1["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg1["ligand"])
    R, L = oracle.Receptor(cfg1["receptor"]), oracle.Ligand(cfg1["ligand"])
    g0 = cfg1["genes"][:24]
    n, G = g0.shape
    rho, eps = 0.8, 1e-2
    tol = VARIANT_TOL[variant]
    for t in (0, 1, 6, 40):
        if t == 0:
            st = np.zeros((n, 3, G), np.float32)
            st[:, 0] = g0
        else:
            _, _, st = ctx.local_search(rid, lid, g0.copy(), t, variant=variant, want_state=True)
        best1, gb1, st1 = ctx.local_search(rid, lid, g0.copy(), 1, variant=variant, state=st,
                                           resume=True, want_state=True)
        checked = 0
        for p in range(n):
            e_ref, g_ref, x_ref, _ = oracle.score(R, L, st[p, 0])
            if near_face(cfg1["receptor"], x_ref):
                continue
            b_ref, gb_ref, st_ref = oracle.local_search(R, L, st[p, 0], 1, state=st[p])
            assert abs(best1[p] - b_ref) <= max(E_REL * abs(b_ref), E_ABS)
            tol_g = tol * max(np.max(np.abs(g_ref)), 1.0)
            eg2, ed2 = st[p, 1].astype(np.float64), st[p, 2].astype(np.float64)
            A, B = np.sqrt(ed2 + eps), rho * eg2 + eps
            d_ref = st_ref[0] - st[p, 0].astype(np.float64)
            d_ref[6:] = ang_diff(st_ref[0, 6:], st[p, 0, 6:].astype(np.float64))
            dd = st1[p, 0].astype(np.float64) - st_ref[0]
            dd[6:] = ang_diff(st1[p, 0, 6:].astype(np.float64), st_ref[0, 6:])
            bound_d = A / np.sqrt(B) * tol_g * 1.5 + 1e-6
            assert np.all(np.abs(dd) <= bound_d), (t, p, dd, bound_d)
            bound_eg = (1 - rho) * (2 * np.abs(g_ref) * tol_g + tol_g ** 2) * 1.5 + 1e-5 * np.abs(st_ref[1]) + 1e-12
            assert np.all(np.abs(st1[p, 1] - st_ref[1]) <= bound_eg), (t, p)
            bound_ed = (1 - rho) * (2 * np.abs(d_ref) * bound_d + bound_d ** 2) + 1e-5 * np.abs(st_ref[2]) + 1e-12
            assert np.all(np.abs(st1[p, 2] - st_ref[2]) <= bound_ed), (t, p)
            checked += 1
        assert checked >= n // 2
    ctx.close()


def test_local_search_returns_its_best(pkg, torch, cfg0):
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(cfg0["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg0["ligand"])
    e0, _ = ctx.score_poses(rid, lid, cfg0["genes"], with_grad=False)
    best, gb, st = ctx.local_search(rid, lid, cfg0["genes"].copy(), 300, want_state=True)
    assert np.all(best <= e0 * (1 + 1e-6) + 1e-3)
    # the returned genotype has the returned energy (oracle, FP64)
    refs = oracle_scores(cfg0, gb)
    for p, (e, _, _, _) in enumerate(refs):
        assert abs(best[p] - e) <= max(E_REL * abs(e), E_ABS), (p, best[p], e)
    # zero iterations: +inf, genes untouched
    b0, g00, _ = ctx.local_search(rid, lid, cfg0["genes"].copy(), 0)
    assert np.all(np.isinf(b0)) and np.array_equal(g00, cfg0["genes"])
    ctx.close()


def test_local_search_matches_oracle_statistically(pkg, torch, cfg0):
    """Whole 300-step searches diverge chaotically between FP32 and FP64;
    like Sec. 5.1 compare the distribution of best energies instead."""
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(cfg0["receptor"])
    lid = ctx.upload_ligand_torsion_tree(cfg0["ligand"])
    best, _, _ = ctx.local_search(rid, lid, cfg0["genes"].copy(), 300)
    ref, _ = oracle.local_search_batch(cfg0["receptor"], cfg0["ligand"], cfg0["genes"], 300)
    q_gpu = np.quantile(best, [0.1, 0.5])
    q_ref = np.quantile(ref, [0.1, 0.5])
    assert np.all(np.abs(q_gpu - q_ref) <= 0.1 * np.abs(q_ref) + 1.0), (q_gpu, q_ref)
    ctx.close()


def test_lga_n32_full_batch_sampled(pkg, torch):
    """Full-size batch of the benchmark (3000 genotypes x 300 steps, the
    launch configuration bench.py times); sampled genotypes checked."""
    w = synth.workload("lga_n32")
    ctx = make_ctx(pkg)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    genes = torch.from_numpy(w["genes"]).cuda()
    best = torch.empty(genes.shape[0], device="cuda")
    ctx.local_search_dev(rid, lid, genes, best, 300)
    b = best.cpu().numpy()
    gb = genes.cpu().numpy()
    assert np.all(np.isfinite(b))
    idx = np.linspace(0, genes.shape[0] - 1, 16).astype(int)
    refs = oracle_scores(w, gb[idx])
    for k, p in enumerate(idx):
        e = refs[k][0]
        assert abs(b[p] - e) <= max(E_REL * abs(e), E_ABS), (p, b[p], e)
    ctx.close()


# --------------------------------------------------------------- reduction
def _reduce_inputs(seed, nb, threads):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(nb, threads, 4)) * 10.0 ** rng.integers(-3, 4, (nb, threads, 4))
    x[0, :, 1] = 1.0                          # exact small integers
    x[1, ::2, 2] = 1e6                        # cancelling outliers
    x[1, 1::2, 2] = -1e6
    return x.astype(np.float32)


@pytest.mark.parametrize("variant", [100, 0, 1, 2, 102])
@pytest.mark.parametrize("threads", [64, 192, 256, 384, 1024])
def test_reduce4_bench_parity(pkg, torch, variant, threads):
    ctx = make_ctx(pkg)
    nb = 19
    x = _reduce_inputs(threads + variant, nb, threads)
    xt = torch.from_numpy(x).cuda()
    out = ctx.reduce4_bench_dev(variant, xt, threads, reps=3).cpu().numpy()
    ref = np.array([[oracle.sum_neumaier(x[b, :, c]) for c in range(4)] for b in range(nb)])
    scale = np.abs(x.astype(np.float64)).sum(axis=1)
    tol = 2e-6 if variant in (100, 0, 2) else 4e-6
    for b in range(nb):
        assert np.all(out[b] == out[b, 0]), "every thread gets the same sum"
        assert np.all(np.abs(out[b, 0] - ref[b]) <= tol * scale[b]), (b, out[b, 0], ref[b])
    assert np.all(out[0, 0, 1] == threads)
    ctx.close()


@pytest.mark.parametrize("threads", [32, 64, 96, 256, 1024])
def test_reduce4_paper_half_within_fp16_bound(pkg, torch, threads):
    """Sec. 4.2 in FP16: inputs rounded to FP16 (2^-11 relative each), V
    accumulated over ceil(T/64) chunk products and W = Q.V rounded once more;
    every rounding is bounded by 2^-11 of the sum of magnitudes it covers,
    and up to 16 roundings are allowed inside each product."""
    ctx = make_ctx(pkg)
    rng = np.random.default_rng(threads)
    nb = 19
    x = rng.normal(size=(nb, threads, 4)).astype(np.float32)
    x[0, :, 1] = 1.0                              # exact in FP16 up to 2048
    xt = torch.from_numpy(x).cuda()
    out = ctx.reduce4_bench_dev(pkg.REDUCE4_PAPER_HALF, xt, threads, reps=2).cpu().numpy()
    ref = x.astype(np.float64).sum(axis=1)
    scale = np.abs(x.astype(np.float64)).sum(axis=1)
    n_round = 2 + (threads + 63) // 64 + 16
    for b in range(nb):
        assert np.all(out[b] == out[b, 0])
        assert np.all(np.abs(out[b, 0] - ref[b]) <= n_round * 2.0 ** -11 * scale[b]), b
    assert np.all(out[0, :, 1] == threads)
    ctx.close()


def test_reduce4_paper_half_overflows_above_fp16_range(pkg, torch):
    """A total beyond 65504 is not representable in the paper's FP16 V / W."""
    ctx = make_ctx(pkg)
    x = np.full((2, 1024, 4), 100.0, np.float32)      # totals 102400
    x[1] = 1.0                                         # totals 1024: exact
    out = ctx.reduce4_bench_dev(pkg.REDUCE4_PAPER_HALF, torch.from_numpy(x).cuda(), 1024,
                                reps=1).cpu().numpy()
    assert np.all(np.isinf(out[0]))
    assert np.all(out[1] == 1024.0)
    ctx.close()


def test_reduce4_tcgen05_rejects_odd_warp_counts(pkg, torch):
    ctx = make_ctx(pkg)
    x = torch.zeros(96 * 4, device="cuda")
    with pytest.raises(pkg.AdgbError):
        ctx.reduce4_bench_dev(pkg.REDUCE4_TCGEN05_TF32X2, x, 96, reps=1)
    ctx.close()


def test_alu_probe(pkg, torch):
    """The ALU throughput probe runs its chains to finite values and refuses
    bad shapes (it measures the roofline's denominator)."""
    ctx = make_ctx(pkg)
    out = torch.empty(4 * 64, device="cuda")
    for kind in (0, 1, 2, 3):
        ctx.alu_bench_dev(kind, 4, 64, 3, out)
        assert torch.isfinite(out).all()
    for bad in ((4, 4, 64, 3), (0, 4, 48, 3), (0, 0, 64, 3), (0, 4, 512, 3)):
        with pytest.raises(pkg.AdgbError):
            ctx.alu_bench_dev(*bad, out)
    ctx.close()


def test_l2_probe(pkg, torch):
    """The L2 read probe reads what it says: over a buffer of ones every
    thread's sum is the number of float4 it read (reps streaming, 6 a
    repetition gathering; the buffer holds 50 cells of 20 float4 and a ragged
    tail), and it refuses bad shapes and cell sizes."""
    ctx = make_ctx(pkg)
    buf = torch.ones(4 * (50 * 20 + 7), device="cuda")
    out = torch.empty(3 * 64, device="cuda")
    ctx.l2_bench_dev(0, buf, 3, 64, 5, out)
    assert torch.equal(out, torch.full_like(out, 5.0))
    ctx.l2_bench_dev(1, buf, 3, 64, 5, out, cell_float4=20)
    assert torch.equal(out, torch.full_like(out, 30.0))
    for bad in ((2, buf, 3, 64, 5, out), (0, buf, 3, 48, 5, out), (0, buf, 0, 64, 5, out),
                (0, buf, 3, 64, 0, out)):
        with pytest.raises(pkg.AdgbError):
            ctx.l2_bench_dev(*bad)
    for cell in (5, 7, 50 * 20 + 8):
        with pytest.raises(pkg.AdgbError):
            ctx.l2_bench_dev(1, buf, 3, 64, 5, out, cell_float4=cell)
    ctx.close()


def test_tcgen05_wait_gives_up_cleanly(pkg, torch):
    """Failure path of the bounded tensor-core completion wait: with nothing
    committed every wait gives up (after a short bounded wait), the outputs
    are NaN, the tensor memory is released and the context keeps working."""
    ctx = make_ctx(pkg)
    x = torch.ones(8 * 256 * 4, device="cuda")
    out = ctx.reduce4_bench_dev(103, x, 256, reps=2)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    ok = ctx.reduce4_bench_dev(pkg.REDUCE4_TCGEN05_TF32X2, x, 256, reps=2)
    assert torch.all(ok == 256.0)
    ctx.close()
