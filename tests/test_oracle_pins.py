"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test fixes one part of the definition so that a plausible mistake (a
dropped term, a wrong sign, a swapped axis, a wrong exponent) fails:
finite differences for every gradient, closed forms of the pair terms,
exactness of trilinear interpolation on tensor-product polynomials,
rotations compared with scipy's rotation-vector routine, invariances of the
intramolecular energy, the zero pose, the ADADELTA first step and its
convergence, brute-force / correctly rounded sums, and the Tensor-Core
reduction layout printed in Sec. 4.2.
"""
import math
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------ helpers
def tiny_receptor(n=12, spacing=0.5, n_type_maps=2, fill=None):
    half = 0.5 * (n - 1) * spacing
    origin = np.full(3, -half, np.float32)
    M = n_type_maps + 2
    maps = np.zeros((M, n, n, n), np.float32)
    if fill is not None:
        ax = origin[0] + spacing * np.arange(n)
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        for m in range(M):
            maps[m] = fill(m, X, Y, Z)
    return dict(nx=n, ny=n, nz=n, spacing=spacing, origin=origin,
                n_type_maps=n_type_maps, maps=maps)


def two_atom_ligand(r, types=(0, 1), q=(0.0, 0.0), R=(3.0, 4.0), eps=(0.1, 0.2),
                    vol=(0.0, 0.0), solpar=(0.0, 0.0), hb_role=(0, 0)):
    xyz = np.array([[-r / 2, 0, 0], [r / 2, 0, 0]], np.float64)
    return dict(n_atoms=2, n_types=2, n_tors=0, type=np.array(types, np.int32),
                charge=np.array(q, np.float32), xyz=xyz,
                tors_bond=np.zeros((0, 2), np.int32), mov_off=np.zeros(1, np.int32),
                mov_atoms=np.zeros(0, np.int32), pairs=np.array([[0, 1]], np.int32),
                R=np.array(R, np.float32), eps=np.array(eps, np.float32),
                vol=np.array(vol, np.float32), solpar=np.array(solpar, np.float32),
                hb_role=np.array(hb_role, np.int32), hb_R=np.float32(1.9),
                hb_eps=np.float32(5.0))


def intra(oracle_mod, lig, rec=None):
    rec = rec or tiny_receptor(n=4, spacing=20.0)
    ei, ea, g = oracle_mod.energy(rec, lig, lig["xyz"])
    return ea, g


def away_from_faces(rec, x, tol=1e-4):
    u = (x - np.asarray(rec["origin"], np.float64)) / rec["spacing"]
    return np.all(np.abs(u - np.round(u)) * rec["spacing"] > tol)


@pytest.fixture(scope="module")
def cfg0():
    return synth.workload("plain_n16", n_poses=16)


@pytest.fixture(scope="module")
def cfg1():
    return synth.workload("lga_n32", n_poses=8)


# -------------------------------------------------- finite differences
@pytest.mark.parametrize("which", ["cfg0", "cfg1"])
def test_gene_gradient_matches_central_fd(oracle_mod, which, request):
    w = request.getfixturevalue(which)
    R, L = oracle_mod.Receptor(w["receptor"]), oracle_mod.Ligand(w["ligand"])
    h, checked = 1e-6, 0
    for g0 in w["genes"].astype(np.float64):
        E, gg, x, _ = oracle_mod.score(R, L, g0)
        if not away_from_faces(w["receptor"], x, 1e-3):
            continue
        fd = np.empty_like(gg)
        for k in range(len(g0)):
            gp, gm = g0.copy(), g0.copy()
            gp[k] += h
            gm[k] -= h
            fd[k] = (oracle_mod.score(R, L, gp)[0] - oracle_mod.score(R, L, gm)[0]) / (2 * h)
        scale = max(np.max(np.abs(gg)), 1.0)
        assert np.max(np.abs(fd - gg)) / scale < 1e-5
        checked += 1
    assert checked >= len(w["genes"]) // 2


def test_atom_gradient_matches_central_fd(oracle_mod, cfg1):
    R, L = oracle_mod.Receptor(cfg1["receptor"]), oracle_mod.Ligand(cfg1["ligand"])
    x = oracle_mod.pose_coords(L, cfg1["genes"][0])
    ei, ea, g = oracle_mod.energy(R, L, x)
    h = 1e-6
    fd = np.zeros_like(g)
    for i in range(x.shape[0]):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            ep = sum(oracle_mod.energy(R, L, xp)[:2])
            em = sum(oracle_mod.energy(R, L, xm)[:2])
            fd[i, d] = (ep - em) / (2 * h)
    assert np.max(np.abs(fd - g)) / max(np.max(np.abs(g)), 1.0) < 1e-5


# --------------------------------------------------------- closed forms
def test_vdw_minimum_and_zero_crossing(oracle_mod):
    # 12-6 term with Lorentz-Berthelot mixing: minimum at R_ij=(Ri+Rj)/2,
    # depth w_vdw*sqrt(eps_i eps_j); zero at R_ij * 2^(-1/6).
    Ri, Rj, ei, ej = 3.0, 4.0, 0.1, 0.2
    Rij, eij = 0.5 * (Ri + Rj), math.sqrt(ei * ej)
    e_min, g = intra(oracle_mod, two_atom_ligand(Rij))
    assert e_min == pytest.approx(-0.1662 * eij, rel=1e-6)
    assert np.max(np.abs(g)) < 1e-7 * 0.1662
    e0, _ = intra(oracle_mod, two_atom_ligand(Rij * 2 ** (-1 / 6)))
    assert abs(e0) < 1e-9
    # strictly above the minimum on both sides
    assert intra(oracle_mod, two_atom_ligand(Rij * 0.98))[0] > e_min
    assert intra(oracle_mod, two_atom_ligand(Rij * 1.02))[0] > e_min


def test_hbond_12_10_minimum(oracle_mod):
    # donor-acceptor: 5 (R/r)^12 - 6 (R/r)^10, minimum at R = 1.9 A of depth
    # w_hb * eps_hb, zero crossing at R / sqrt(6/5)
    lig = lambda r: two_atom_ligand(r, hb_role=(1, 2))
    Rh = float(np.float32(1.9))   # the parameters reach both sides as float32
    e_min, g = intra(oracle_mod, lig(Rh))
    assert e_min == pytest.approx(-0.1209 * 5.0, rel=1e-6)
    assert np.max(np.abs(g)) < 1e-6
    assert abs(intra(oracle_mod, lig(Rh / math.sqrt(1.2)))[0]) < 1e-9
    # same roles do not bond: falls back to the 12-6 term
    e66, _ = intra(oracle_mod, two_atom_ligand(3.5, hb_role=(1, 1)))
    assert e66 == pytest.approx(-0.1662 * math.sqrt(0.1 * 0.2), rel=1e-6)


def test_coulomb_dielectric_limits(oracle_mod):
    # E = w_el*332.06363*q1*q2/(r eps(r)) with Mehler & Solmajer's sigmoidal
    # dielectric, which rises monotonically from about 1.35 at contact to
    # water's 78.4 at long range (about half of it near 8 A).
    q1, q2 = float(np.float32(0.4)), float(np.float32(-0.3))
    C = 0.1406 * 332.06363 * q1 * q2
    mk = lambda r: two_atom_ligand(r, q=(0.4, -0.3), eps=(0.0, 0.0))
    epsr = lambda r: C / (r * intra(oracle_mod, mk(r))[0])
    assert epsr(400.0) == pytest.approx(78.4, rel=1e-6)
    assert 35.0 < epsr(8.0) < 55.0
    assert 2.5 < epsr(0.5) < 3.1
    vals = [epsr(r) for r in (0.5, 1, 2, 4, 8, 16, 32, 64)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    # below the clash clamp the energy is frozen at r = 0.5 with zero force
    e_a, g_a = intra(oracle_mod, mk(0.3))
    e_b, _ = intra(oracle_mod, mk(0.5))
    assert e_a == pytest.approx(e_b, rel=1e-12)
    assert np.max(np.abs(g_a)) == 0.0


def test_desolvation_gaussian(oracle_mod):
    # (S_i V_j + S_j V_i) exp(-r^2 / (2 * 3.6^2)), S = solpar + 0.01097 |q|
    sp, vol, q = (-0.001, -0.0007), (20.0, 30.0), (0.0, 0.0)
    mk = lambda r: two_atom_ligand(r, eps=(0.0, 0.0), vol=vol, solpar=sp, q=q)
    e0 = 0.1322 * (sp[0] * vol[1] + sp[1] * vol[0])
    e_small, _ = intra(oracle_mod, mk(1e-9))
    assert e_small == pytest.approx(float(np.float32(sp[0])) * 0.1322 * 30.0
                                    + float(np.float32(sp[1])) * 0.1322 * 20.0, rel=1e-9)
    e_s, _ = intra(oracle_mod, mk(3.6))
    assert e_s / e_small == pytest.approx(math.exp(-0.5), rel=1e-9)
    assert e_small == pytest.approx(e0, rel=1e-6)
    # the charge enters S through 0.01097 |q|; with q = +-0.5 and no
    # Coulomb partner (q on one atom only) S_0 grows by 0.005485
    lig = two_atom_ligand(3.6, eps=(0.0, 0.0), vol=vol, solpar=sp, q=(-0.5, 0.0))
    e_q, _ = intra(oracle_mod, lig)
    s0 = float(np.float32(sp[0])) + 0.01097 * 0.5
    expect = 0.1322 * (s0 * 30.0 + float(np.float32(sp[1])) * 20.0) * math.exp(-0.5)
    assert e_q == pytest.approx(expect, rel=1e-9)


def test_trilinear_exact_on_tensor_product_polynomial(oracle_mod):
    # trilinear interpolation reproduces span{1,x}x{1,y}x{1,z} exactly; a
    # wrong corner weight or swapped axis would not.
    co = np.array([[0.3, 1.1, -0.7, 0.4, 0.05, -0.08, 0.02, 0.003],
                   [-1.0, 0.2, 0.5, -0.9, 0.01, 0.06, -0.04, -0.002],
                   [0.7, -0.3, 0.8, 0.2, -0.03, 0.02, 0.07, 0.001],
                   [0.1, 0.6, -0.2, -0.5, 0.04, -0.05, 0.01, -0.004]])

    def poly(m, X, Y, Z):
        c = co[m]
        return (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * Y + c[5] * Y * Z
                + c[6] * X * Z + c[7] * X * Y * Z)

    rec = tiny_receptor(n=12, spacing=0.5, n_type_maps=2, fill=poly)
    maps64 = rec["maps"].astype(np.float64)
    rng = np.random.default_rng(5)
    for _ in range(20):
        pos = rng.uniform(-2.4, 2.4, 3)
        q = float(np.float32(rng.normal(0, 0.4)))
        lig = dict(n_atoms=1, n_types=2, n_tors=0, type=np.array([1], np.int32),
                   charge=np.array([q], np.float32), xyz=pos[None, :],
                   tors_bond=np.zeros((0, 2), np.int32), mov_off=np.zeros(1, np.int32),
                   mov_atoms=np.zeros(0, np.int32), pairs=np.zeros((0, 2), np.int32),
                   R=np.ones(2, np.float32), eps=np.ones(2, np.float32),
                   vol=np.ones(2, np.float32), solpar=np.ones(2, np.float32),
                   hb_role=np.zeros(2, np.int32), hb_R=np.float32(1.9), hb_eps=np.float32(5.0))
        ei, ea, g = oracle_mod.energy(rec, lig, pos[None, :])
        X, Y, Z = pos
        # the maps hold float32-rounded samples of the polynomial: compare with
        # the polynomial itself to the float32 rounding of the samples
        expect = poly(1, X, Y, Z) + q * poly(2, X, Y, Z) + abs(q) * poly(3, X, Y, Z)
        assert ei == pytest.approx(expect, abs=1e-5)
        eps = 1e-6
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[d] += eps
            pm[d] -= eps
            f = lambda p: (poly(1, *p) + q * poly(2, *p) + abs(q) * poly(3, *p))
            assert g[0, d] == pytest.approx((f(pp) - f(pm)) / (2 * eps), abs=1e-4)
        assert ea == 0.0
    assert maps64.shape == (4, 12, 12, 12)


def test_trilinear_indexing_axis_order(oracle_mod):
    # map = x only: the x-gradient is 1 and the others 0, for every map slot
    rec = tiny_receptor(n=8, spacing=0.375, n_type_maps=1, fill=lambda m, X, Y, Z: X if m == 0 else 0 * X)
    pos = np.array([[0.11, -0.52, 0.33]])
    lig = dict(n_atoms=1, n_types=1, n_tors=0, type=np.array([0], np.int32),
               charge=np.array([0.0], np.float32), xyz=pos,
               tors_bond=np.zeros((0, 2), np.int32), mov_off=np.zeros(1, np.int32),
               mov_atoms=np.zeros(0, np.int32), pairs=np.zeros((0, 2), np.int32),
               R=np.ones(1, np.float32), eps=np.ones(1, np.float32),
               vol=np.ones(1, np.float32), solpar=np.ones(1, np.float32),
               hb_role=np.zeros(1, np.int32), hb_R=np.float32(1.9), hb_eps=np.float32(5.0))
    ei, _, g = oracle_mod.energy(rec, lig, pos)
    assert ei == pytest.approx(0.11, abs=1e-6)
    assert g[0] == pytest.approx([1.0, 0.0, 0.0], abs=1e-6)


def test_out_of_grid_penalty(oracle_mod):
    rec = tiny_receptor(n=8, spacing=0.5)
    hi = float(rec["origin"][0]) + 7 * 0.5
    for delta in (0.1, 0.7, 2.0):
        pos = np.array([[hi + delta, 0.0, 0.0]])
        lig = two_atom_ligand(1.0)
        lig.update(n_atoms=1, type=np.array([0], np.int32), charge=np.array([0.0], np.float32),
                   xyz=pos, pairs=np.zeros((0, 2), np.int32))
        ei, _, g = oracle_mod.energy(rec, lig, pos)
        assert ei == pytest.approx(10.0 * delta ** 2, rel=1e-9)
        assert g[0] == pytest.approx([20.0 * delta, 0.0, 0.0], rel=1e-9)


# ------------------------------------------------------ pose geometry
def test_zero_pose_reproduces_input_exactly(oracle_mod, cfg1):
    lig = cfg1["ligand"]
    G = 6 + lig["n_tors"]
    x = oracle_mod.pose_coords(lig, np.zeros(G))
    assert np.array_equal(x, lig["xyz"].astype(np.float64))
    # translation only: exactly input + t
    t = np.array([1.25, -3.5, 0.75])
    g = np.zeros(G)
    g[:3] = t
    x = oracle_mod.pose_coords(lig, g)
    assert np.array_equal(x, lig["xyz"].astype(np.float64) + t)
    # rotation axis genes without an angle change nothing
    g = np.zeros(G)
    g[3:5] = (0.7, 1.9)
    assert np.array_equal(oracle_mod.pose_coords(lig, g), lig["xyz"].astype(np.float64))


def test_rigid_rotation_matches_scipy_rotvec(oracle_mod, cfg1):
    from scipy.spatial.transform import Rotation
    lig = cfg1["ligand"]
    G = 6 + lig["n_tors"]
    rng = np.random.default_rng(3)
    for _ in range(5):
        phi, theta, alpha = rng.uniform(-np.pi, np.pi), rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)
        t = rng.normal(size=3)
        g = np.zeros(G)
        g[:6] = (*t, phi, theta, alpha)
        u = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
        Rm = Rotation.from_rotvec(alpha * u).as_matrix()
        expect = lig["xyz"].astype(np.float64) @ Rm.T + t
        assert np.max(np.abs(oracle_mod.pose_coords(lig, g) - expect)) < 1e-12


def test_torsions_match_leaf_to_root_rotations(oracle_mod, cfg1):
    # independent construction: apply each torsion's rotation about its
    # REFERENCE bond axis from the deepest torsion to the root (scipy
    # matrices), then the rigid motion; must equal the oracle's root-to-leaf
    # pass on updated axes.
    from scipy.spatial.transform import Rotation
    lig = cfg1["ligand"]
    T = lig["n_tors"]
    ref = lig["xyz"].astype(np.float64)
    rng = np.random.default_rng(11)
    for _ in range(5):
        g = np.concatenate([rng.normal(size=3), [0.3, 1.2, 0.8], rng.uniform(-np.pi, np.pi, T)])
        p = ref.copy()
        for k in reversed(range(T)):
            a, b = lig["tors_bond"][k]
            ax = ref[b] - ref[a]
            ax /= np.linalg.norm(ax)
            Rk = Rotation.from_rotvec(g[6 + k] * ax).as_matrix()
            mv = lig["mov_atoms"][lig["mov_off"][k]:lig["mov_off"][k + 1]]
            p[mv] = (p[mv] - ref[b]) @ Rk.T + ref[b]
        u = np.array([np.sin(g[4]) * np.cos(g[3]), np.sin(g[4]) * np.sin(g[3]), np.cos(g[4])])
        expect = p @ Rotation.from_rotvec(g[5] * u).as_matrix().T + g[:3]
        assert np.max(np.abs(oracle_mod.pose_coords(lig, g) - expect)) < 1e-12


def test_intra_energy_invariant_under_rigid_motion(oracle_mod, cfg1):
    R, L = oracle_mod.Receptor(cfg1["receptor"]), oracle_mod.Ligand(cfg1["ligand"])
    lig = cfg1["ligand"]
    g0 = cfg1["genes"][2].astype(np.float64)
    _, ea0, _ = oracle_mod.energy(R, L, oracle_mod.pose_coords(L, g0))
    rng = np.random.default_rng(7)
    for _ in range(5):
        g = g0.copy()
        g[:6] = (*rng.normal(size=3) * 4, rng.uniform(-3, 3), rng.uniform(0, 3), rng.uniform(0, 6))
        _, ea, _ = oracle_mod.energy(R, L, oracle_mod.pose_coords(L, g))
        assert ea == pytest.approx(ea0, rel=1e-12)
    # bond lengths of the tree never change under any genotype
    x = oracle_mod.pose_coords(L, g0)
    ref = lig["xyz"].astype(np.float64)
    for (a, b) in lig["tors_bond"]:
        assert np.linalg.norm(x[a] - x[b]) == pytest.approx(np.linalg.norm(ref[a] - ref[b]), rel=1e-12)


def test_translation_gradient_is_sum_of_atom_gradients(oracle_mod, cfg0):
    R, L = oracle_mod.Receptor(cfg0["receptor"]), oracle_mod.Ligand(cfg0["ligand"])
    for g0 in cfg0["genes"][:4]:
        E, gg, x, ag = oracle_mod.score(R, L, g0)
        assert gg[:3] == pytest.approx(ag.sum(axis=0), rel=1e-12, abs=1e-9)
        # intramolecular forces are internal: they cancel in the net force
        ei, ea, gi = oracle_mod.energy(R, L, x)
        lig_only = dict(cfg0["ligand"])
        rec0 = tiny_receptor(n=4, spacing=40.0, n_type_maps=cfg0["receptor"]["n_type_maps"])
        _, _, g_intra = oracle_mod.energy(rec0, lig_only, x)
        assert np.abs(g_intra.sum(axis=0)).max() < 1e-9 * max(1.0, np.abs(g_intra).max())


# -------------------------------------------------------------- ADADELTA
def test_adadelta_first_step_closed_form(oracle_mod):
    rho, eps = 0.8, 1e-2
    g = np.array([3.0, -0.5, 1e-3, 0.0, 250.0, -7.0, 2.0])
    om = np.linspace(-1, 1, 7)
    om1, eg2, ed2 = oracle_mod.adadelta_step(g, om, np.zeros(7), np.zeros(7), rho, eps)
    d = -math.sqrt(eps) / np.sqrt((1 - rho) * g ** 2 + eps) * g
    assert om1[:6] == pytest.approx(om[:6] + d[:6], rel=1e-14, abs=1e-15)
    # gene 6 is a torsion: wrapped into [-pi, pi)
    assert -np.pi <= om1[6] < np.pi
    assert eg2 == pytest.approx((1 - rho) * g ** 2)
    assert ed2 == pytest.approx((1 - rho) * d ** 2)
    # the step never exceeds sqrt(eps/(1-rho)) in size on the first update
    assert np.all(np.abs(d) <= math.sqrt(eps / (1 - rho)) + 1e-15)


def test_adadelta_converges_on_quadratic_bowl(oracle_mod):
    # Near the optimum E[g^2] and E[d^2] are small against eps, so the update
    # is d ~ -g = -a (Omega - c): a linear map with factor (1 - a), which
    # contracts for curvatures 0 < a < 2 (ADADELTA has no learning rate).
    a = np.array([1.0, 1.5, 0.25, 0.8, 0.5, 1.2])
    c = np.array([0.3, -0.2, 0.9, -0.4, 0.1, 0.25])
    om = np.zeros(6)
    eg2, ed2 = np.zeros(6), np.zeros(6)
    for _ in range(3000):
        om, eg2, ed2 = oracle_mod.adadelta_step(a * (om - c), om, eg2, ed2, 0.8, 1e-2)
    assert np.max(np.abs(om - c)) < 1e-6
    # a stiff direction (a = 4, factor -3) does not settle
    om, eg2, ed2 = np.zeros(6), np.zeros(6), np.zeros(6)
    a4 = np.full(6, 4.0)
    for _ in range(200):
        om, eg2, ed2 = oracle_mod.adadelta_step(a4 * (om - c), om, eg2, ed2, 0.8, 1e-2)
    assert np.max(np.abs(om - c)) > 0.1


def test_local_search_lowers_energy_and_returns_its_best(oracle_mod, cfg0):
    R, L = oracle_mod.Receptor(cfg0["receptor"]), oracle_mod.Ligand(cfg0["ligand"])
    for g0 in cfg0["genes"][:4]:
        e0 = oracle_mod.score(R, L, g0)[0]
        best, bg, st = oracle_mod.local_search(R, L, g0, 50)
        assert best <= e0
        # the returned genotype really has the returned energy
        assert oracle_mod.score(R, L, bg)[0] == pytest.approx(best, rel=1e-12)
        # one iteration = the initial evaluation only
        b1, g1, _ = oracle_mod.local_search(R, L, g0, 1)
        assert b1 == pytest.approx(e0, rel=1e-15) and np.array_equal(g1, g0.astype(np.float64))


# ------------------------------------------------------------ reductions
def test_sums_against_correctly_rounded_fsum(oracle_mod):
    rng = np.random.default_rng(0)
    x = rng.normal(size=10000) * 10.0 ** rng.integers(-6, 7, 10000)
    exact = math.fsum(x)
    assert oracle_mod.sum_neumaier(x) == exact
    assert abs(oracle_mod.sum_naive(x) - exact) <= 1e-12 * np.abs(x).sum()
    adv = np.array([1e16, 1.0, -1e16, 3.0, 1e6, -1e6, 0.5])
    assert oracle_mod.sum_neumaier(adv) == math.fsum(adv) == 4.5
    assert oracle_mod.sum_naive(np.arange(1, 1001, dtype=np.float64)) == 500500.0


def test_tcu_reduction_layout_of_section_4_2():
    """Sec. 4.2: A (16x16, 64 vectors), P = ones, Q = blocks of I4; V <- AP + V
    over 64-vector tiles and W = QV leave the four sums in W[0..3][0]."""
    rows = []
    with open(os.path.join(HERE, "golden", "tcu_layout_sec4_2.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    comp = {"x": 0, "y": 1, "z": 2, "e": 3}

    def A_entry(r, c):          # our reading of the printed layout
        return (r % 4, 4 * c + r // 4)

    for m, r, c, sym in rows:
        if m == "A":
            k, v = A_entry(int(r), int(c))
            assert (k, v) == (comp[sym[0]], int(sym[1:]))
    rng = np.random.default_rng(1)
    n_tiles = 3
    u = rng.normal(size=(64 * n_tiles, 4))
    P = np.ones((16, 16))
    Q = np.kron(np.ones((4, 4)), np.eye(4))
    V = np.zeros((16, 16))
    for t in range(n_tiles):
        A = np.zeros((16, 16))
        for r in range(16):
            for c in range(16):
                k, v = A_entry(r, c)
                A[r, c] = u[64 * t + v, k]
        V = A @ P + V
    W = Q @ V
    for m, r, c, sym in rows:
        r = int(r)
        if m == "V":
            k = comp[sym.split("_")[1]]
            res = 0 if sym.endswith("4i") else int(sym.split("+")[1])
            want = sum(u[64 * t + 4 * i + res, k] for t in range(n_tiles) for i in range(16))
            assert np.allclose(V[r], want)
        if m == "W":
            k = comp[sym.split("_")[1]]
            assert np.allclose(W[r], u[:, k].sum())
    assert np.allclose(W[:4, 0], u.sum(axis=0))


# ------------------------------------------- gradient magnitudes (conditioning)
def test_gradient_magnitude_closed_form_constant_maps(oracle_mod):
    # one atom at the rotation centre in constant maps: the gradient is zero
    # and each axis' magnitude is the corner shares' absolute sum,
    # 2 (|c_t| + |q c_e| + |q| |c_d|) / h (the eight y-z weights sum to 2)
    ct, ce, cd, h = 1.5, -0.7, 0.4, 0.5
    vals = {0: ct, 1: ce, 2: cd}
    rec = tiny_receptor(n=10, spacing=h, n_type_maps=1,
                        fill=lambda m, X, Y, Z: vals[m] + 0 * X)
    q = -0.35
    lig = dict(n_atoms=1, n_types=1, n_tors=0, type=np.array([0], np.int32),
               charge=np.array([q], np.float32), xyz=np.zeros((1, 3)),
               tors_bond=np.zeros((0, 2), np.int32), mov_off=np.zeros(1, np.int32),
               mov_atoms=np.zeros(0, np.int32), pairs=np.zeros((0, 2), np.int32),
               R=np.ones(1, np.float32), eps=np.ones(1, np.float32),
               vol=np.ones(1, np.float32), solpar=np.ones(1, np.float32),
               hb_role=np.zeros(1, np.int32), hb_R=np.float32(1.9), hb_eps=np.float32(5.0))
    qf = float(np.float32(q))
    want = 2.0 * (abs(ct) + abs(qf * ce) + abs(qf) * abs(cd)) / h
    rng = np.random.default_rng(3)
    for _ in range(5):
        genes = np.concatenate([rng.uniform(-1.5, 1.5, 3), rng.uniform(0, 3, 3)])
        _, g, _, _ = oracle_mod.score(rec, lig, genes)
        m = oracle_mod.score_magnitude(rec, lig, genes)
        assert np.allclose(g, 0.0, atol=1e-9)
        assert m[:3] == pytest.approx([want] * 3, rel=1e-5)   # maps hold float32 values
        assert np.all(m[3:] == 0.0)                            # no lever arm
        # coordinate rounding: no pairs, so nothing for the translation; the
        # rotation genes' lever x - t is zero but computed from coordinates of
        # size |x|_inf, so each takes sum_d |g|_d |x|_inf = 3 want |x|_inf
        _, pm = oracle_mod.score_magnitude(rec, lig, genes, with_positions=True)
        assert np.all(pm[:3] == 0.0)
        assert pm[3:] == pytest.approx([3 * want * np.max(np.abs(genes[:3]))] * 3, rel=1e-5)
    # outside the grid along x: only the wall's gradient, 2 W_OUT d
    hi = float(rec["origin"][0]) + 9 * h
    genes = np.array([hi + 0.6, 0.0, 0.0, 0.0, 0.0, 0.0])
    m = oracle_mod.score_magnitude(rec, lig, genes)
    assert m[0] == pytest.approx(2 * 10.0 * 0.6, rel=1e-9)


@pytest.mark.parametrize("which", ["cfg0", "cfg1"])
def test_gradient_magnitude_bounds_the_gradient(oracle_mod, which, request):
    # triangle inequality: the absolute sum of the contributions bounds the sum
    w = request.getfixturevalue(which)
    R, L = oracle_mod.Receptor(w["receptor"]), oracle_mod.Ligand(w["ligand"])
    for p in range(min(12, w["genes"].shape[0])):
        _, g, _, _ = oracle_mod.score(R, L, w["genes"][p])
        m = oracle_mod.score_magnitude(R, L, w["genes"][p])
        assert np.all(m >= np.abs(g) * (1 - 1e-12) - 1e-12), (p, m, g)
        assert np.all(np.isfinite(m))
        # coordinate rounding: a pair force enters a gene through the difference
        # of its atoms' velocities, which is zero for the translation genes
        m2, pm = oracle_mod.score_magnitude(R, L, w["genes"][p], with_positions=True)
        assert np.array_equal(m2, m)
        assert np.all(pm[:3] == 0.0) and np.all(pm >= 0.0) and np.all(np.isfinite(pm))
