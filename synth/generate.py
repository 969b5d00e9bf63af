"""Seeded generators for receptors, ligands and poses.

Recipe (stands in for the paper's PDB complexes 1stp/7cpa/1ac8/3tmn/3ce3,
Sec. 5, which are not available):

* Receptor: a cubic grid of n^3 points at 0.375 A spacing, centred on the
  origin.  Map m (n_type_maps affinity maps, then the electrostatic map e and
  the desolvation map d) is a sum of 50 isotropic Gaussians, amplitude
  U[-2,2] kcal/mol, centre U(box), sigma U[1,4] A.  The affinity maps also
  carry a steric wall near the box faces: sum over the six faces of
  min((1.5 A / d_face)^12, 1e4).  Stored as float32 [M][nz][ny][nx].
* Ligand: a random bond tree (bond length 1.5 A, bond angle 109.5 deg, random
  dihedrals, valence <= 4), rebuilt until every pair that is not bonded is
  more than 2.0 A apart.  Atom types are uniform over the type classes;
  partial charges ~N(0, 0.3) e shifted to net zero.  T rotatable bonds are
  drawn from the tree bonds whose two atoms are both non-terminal; the root
  fragment holds atom 0.  Each torsion moves the atoms beyond its child atom.
  Torsions are listed root to leaf.  The intramolecular pair list holds the
  pairs i<j that are more than three bonds apart and not in the same rigid
  fragment.  Per-type force-field parameters are seeded: equilibrium
  distance R U[3.0,4.2] A, well depth eps U[0.02,0.2] kcal/mol, atomic
  volume V U[10,35] A^3, atomic solvation parameter U[-0.0015,-0.0005];
  type 0 is a hydrogen-bond donor and type 1 an acceptor (12-10 term with
  R=1.9 A, eps=5.0 kcal/mol).
* Poses: translation uniform in the central 60% of the box, rotation from a
  uniform random unit quaternion (Shoemake's method) expressed as axis
  (azimuth phi, polar theta) and angle alpha, torsions uniform in [-pi, pi).

All values handed to either implementation are float32 (int32 for indices);
the oracle widens the very same numbers to float64.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

BASE_SEED = 241010447

# Named workloads (sizes only).  Index = position in the project's list of
# benchmark configurations.
WORKLOADS = {
    "plain_n16": dict(index=0, grid=40, n_type_maps=6, n_atoms=16, n_types=6,
                      n_tors=4, n_poses=64, ls_iters=300),
    "lga_n32": dict(index=1, grid=64, n_type_maps=8, n_atoms=32, n_types=8,
                    n_tors=8, n_runs=20, pop=150, n_gens=27, ls_iters=300),
    "uneven_512": dict(index=2, grid=72, n_type_maps=10, n_ligands=512,
                       atoms=(10, 128), tors=(0, 32), n_types=10,
                       poses_per_ligand=64, ls_iters=300),
    "serving": dict(index=3, grids=(48, 64, 80, 96), n_type_maps=10,
                    rate_hz=200.0, duration_s=60.0, atoms=(10, 256),
                    tors=(0, 40), n_runs=10, pop=150, evals_per_run=2.5e6),
    "stress_n256": dict(index=4, grid=128, n_type_maps=14, n_atoms=256,
                        n_types=14, n_tors=40, n_poses=8192, ls_iters=500),
}

SPACING = 0.375


def _rng(seed):
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


# ---------------------------------------------------------------- receptor
def make_receptor(seed: int, n: int, n_type_maps: int, spacing: float = SPACING,
                  n_gauss: int = 50, wall: bool = True) -> dict:
    """Gaussian-sum grid maps; see the module docstring for the recipe."""
    rng = _rng(seed)
    M = n_type_maps + 2
    half = 0.5 * (n - 1) * spacing
    origin = np.full(3, -half)
    ax = origin[0] + spacing * np.arange(n)          # same axis for x, y, z
    lo, hi = -half, half
    maps = np.zeros((M, n, n, n), dtype=np.float64)  # [m][z][y][x]
    for m in range(M):
        amp = rng.uniform(-2.0, 2.0, n_gauss)
        cen = rng.uniform(lo, hi, (n_gauss, 3))
        sig = rng.uniform(1.0, 4.0, n_gauss)
        acc = np.zeros((n, n, n))
        for g in range(n_gauss):
            s2 = 2.0 * sig[g] ** 2
            ex = np.exp(-(ax - cen[g, 0]) ** 2 / s2)
            ey = np.exp(-(ax - cen[g, 1]) ** 2 / s2)
            ez = np.exp(-(ax - cen[g, 2]) ** 2 / s2)
            acc += amp[g] * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
        maps[m] = acc
    if wall:
        # distance of each axis coordinate to the nearer of the two faces
        with np.errstate(divide="ignore"):
            f_lo = np.minimum((1.5 / (ax - lo)) ** 12, 1e4)
            f_hi = np.minimum((1.5 / (hi - ax)) ** 12, 1e4)
        w1 = f_lo + f_hi
        wall3 = w1[:, None, None] + w1[None, :, None] + w1[None, None, :]
        maps[:n_type_maps] += wall3[None]
    return dict(nx=n, ny=n, nz=n, spacing=float(spacing),
                origin=origin.astype(np.float32), n_type_maps=int(n_type_maps),
                maps=maps.astype(np.float32))


# ------------------------------------------------------------------ ligand
def _perp_basis(w):
    a = np.array([1.0, 0.0, 0.0]) if abs(w[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(w, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(w, e1)
    return e1, e2


def _grow_tree(rng, n_atoms, chain_bias=0.5, bond=1.5, min_nb=2.0,
               max_tries=60):
    """Random bond tree with 3D coordinates (restarts until it fits)."""
    ang = math.radians(109.5)
    for _restart in range(200):
        xyz = np.zeros((n_atoms, 3))
        parent = np.full(n_atoms, -1)
        deg = np.zeros(n_atoms, dtype=int)
        ok = True
        for i in range(1, n_atoms):
            placed = False
            for _t in range(max_tries):
                if rng.random() < chain_bias and deg[i - 1] < 4:
                    p = i - 1
                else:
                    cand = np.nonzero(deg[:i] < 4)[0]
                    p = int(cand[rng.integers(len(cand))])
                ref = parent[p] if parent[p] >= 0 else -1
                if ref < 0:
                    kids = [c for c in range(i) if parent[c] == p]
                    ref = kids[0] if kids else -1
                if ref < 0:
                    d = rng.normal(size=3)
                    d /= np.linalg.norm(d)
                else:
                    w = xyz[ref] - xyz[p]
                    w /= np.linalg.norm(w)
                    e1, e2 = _perp_basis(w)
                    dih = rng.uniform(-math.pi, math.pi)
                    d = (math.cos(ang) * w
                         + math.sin(ang) * (math.cos(dih) * e1 + math.sin(dih) * e2))
                pos = xyz[p] + bond * d
                dist = np.linalg.norm(xyz[:i] - pos, axis=1)
                dist[p] = np.inf  # the new bond itself
                if np.all(dist > min_nb):
                    xyz[i] = pos
                    parent[i] = p
                    deg[p] += 1
                    deg[i] += 1
                    placed = True
                    break
            if not placed:
                ok = False
                break
        if ok:
            return xyz, parent
    raise RuntimeError("could not grow a ligand tree")


def make_ligand(seed: int, n_atoms: int, n_types: int, n_tors: int,
                chain_bias: float = 0.5) -> dict:
    """Random ligand with torsion tree and pair list (module docstring)."""
    if not (2 <= n_atoms <= 256):
        raise ValueError("n_atoms out of range")
    rng = _rng(seed)
    xyz, parent = _grow_tree(rng, n_atoms, chain_bias)
    N = n_atoms
    adj = [[] for _ in range(N)]
    for i in range(1, N):
        adj[i].append(parent[i])
        adj[parent[i]].append(i)
    deg = np.array([len(a) for a in adj])
    # BFS depth from atom 0 (the tree is rooted there by construction)
    depth = np.zeros(N, dtype=int)
    order = [0]
    for v in order:
        for w in adj[v]:
            if w != 0 and parent[w] == v:
                depth[w] = depth[v] + 1
                order.append(w)
    eligible = [(int(parent[c]), int(c)) for c in range(1, N)
                if deg[c] > 1 and deg[parent[c]] > 1]
    T = min(int(n_tors), len(eligible))
    pick = rng.choice(len(eligible), size=T, replace=False) if T else np.zeros(0, int)
    bonds = sorted((eligible[k] for k in pick), key=lambda ab: (depth[ab[1]], ab[1]))

    def subtree(b):
        out, stack = [], [b]
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if parent[w] == v:
                    out.append(w)
                    stack.append(w)
        return sorted(out)

    moving = [subtree(b) for (_a, b) in bonds]
    offsets = np.zeros(T + 1, dtype=np.int32)
    for k in range(T):
        offsets[k + 1] = offsets[k] + len(moving[k])
    mov_atoms = (np.concatenate([np.asarray(m, dtype=np.int32) for m in moving])
                 if T and offsets[-1] else np.zeros(0, dtype=np.int32))
    # rigid fragment of each atom: the deepest torsion whose moving set holds it
    frag = np.full(N, -1)
    for k in range(T):  # root->leaf, so deeper torsions overwrite
        frag[moving[k]] = k
    # graph distances by BFS
    gd = np.full((N, N), 10 ** 6, dtype=int)
    for s in range(N):
        gd[s, s] = 0
        q = deque([s])
        while q:
            v = q.popleft()
            for w in adj[v]:
                if gd[s, w] > gd[s, v] + 1:
                    gd[s, w] = gd[s, v] + 1
                    q.append(w)
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)
             if gd[i, j] > 3 and frag[i] != frag[j]]
    types = rng.integers(0, n_types, N).astype(np.int32)
    q = rng.normal(0.0, 0.3, N)
    q -= q.mean()
    # per-type force-field parameters (seeded, synthetic)
    R = rng.uniform(3.0, 4.2, n_types)
    eps = rng.uniform(0.02, 0.2, n_types)
    vol = rng.uniform(10.0, 35.0, n_types)
    solpar = rng.uniform(-0.0015, -0.0005, n_types)
    hb_role = np.zeros(n_types, dtype=np.int32)
    if n_types >= 2:
        hb_role[0], hb_role[1] = 1, 2
    centre = xyz.mean(axis=0)
    return dict(
        n_atoms=N, n_types=int(n_types), n_tors=T,
        type=types, charge=q.astype(np.float32),
        xyz=(xyz - centre).astype(np.float32),
        tors_bond=np.asarray(bonds, dtype=np.int32).reshape(T, 2),
        mov_off=offsets, mov_atoms=mov_atoms.astype(np.int32),
        pairs=np.asarray(pairs, dtype=np.int32).reshape(-1, 2),
        R=R.astype(np.float32), eps=eps.astype(np.float32),
        vol=vol.astype(np.float32), solpar=solpar.astype(np.float32),
        hb_role=hb_role, hb_R=np.float32(1.9), hb_eps=np.float32(5.0),
    )


# ------------------------------------------------------------------- poses
def make_poses(seed: int, n_poses: int, receptor: dict, n_tors: int,
               central: float = 0.6) -> np.ndarray:
    """Random genotypes [n][6+T] float32 (module docstring)."""
    rng = _rng(seed)
    lo = receptor["origin"].astype(np.float64)
    ext = (np.array([receptor["nx"], receptor["ny"], receptor["nz"]]) - 1) * receptor["spacing"]
    c = lo + 0.5 * ext
    t = c + (rng.random((n_poses, 3)) - 0.5) * central * ext
    u1, u2, u3 = rng.random(n_poses), rng.random(n_poses), rng.random(n_poses)
    qx = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    qy = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    qz = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    qw = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    alpha = 2.0 * np.arccos(np.clip(qw, -1.0, 1.0))
    vn = np.sqrt(qx * qx + qy * qy + qz * qz)
    vn = np.where(vn < 1e-12, 1.0, vn)
    phi = np.arctan2(qy / vn, qx / vn)
    theta = np.arccos(np.clip(qz / vn, -1.0, 1.0))
    psi = rng.uniform(-np.pi, np.pi, (n_poses, n_tors))
    g = np.concatenate([t, phi[:, None], theta[:, None], alpha[:, None], psi], axis=1)
    return g.astype(np.float32)


# -------------------------------------------------------------- workloads
def make_uneven_batch(seed: int, n_ligands: int, atoms=(10, 128), tors=(0, 32),
                      n_types: int = 10) -> list:
    """Ligands of uneven size (atom count and torsions drawn uniformly)."""
    rng = _rng(seed)
    out = []
    for k in range(n_ligands):
        na = int(rng.integers(atoms[0], atoms[1] + 1))
        nt = int(rng.integers(tors[0], tors[1] + 1))
        out.append(make_ligand(seed * 1000 + k + 1, na, n_types, nt))
    return out


def workload(name: str, n_poses: int | None = None, small: bool = False) -> dict:
    """Receptor, ligand and poses of a named single-ligand workload.

    ``small`` keeps the ligand and grid but shrinks the pose count, for
    parity tests at sizes the oracle finishes in seconds.
    """
    w = WORKLOADS[name]
    s = BASE_SEED + w["index"]
    rec = make_receptor(s, w["grid"], w["n_type_maps"])
    lig = make_ligand(s + 17, w["n_atoms"], w["n_types"], w["n_tors"],
                      chain_bias=0.7 if name == "stress_n256" else 0.5)
    if n_poses is None:
        n_poses = w.get("n_poses", w.get("n_runs", 1) * w.get("pop", 1))
    poses = make_poses(s + 31, n_poses, rec, lig["n_tors"])
    return dict(name=name, receptor=rec, ligand=lig, genes=poses,
                ls_iters=w["ls_iters"])
