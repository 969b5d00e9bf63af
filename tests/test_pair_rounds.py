"""Host-side pair schedule for ligands of at most 32 atoms (no GPU): the
library splits the intramolecular pair list (the pair sum of Eq. 1) into
matching rounds in which each lane (atom) computes at most one pair and
receives the reaction force of at most one pair.  Checked here from the
exported round words alone: every caller pair exactly once, the matching
property, the force-source lanes, the H-bond flag, and the round count
ceil(max degree / 2) that a balanced orientation plus bipartite edge
colouring reaches (Konig's theorem)."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def pkg():
    import paper_2410_10447_gb300 as P
    P.build()
    P.load()
    return P


def with_pairs(lig, pairs):
    out = dict(lig)
    out["pairs"] = np.asarray(pairs, np.int32).reshape(-1, 2)
    return out


def check_schedule(pkg, lig):
    N = int(lig["n_atoms"])
    pairs = np.asarray(lig["pairs"]).reshape(-1, 2)
    R, maxdeg, words, perm = pkg.ligand_pair_rounds(lig)
    deg = np.zeros(N, int)
    for i, j in pairs:
        deg[i] += 1
        deg[j] += 1
    assert maxdeg == (deg.max() if len(pairs) else 0)
    if N > 32 or len(pairs) == 0:
        assert R == 0
        return R
    assert R == (maxdeg + 1) // 2
    roles = np.asarray(lig["hb_role"])
    types = np.asarray(lig["type"])
    want = {}
    for i, j in pairs:
        ri, rj = roles[types[i]], roles[types[j]]
        want[frozenset((int(i), int(j)))] = int((ri, rj) in ((1, 2), (2, 1)))
    seen = {}
    for r in range(R):
        w = words[r]
        partner = (w & 31).astype(int)
        src = ((w >> 8) & 31).astype(int)
        hb = ((w >> 24) & 1).astype(int)
        assert np.all((w & ~np.uint32(31 | 31 << 8 | 1 << 24)) == 0)
        has = partner != np.arange(32)
        assert not np.any(has[N:]), "lanes without an atom compute no pair"
        heads = partner[has]
        assert len(set(heads.tolist())) == len(heads), "a lane receives at most one force a round"
        assert np.all(heads < N)
        for a in range(32):
            if has[a]:
                key = frozenset((int(perm[a]), int(perm[partner[a]])))
                assert key not in seen, "pair scheduled twice"
                seen[key] = r
                assert hb[a] == want[key]
                assert src[partner[a]] == a
            else:
                assert hb[a] == 0
        for b in range(32):
            if b not in heads:
                assert not has[src[b]], "no force received: the source lane has no pair (exact zero)"
    assert set(seen) == set(want), "every pair exactly once"
    return R


@pytest.mark.parametrize("n_atoms, n_tors", [(2, 0), (5, 1), (16, 4), (24, 6), (31, 6), (32, 8),
                                             (32, 0), (33, 8)])
def test_synthetic_ligands(pkg, n_atoms, n_tors):
    lig = synth.make_ligand(41_000 + n_atoms, n_atoms, 8, n_tors)
    check_schedule(pkg, lig)


def test_benchmark_ligand(pkg):
    lig = synth.workload("lga_n32", n_poses=1)["ligand"]
    R = check_schedule(pkg, lig)
    assert R > 0


@pytest.mark.parametrize("seed", range(6))
def test_random_pair_sets(pkg, seed):
    """Dense, sparse, odd-degree and star-shaped pair sets on 32 atoms."""
    rng = np.random.default_rng(seed)
    lig = synth.make_ligand(42_000 + seed, 32, 8, 4)
    full = [(i, j) for i in range(32) for j in range(i + 1, 32)]
    keep = [1.0, 0.9, 0.5, 0.1, 0.03, None][seed]
    if keep is None:
        pairs = [(0, j) for j in range(1, 32)] + [(1, 2), (3, 4)]
    else:
        pairs = [p for p in full if rng.random() < keep] or [(0, 1)]
    R = check_schedule(pkg, with_pairs(lig, pairs))
    if keep == 1.0:
        assert R == 16
