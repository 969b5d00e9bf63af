"""Host-side pair schedule (no GPU): the library splits the intramolecular
pair list (the pair sum in Sec. 2.1's scoring function; the schedule has no
paper counterpart) into rounds in which each lane (atom) computes at most
one pair and receives the reaction forces of at most two
pairs; 32 lanes up to 32 atoms (one warp), the atoms rounded up to 32 above
112 atoms (a block of threads), none between (the force buffer is faster).
Checked here from the exported round words alone: every caller pair exactly
once, at most one computed and two received pairs
a lane a round, the force-source lanes and their flags, lanes past the last
atom idle and pointing at a real atom, the H-bond flag, and the round count
max(ceil(pairs / atoms), ceil(max degree / 3)), the lower bound of the scheme
(one lane an atom; an atom in at most three pairs a round), reached through
an out-degree-bounded orientation and a bipartite edge colouring (Konig's
theorem)."""
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
    R, lanes, maxdeg, words, perm = pkg.ligand_pair_rounds(lig)
    deg = np.zeros(N, int)
    for i, j in pairs:
        deg[i] += 1
        deg[j] += 1
    assert maxdeg == (deg.max() if len(pairs) else 0)
    if len(pairs) == 0 or 32 < N <= 112:   # no pairs; or the force buffer is faster
        assert R == 0 and lanes == 0
        return R
    assert lanes == (32 if N <= 32 else -(-N // 32) * 32)
    assert words.shape == (R, lanes)
    assert R >= max(-(-len(pairs) // N), -(-maxdeg // 3))
    roles = np.asarray(lig["hb_role"])
    types = np.asarray(lig["type"])
    want = {}
    for i, j in pairs:
        ri, rj = roles[types[i]], roles[types[j]]
        want[frozenset((int(i), int(j)))] = int((ri, rj) in ((1, 2), (2, 1)))
    seen = {}
    ids = np.arange(lanes)
    for r in range(R):
        w = words[r].astype(np.int64)
        partner = w & 255
        src = [(w >> 8) & 255, (w >> 16) & 255]
        used = [(w >> 25) & 1, (w >> 26) & 1]
        hb = (w >> 24) & 1
        assert np.all(w & ~(255 | 255 << 8 | 255 << 16 | 7 << 24) == 0)
        assert np.all(partner < N), "every partner is a real atom"
        assert np.all(src[0] < lanes) and np.all(src[1] < lanes)
        has = (partner != ids) & (ids < N)
        assert np.all(partner[N:] == 0) and not np.any(used[0][N:]) and not np.any(used[1][N:])
        received = {b: [] for b in range(lanes)}
        for k in range(2):
            for b in np.nonzero(used[k])[0]:
                received[int(b)].append(int(src[k][b]))
        for a in np.nonzero(has)[0]:
            key = frozenset((int(perm[a]), int(perm[partner[a]])))
            assert key not in seen, "pair scheduled twice"
            seen[key] = r
            assert hb[a] == want[key]
            b = int(partner[a])
            assert received[b].count(int(a)) == 1, "the partner receives the force once"
        assert not np.any(hb[~has])
        for b in range(lanes):
            assert len(received[b]) <= 2
            for a in received[b]:
                assert has[a] and partner[a] == b, "a used slot names a lane whose pair has atom b second"
    assert set(seen) == set(want), "every pair exactly once"
    return R


@pytest.mark.parametrize("n_atoms, n_tors", [(2, 0), (5, 1), (16, 4), (24, 6), (31, 6), (32, 8),
                                             (32, 0), (33, 8), (48, 12), (64, 16), (100, 20),
                                             (129, 32), (256, 40)])
def test_synthetic_ligands(pkg, n_atoms, n_tors):
    lig = synth.make_ligand(41_000 + n_atoms, n_atoms, 8, n_tors)
    check_schedule(pkg, lig)


def test_benchmark_ligand(pkg):
    lig = synth.workload("lga_n32", n_poses=1)["ligand"]
    R = check_schedule(pkg, lig)
    assert R == 11              # 330 pairs / 32 lanes; max degree 28 needs only 10


def test_dense_subset_raises_the_round_count(pkg):
    """20 of 32 atoms pairwise linked, the rest bare: 190 pairs on 20 lanes
    need ceil(190 / 20) = 10 rounds although max(ceil(190 / 32), ceil(19 / 3))
    is 7: no orientation gives every atom at most 7 out-edges."""
    lig = synth.make_ligand(43_000, 32, 8, 4)
    pairs = [(i, j) for i in range(20) for j in range(i + 1, 20)]
    assert check_schedule(pkg, with_pairs(lig, pairs)) == 10


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
    deg = np.bincount(np.asarray(pairs).ravel(), minlength=32)
    if keep != 1.0:
        assert R == max(-(-len(pairs) // 32), -(-deg.max() // 3))
    if keep == 1.0:
        assert R == 16          # 496 pairs / 32 lanes (degree 31 alone: 11 rounds)


def test_largest_pair_list(pkg):
    """The maximum: 256 atoms, every pair (32,640).  Lanes need all 8 bits of
    the word's lane fields; 128 rounds = ceil(32640 / 256)."""
    lig = synth.make_ligand(44_000, 256, 8, 40)
    pairs = [(i, j) for i in range(256) for j in range(i + 1, 256)]
    assert check_schedule(pkg, with_pairs(lig, pairs)) == 128
