"""Pins of the oracle's Lamarckian GA pieces (Sec. 2.1; the rules are this
project's reading, stated in oracle/adgb_oracle.c): the Philox4x32-10
generator against its published known-answer vectors, properties every
generation must have whatever the random stream, and statistics of the
stream.  Cross-implementation agreement with the CUDA library is checked by
the GPU tests."""
import math

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def w():
    return synth.workload("plain_n16", n_poses=40)


def test_philox_known_answer_vectors(oracle_mod, philox_kat):
    # Salmon et al. (SC'11) publish these words with their reference
    # implementation; a swapped round multiplier, a wrong Weyl key increment
    # or a key bumped before the first round changes every output word
    kat = philox_kat
    assert len(kat) == 3
    for ctr, key, want in kat:
        assert list(oracle_mod.philox(ctr, key)) == want, (ctr, key)


def test_philox_statistics(oracle_mod):
    # 2^14 calls: the 65536 words are uniform over 16 bins (chi-square, 15
    # d.o.f., 0.1% critical value 37.7) and every bit is set about half the
    # time; a single flipped counter bit flips about half the output bits
    words = []
    for i in range(1 << 14):
        words += oracle_mod.philox([i, 7, 3, 1], [0x1234, 0x9876])
    w = np.array(words, np.uint64)
    counts = np.bincount((w >> 28).astype(int), minlength=16)
    chi2 = ((counts - w.size / 16) ** 2 / (w.size / 16)).sum()
    assert chi2 < 37.7
    bits = np.array([((w >> b) & 1).mean() for b in range(32)])
    assert np.all(np.abs(bits - 0.5) < 0.02)
    a = oracle_mod.philox([5, 6, 7, 8], [1, 2])
    flips = []
    for b in range(128):
        c = [5, 6, 7, 8]
        c[b // 32] ^= 1 << (b % 32)
        o = oracle_mod.philox(c, [1, 2])
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, o)))
    assert 56 < np.mean(flips) < 72
    assert len(set(tuple(oracle_mod.philox([i, 0, 0, 0], [0, 0])) for i in range(5000))) == 5000


def test_initial_population_ranges(oracle_mod, w):
    rec = w["receptor"]
    T = w["ligand"]["n_tors"]
    lo = np.asarray(rec["origin"], np.float64)
    ext = (rec["nx"] - 1) * rec["spacing"]
    G = np.array([oracle_mod.init_individual(rec, T, 99, r, k) for r in range(3) for k in range(200)])
    assert np.all(G[:, :3] >= lo + 0.2 * ext - 1e-9) and np.all(G[:, :3] <= lo + 0.8 * ext + 1e-9)
    assert np.all(np.abs(G[:, 3]) <= np.pi) and np.all((G[:, 4] >= 0) & (G[:, 4] <= np.pi))
    assert np.all((G[:, 5] >= 0) & (G[:, 5] < 2 * np.pi)) and np.all(np.abs(G[:, 6:]) <= np.pi)
    # the axis is uniform on the sphere: cos(theta) is uniform in [-1, 1]
    assert abs(np.cos(G[:, 4]).mean()) < 0.1
    # deterministic in (seed, run, k), different across them
    assert np.array_equal(G[0], oracle_mod.init_individual(rec, T, 99, 0, 0))
    assert not np.array_equal(G[0], G[1])


def test_ga_generation_properties(oracle_mod, w):
    rng = np.random.default_rng(4)
    pop, G = 40, 6 + w["ligand"]["n_tors"]
    genes = rng.normal(size=(pop, G))
    energies = rng.normal(size=pop) * 10
    energies[7] = energies.min() - 5
    prm = oracle_mod.dock_params(pop=pop, p_cross=0.8, p_mut=0.1, ls_rate=0.5, seed=11)
    new, fl = oracle_mod.ga_generation(genes, energies, prm, 2, 5)
    assert np.array_equal(new[0], genes[7])                      # elitism
    mutated = 0
    for k in range(1, pop):
        child = new[k]
        # every gene comes from some parent, or is a bounded mutation of one
        src = np.abs(genes - child[None, :])
        for j in range(G):
            d = src[:, j].min()
            if d > 1e-12:
                scale = 2.0 if j < 3 else np.pi / 2
                if j >= 6:
                    dd = np.abs((genes[:, j] - child[j] + np.pi) % (2 * np.pi) - np.pi).min()
                    d = dd
                assert d <= scale + 1e-12
                mutated += 1
    frac = mutated / ((pop - 1) * G)
    assert 0.03 < frac < 0.2
    assert np.all(np.abs(new[:, 6:]) <= np.pi)
    assert 0.2 < fl.mean() < 0.8
    # with no crossover and no mutation each child is a tournament winner:
    # its energy is not above the median-of-two of random picks, i.e. the
    # children's parents have lower energy on average than the population
    prm0 = oracle_mod.dock_params(pop=pop, p_cross=0.0, p_mut=0.0, seed=12)
    new0, _ = oracle_mod.ga_generation(genes, energies, prm0, 0, 1)
    idx = [int(np.argmin(np.abs(genes - c[None, :]).sum(axis=1))) for c in new0]
    assert all(np.array_equal(new0[k], genes[idx[k]]) for k in range(pop))
    assert energies[idx[1:]].mean() < energies.mean()


def test_dock_accounting_and_best(oracle_mod, w):
    prm = oracle_mod.dock_params(n_runs=2, pop=12, max_gens=3, ls_iters=15, ls_rate=0.5, seed=5)
    bg, be, ev = oracle_mod.dock(w["receptor"], w["ligand"], prm)
    R, L = oracle_mod.Receptor(w["receptor"]), oracle_mod.Ligand(w["ligand"])
    for r in range(2):
        assert oracle_mod.score(R, L, bg[r])[0] == pytest.approx(be[r], rel=1e-12)
        init = [oracle_mod.score(R, L, oracle_mod.init_individual(w["receptor"], L.n_tors, 5, r, k))[0]
                for k in range(12)]
        assert be[r] <= min(init)
        # 12 initial scores, then per generation 15 or 1 evaluations per individual
        n_ls = (ev[r] - 12 - 3 * 12) / 14
        assert n_ls == int(n_ls) and 0 <= n_ls <= 36
    # the evaluation budget stops a run early
    prm2 = oracle_mod.dock_params(n_runs=1, pop=12, max_gens=10, max_evals=100, ls_iters=15, ls_rate=1.0, seed=5)
    _, _, ev2 = oracle_mod.dock(w["receptor"], w["ligand"], prm2)
    assert ev2[0] == 12 + 12 * 15


# ----------------------------------------------------------- early stopping
def test_converged_is_the_std_of_the_lowest(oracle_mod):
    """The early-stopping test reduces to numpy's population standard
    deviation of the sorted lowest energies."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        pop = int(rng.integers(2, 300))
        top = int(rng.integers(2, pop + 1))
        e = rng.normal(-10.0, 10.0 ** rng.uniform(-3, 1), pop)
        tol = float(10.0 ** rng.uniform(-3, 1))
        ref = np.std(np.sort(e)[:top]) < tol
        assert oracle_mod.converged(e, top, tol) == ref
        assert oracle_mod.converged(rng.permutation(e), top, tol) == ref
    # worked case: lowest three are -10.1, -10.0, -9.9 -> std = sqrt(0.02 / 3) = 0.08165
    e = np.array([5.0, -10.0, 7.0, -9.9, -10.1, 3.0])
    assert oracle_mod.converged(e, 3, 0.082) and not oracle_mod.converged(e, 3, 0.0816)
    # non-finite among the lowest: not converged; above them: irrelevant
    assert not oracle_mod.converged(np.array([-1.0, np.nan, -1.0, 4.0]), 2, 1.0)
    assert oracle_mod.converged(np.array([-1.0, np.inf, -1.0, 4.0]), 2, 1.0)


def test_dock_early_stopping_accounting(oracle_mod, w):
    rec, lig = w["receptor"], w["ligand"]
    base = dict(n_runs=3, pop=12, max_gens=6, ls_iters=5, ls_rate=1.0, seed=3)
    full = 12 + 6 * 12 * 5
    _, _, ev = oracle_mod.dock(rec, lig, oracle_mod.dock_params(**base))
    assert np.all(ev == full)
    _, _, ev = oracle_mod.dock(rec, lig, oracle_mod.dock_params(conv_every=2, conv_top=4,
                                                                  conv_tol=1e6, **base))
    assert np.all(ev == 12 + 2 * 12 * 5)
    b0, e0, ev0 = oracle_mod.dock(rec, lig, oracle_mod.dock_params(**base))
    b1, e1, ev1 = oracle_mod.dock(rec, lig, oracle_mod.dock_params(conv_every=2, conv_top=4,
                                                                     conv_tol=1e-12, **base))
    assert np.array_equal(ev0, ev1) and np.array_equal(e0, e1) and np.array_equal(b0, b1)


def test_dock_with_solis_wets_accounting(oracle_mod, w):
    """The oracle's LGA with Solis-Wets searches counts the evaluations they
    spend (at most ls_iters each) and keeps the best energy it saw."""
    rec, lig = w["receptor"], w["ligand"]
    prm = oracle_mod.dock_params(n_runs=3, pop=10, max_gens=3, ls_iters=30, ls_rate=1.0, seed=8,
                                 ls_method=1)
    bg, be, ev = oracle_mod.dock(rec, lig, prm)
    assert np.all(ev >= 10 + 3 * 10) and np.all(ev <= 10 + 3 * 10 * 30)
    R, L = oracle_mod.Receptor(rec), oracle_mod.Ligand(lig)
    for r in range(3):
        assert oracle_mod.score(R, L, bg[r])[0] == pytest.approx(be[r], rel=1e-12, abs=1e-12)
    bg2, be2, ev2 = oracle_mod.dock(rec, lig, prm)
    assert np.array_equal(be, be2) and np.array_equal(ev, ev2)
