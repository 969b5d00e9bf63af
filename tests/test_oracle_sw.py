"""Pins of the oracle's Solis-Wets local search (Solis and Wets, 1981; the
project's reading is written out in oracle/adgb_oracle.c): the normal
deviates, and properties every search must have whatever the random stream.
Cross-implementation agreement with the CUDA library is checked by the GPU
tests."""
import math

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def w():
    return synth.workload("plain_n16", n_poses=24)


def test_sw_normal_is_box_muller_of_philox_words(oracle_mod):
    """Deviate j of a step is the Box-Muller transform of Philox4x32-10 words
    (counter (genotype, step, 0x5357 << 16 | call, j // 4)): cos for even j,
    sin for odd j, words (x, y) for j % 4 < 2 and (z, w) otherwise."""
    seed = 0x1234_5678_9ABC
    for genotype, step, call in ((0, 0, 0), (7, 13, 2), (2999, 299, 65535)):
        for j in range(12):
            o = oracle_mod.philox([genotype, step, 0x53570000 | call, j // 4],
                                  [seed & 0xFFFFFFFF, seed >> 32])
            a, b = (o[2], o[3]) if (j >> 1) & 1 else (o[0], o[1])
            u1 = ((a >> 8) + 1) / 16777216.0
            u2 = (b >> 8) / 16777216.0
            r = math.sqrt(-2.0 * math.log(u1))
            ref = r * (math.sin(2 * math.pi * u2) if j & 1 else math.cos(2 * math.pi * u2))
            assert oracle_mod.sw_normal(seed, genotype, step, call, j) == pytest.approx(ref, abs=1e-15)


def test_sw_normal_statistics(oracle_mod):
    z = np.array([oracle_mod.sw_normal(99, g, s, 0, j)
                  for g in range(40) for s in range(50) for j in range(10)])
    n = len(z)                                            # 20000
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.std() - 1.0) < 0.02
    for k, p in ((1, 0.682689), (2, 0.954500), (3, 0.997300)):
        frac = np.mean(np.abs(z) < k)
        assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n), (k, frac)
    zz = z.reshape(-1, 10)
    c = np.corrcoef(zz.T)
    assert np.max(np.abs(c - np.eye(10))) < 4.5 / math.sqrt(len(zz))   # genes uncorrelated


def test_sw_search_properties(oracle_mod, w):
    rec, lig = w["receptor"], w["ligand"]
    R, L = oracle_mod.Receptor(rec), oracle_mod.Ligand(lig)
    p = oracle_mod.sw_params(max_evals=120, seed=11)
    for k in range(8):
        g0 = w["genes"][k]
        e0 = oracle_mod.score(R, L, g0)[0]
        e, g, ev, st = oracle_mod.sw_search(R, L, g0, p, genotype=k)
        G = len(g0)
        assert e <= e0                                    # x only moves downhill
        assert oracle_mod.score(R, L, g)[0] == pytest.approx(e, rel=1e-12, abs=1e-12)
        assert 1 <= ev <= 120
        assert np.array_equal(st[:G], g) and st[2 * G + 3] == e
        if ev < 120:
            assert st[2 * G] < p.rho_min                   # stopped by the step scale
        rho = st[2 * G]
        assert math.log2(rho / p.rho0) == round(math.log2(rho / p.rho0))   # powers of two
        assert np.all(np.abs(g[6:]) <= math.pi)
    # deterministic; another call id draws another stream
    a = oracle_mod.sw_search(R, L, w["genes"][0], p, genotype=0)
    b = oracle_mod.sw_search(R, L, w["genes"][0], p, genotype=0)
    c = oracle_mod.sw_search(R, L, w["genes"][0], oracle_mod.sw_params(max_evals=120, seed=11, call=1),
                             genotype=0)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[1], c[1])


def test_sw_step_rules(oracle_mod, w):
    """Resumed searches of one and two evaluations apply one step's rules."""
    rec, lig = w["receptor"], w["ligand"]
    R, L = oracle_mod.Receptor(rec), oracle_mod.Ligand(lig)
    G = 6 + lig["n_tors"]
    wrap = lambda v: np.concatenate([v[:6], (v[6:] + np.pi) % (2 * np.pi) - np.pi])
    seen = set()
    for k in range(12):
        for t in (10, 25):
            p = oracle_mod.sw_params(max_evals=t, seed=4, max_succ=2, max_fail=2, angle_scale=0.5)
            _, _, _, st = oracle_mod.sw_search(R, L, w["genes"][k], p, genotype=k)
            x, b = st[:G], st[G:2 * G]
            rho, ns, nf, ex, step = st[2 * G:2 * G + 5]
            if rho < p.rho_min:
                continue
            z = np.array([oracle_mod.sw_normal(4, k, int(step), 0, j) for j in range(G)])
            d = b + rho * np.where(np.arange(G) < 3, 1.0, 0.5) * z
            ep = oracle_mod.score(R, L, wrap(x + d))[0]
            em = oracle_mod.score(R, L, wrap(x - d))[0]
            one = oracle_mod.sw_params(max_evals=1, seed=4, max_succ=2, max_fail=2, angle_scale=0.5)
            e1, g1, ev1, s1 = oracle_mod.sw_search(R, L, x, one, genotype=k, state=st)
            assert ev1 == 1 and s1[2 * G + 4] == step + 1
            if ep < ex:
                seen.add("forward")
                assert np.allclose(g1, wrap(x + d), atol=1e-12) and e1 == pytest.approx(ep)
                assert np.allclose(s1[G:2 * G], 0.2 * b + 0.4 * d, atol=1e-12)
                assert s1[2 * G + 1] == (0 if ns + 1 >= 2 else ns + 1) and s1[2 * G + 2] == 0
                assert s1[2 * G] == (2 * rho if ns + 1 >= 2 else rho)
                continue
            # forward failed with no evaluation left: a failure
            assert np.array_equal(g1, x) and e1 == ex
            assert np.allclose(s1[G:2 * G], 0.5 * b, atol=1e-12)
            assert s1[2 * G + 2] == (0 if nf + 1 >= 2 else nf + 1) and s1[2 * G + 1] == 0
            assert s1[2 * G] == (0.5 * rho if nf + 1 >= 2 else rho)
            two = oracle_mod.sw_params(max_evals=2, seed=4, max_succ=2, max_fail=2, angle_scale=0.5)
            e2, g2, ev2, s2 = oracle_mod.sw_search(R, L, x, two, genotype=k, state=st)
            assert ev2 == 2 and s2[2 * G + 4] == step + 1
            if em < ex:
                seen.add("backward")
                assert np.allclose(g2, wrap(x - d), atol=1e-12) and e2 == pytest.approx(em)
                assert np.allclose(s2[G:2 * G], b - 0.4 * d, atol=1e-12)
            else:
                seen.add("failure")
                assert np.array_equal(g2, x) and np.allclose(s2[G:2 * G], 0.5 * b, atol=1e-12)
    assert {"forward", "failure"} <= seen
    # a scale below rho_min stops at once
    p = oracle_mod.sw_params(max_evals=10, seed=4)
    _, _, _, st = oracle_mod.sw_search(R, L, w["genes"][0], p, genotype=0)
    st[2 * G] = p.rho_min / 2
    e2, g2, ev2, _ = oracle_mod.sw_search(R, L, st[:G], p, genotype=0, state=st)
    assert ev2 == 0 and np.array_equal(g2, st[:G]) and e2 == st[2 * G + 3]
