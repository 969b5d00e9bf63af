"""C ABI checks that need no GPU: the library loads, exports every function
include/adgb.h declares, and rejects malformed ligands / torsion trees."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2410_10447_gb300 as P
    P.build()
    P.load()
    return P


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(",
                             src, flags=re.M):
            line = src[m.start():src.index("\n", m.start())]
            if line.lstrip().startswith(("typedef", "#", "return")):
                continue
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("upload_receptor_grids", "upload_ligand_torsion_tree", "score_poses",
                 "local_search", "score_poses_dev", "local_search_dev", "pose_coords",
                 "adgb_create", "adgb_destroy", "adgb_last_error", "reduce4_bench_dev"):
        assert must in names, must


def test_library_exports_every_declared_symbol(pkg):
    lib = ctypes.CDLL(pkg.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pkg.EXPORTS) <= declared_functions()


def test_create_without_device_fails_cleanly(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(pkg.AdgbError) as ei:
        pkg.Context(0)
    assert ei.value.code == -4  # EDEVICE


@pytest.mark.parametrize("name", ["plain_n16", "lga_n32", "stress_n256"])
def test_generated_ligands_are_valid(pkg, name):
    w = synth.WORKLOADS[name]
    lig = synth.make_ligand(synth.generate.BASE_SEED + w["index"] + 17, w["n_atoms"],
                            w["n_types"], w["n_tors"])
    rc, msg = pkg.validate_ligand_torsion_tree(lig)
    assert rc == 0, msg


def test_uneven_ligands_are_valid(pkg):
    for lig in synth.make_uneven_batch(7, 12):
        rc, msg = pkg.validate_ligand_torsion_tree(lig)
        assert rc == 0, msg


def _base():
    return synth.make_ligand(123, 24, 6, 6)


def _reorder(lig, order):
    """Lists the torsions in another order (moving sets follow)."""
    lig = dict(lig)
    mo, ma = lig["mov_off"], lig["mov_atoms"]
    sets = [ma[mo[k]:mo[k + 1]] for k in range(len(mo) - 1)]
    sets = [sets[k] for k in order]
    lig["tors_bond"] = lig["tors_bond"][order]
    lig["mov_atoms"] = np.concatenate(sets).astype(np.int32)
    lig["mov_off"] = np.concatenate([[0], np.cumsum([len(s) for s in sets])]).astype(np.int32)
    return lig


def test_child_listed_before_parent_is_rejected(pkg):
    lig = _base()
    T = lig["n_tors"]
    mo, ma = lig["mov_off"], lig["mov_atoms"]
    sets = [set(ma[mo[k]:mo[k + 1]]) for k in range(T)]
    pair = next(((k, q) for k in range(T) for q in range(k + 1, T) if sets[q] < sets[k]), None)
    assert pair is not None, "the generated ligand has nested torsions"
    order = list(range(T))
    order[pair[0]], order[pair[1]] = order[pair[1]], order[pair[0]]
    rc, msg = pkg.validate_ligand_torsion_tree(_reorder(lig, order))
    assert rc == -1 and ("listed after" in msg or "nested" in msg), msg


@pytest.mark.parametrize("mutate, words", [
    (lambda L: L.update(n_atoms=257), "n_atoms"),
    (lambda L: L.update(n_types=17), "n_types"),
    (lambda L: L.update(n_tors=41), "n_tors"),
    (lambda L: L["type"].__setitem__(0, 99), "type"),
    (lambda L: L["pairs"].__setitem__((0, 1), L["pairs"][0, 0]), "pair"),
    (lambda L: L["tors_bond"].__setitem__((0, 1), L["tors_bond"][0, 0]), "bond"),
    (lambda L: L["mov_atoms"].__setitem__(0, L["tors_bond"][0, 1]), "own bond atom"),
    (lambda L: L["charge"].__setitem__(3, np.nan), "non-finite"),
    (lambda L: L["eps"].__setitem__(0, -1.0), "parameters"),
])
def test_malformed_ligands_are_rejected(pkg, mutate, words):
    lig = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in _base().items()}
    mutate(lig)
    rc, msg = pkg.validate_ligand_torsion_tree(lig)
    assert rc == -1, msg
    assert words in msg, msg


def test_partial_moving_set_is_rejected(pkg):
    # drop one atom from a torsion's moving set: no longer a whole subtree
    lig = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in _base().items()}
    k = int(np.argmax(np.diff(lig["mov_off"])))
    s, e = lig["mov_off"][k], lig["mov_off"][k + 1]
    assert e - s >= 2
    lig["mov_atoms"] = np.delete(lig["mov_atoms"], s)
    lig["mov_off"][k + 1:] -= 1
    rc, msg = pkg.validate_ligand_torsion_tree(lig)
    assert rc == -1, msg
