"""Seeded synthetic inputs for the AutoDock4 scoring / ADADELTA hot path.

This package is the only code shared by the FP64 oracle tests and the CUDA
path: it draws receptor grid maps, ligands (bond tree, torsion tree, pair
list, force-field type parameters) and random poses.  It contains none of the
method's arithmetic (no energies, no gradients, no coordinate transforms of
poses); everything it returns is an input to the scoring function.
"""
from .generate import (  # noqa: F401
    WORKLOADS,
    make_ligand,
    make_poses,
    make_receptor,
    make_uneven_batch,
    workload,
)
