"""GB300-native AutoDock4 scoring, gradient and ADADELTA local search
(arxiv 2410.10447).  The compute path is libadgb.so (hand-written sm_103a
CUDA kernels behind a C ABI, include/adgb.h); this package is its ctypes
binding and build step.
"""
from .adgb import (  # noqa: F401
    EXPORTS, LS_RESUME, REDUCE4_PAPER_FS, REDUCE4_PAPER_HALF, REDUCE4_TCGEN05_TF32X2, REDUCE_MMA_BF16X3, REDUCE_MMA_TF32X2, REDUCE_SHFL,
    REDUCE_TCGEN05,
    VARIANTS, AdgbError, Context, Server, library_path, load, validate_ligand_torsion_tree,
    ligand_pair_rounds,
)
from .build import build  # noqa: F401
