"""dock_noalloc_dev: the docking entry point for callers that must not
allocate device memory during a call (its working set lives in a fixed
device array inside the library).  Its results must equal dock_dev's on the
same inputs, call after call, although every call reuses the same array.
Kept in a file collected last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_dock_matches_dock_dev_on_consecutive_calls():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_10447_gb300 as P
    P.load(build=True)
    w = synth.workload("plain_n16", n_poses=4)
    ctx = P.Context(0)
    rid = ctx.upload_receptor_grids(w["receptor"])
    lid = ctx.upload_ligand_torsion_tree(w["ligand"])
    G = 6 + w["ligand"]["n_tors"]
    runs = 5
    for call, seed in enumerate((17, 18)):
        prm = P.adgb.dock_params(n_runs=runs, pop=40, max_gens=3, ls_iters=25, seed=seed)
        g_ref = torch.empty(runs, G, device="cuda")
        e_ref = torch.empty(runs, dtype=torch.float64, device="cuda")
        v_ref = torch.empty(runs, dtype=torch.int64, device="cuda")
        ctx.dock_dev(rid, lid, prm, g_ref, e_ref, v_ref)
        g = torch.full((runs, G), float("nan"), device="cuda")
        e = torch.full((runs,), float("nan"), dtype=torch.float64, device="cuda")
        v = torch.full((runs,), -1, dtype=torch.int64, device="cuda")
        ctx.dock_noalloc_dev(rid, lid, prm, g, e, v)
        torch.cuda.synchronize()
        # same kernels on the same inputs: results agree within the energy
        # tolerance of the FP64 rescoring and the coordinate tolerance
        assert np.allclose(g.cpu().numpy(), g_ref.cpu().numpy(), rtol=0, atol=1e-5), call
        assert np.allclose(e.cpu().numpy(), e_ref.cpu().numpy(), rtol=1e-9, atol=1e-9), call
        assert np.array_equal(v.cpu().numpy(), v_ref.cpu().numpy()), call
    # a working set beyond the fixed array is refused, not truncated
    big = P.adgb.dock_params(n_runs=1000, pop=1000, max_gens=1, ls_iters=2, seed=1)
    g = torch.empty(1000, G, device="cuda")
    e = torch.empty(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(P.AdgbError) as ei:
        ctx.dock_noalloc_dev(rid, lid, big, g, e)
    assert ei.value.code == -1 and "exceeds" in str(ei.value)
    ctx.close()
