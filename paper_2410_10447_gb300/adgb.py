"""ctypes binding of libadgb (include/adgb.h).  Argument marshalling only:
every step of scoring and local search runs in the library's CUDA kernels.

Device-pointer calls take torch CUDA tensors and run on the current torch
stream; host calls take numpy arrays (pinned torch CPU tensors also work).
Loading fails loudly when the library has not been built or cannot load:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

ADGB_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ENOTFOUND", -4: "EDEVICE", -5: "ETIMEOUT",
          -6: "EREJECTED", -7: "ECANCELLED"}
REDUCE_SHFL, REDUCE_MMA_TF32X2, REDUCE_MMA_BF16X3, REDUCE_TCGEN05 = 0, 1, 2, 3
REDUCE4_PAPER_FS = 100
REDUCE4_PAPER_HALF = 101
REDUCE4_TCGEN05_TF32X2 = 102
VARIANTS = {"shfl": REDUCE_SHFL, "mma_tf32x2": REDUCE_MMA_TF32X2, "mma_bf16x3": REDUCE_MMA_BF16X3,
            "tcgen05": REDUCE_TCGEN05}
LS_RESUME = 1

# the C ABI's exported entry points (checked against include/adgb.h by the tests)
EXPORTS = ["adgb_create", "adgb_destroy", "adgb_last_error", "upload_receptor_grids",
           "release_receptor", "upload_ligand_torsion_tree", "release_ligand",
           "validate_ligand_torsion_tree", "ligand_pair_rounds",
           "pose_coords_dev", "pose_coords", "score_poses_dev", "score_poses",
           "local_search_dev", "local_search", "reduce4_bench_dev", "dock_dev", "dock",
           "rescore_fp64_dev", "ga_init_population_dev", "ga_generation_dev", "ga_converged_dev",
           "local_search_sw_dev", "local_search_sw", "alu_bench_dev",
           "dock_noalloc_dev", "batch_create", "batch_autotune", "batch_local_search_dev",
           "batch_release", "serve_start", "serve_stop", "serve_last_error", "serve_stats",
           "dock_submit", "dock_poll", "dock_wait", "dock_result", "dock_cancel", "dock_forget",
           "philox4x32_10_dev", "ls_ablation_dev", "device_status", "l2_bench_dev"]
MAX_GENES = 46


class AdgbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class _Options(C.Structure):
    _fields_ = [("threads_per_pose", C.c_int), ("poses_per_block", C.c_int),
                ("reduce_variant", C.c_int), ("pair_rounds", C.c_int),
                ("genotypes_per_warp", C.c_int)]


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("spacing", C.c_float),
                ("origin", C.c_float * 3), ("n_type_maps", C.c_int)]


_i32p = C.POINTER(C.c_int32)
_f32p = C.POINTER(C.c_float)


class _Ligand(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("n_types", C.c_int), ("n_tors", C.c_int),
                ("n_pairs", C.c_int), ("type", _i32p), ("charge", _f32p), ("xyz", _f32p),
                ("tors_bond", _i32p), ("mov_off", _i32p), ("mov_atoms", _i32p),
                ("pairs", _i32p), ("R", _f32p), ("eps", _f32p), ("vol", _f32p),
                ("solpar", _f32p), ("hb_role", _i32p), ("hb_R", C.c_float),
                ("hb_eps", C.c_float)]


class _DockParams(C.Structure):
    _fields_ = [("n_runs", C.c_int), ("pop", C.c_int), ("max_gens", C.c_int),
                ("max_evals", C.c_longlong), ("ls_iters", C.c_int), ("ls_rate", C.c_float),
                ("rho", C.c_float), ("eps", C.c_float), ("p_cross", C.c_float),
                ("p_mut", C.c_float), ("mut_trans", C.c_float), ("mut_angle", C.c_float),
                ("seed", C.c_ulonglong), ("reduce_variant", C.c_int),
                ("conv_every", C.c_int), ("conv_top", C.c_int), ("conv_tol", C.c_float),
                ("ls_method", C.c_int), ("sw_rho0", C.c_float), ("sw_rho_min", C.c_float),
                ("sw_max_succ", C.c_int), ("sw_max_fail", C.c_int), ("sw_angle_scale", C.c_float)]


DOCK_DEFAULTS = dict(n_runs=20, pop=150, max_gens=27, max_evals=2500000, ls_iters=300,
                     ls_rate=1.0, rho=0.8, eps=1e-2, p_cross=0.8, p_mut=0.02, mut_trans=2.0,
                     mut_angle=float(np.pi / 2), seed=2410, reduce_variant=-1,
                     conv_every=0, conv_top=15, conv_tol=0.15, ls_method=0, sw_rho0=1.0,
                     sw_rho_min=0.01, sw_max_succ=4, sw_max_fail=4, sw_angle_scale=1.0)


def dock_params(**kw) -> _DockParams:
    d = dict(DOCK_DEFAULTS)
    d.update(kw)
    return _DockParams(*[d[f] for f, _ in _DockParams._fields_])


class _ServeOptions(C.Structure):
    _fields_ = [("max_active_jobs", C.c_int), ("mem_budget_bytes", C.c_longlong),
                ("threads_per_pose", C.c_int), ("poses_per_block", C.c_int),
                ("reduce_variant", C.c_int)]


class _JobInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("n_runs", C.c_int), ("n_genes", C.c_int),
                ("generations", C.c_int), ("evals", C.c_longlong), ("submit_s", C.c_double),
                ("start_s", C.c_double), ("finish_s", C.c_double)]


class _ServeStats(C.Structure):
    _fields_ = [("queued", C.c_int), ("active", C.c_int), ("ticks", C.c_longlong),
                ("items_run", C.c_longlong), ("device_bytes_in_use", C.c_longlong),
                ("device_bytes_budget", C.c_longlong), ("busy_s", C.c_double),
                ("uptime_s", C.c_double)]


class _LSParams(C.Structure):
    _fields_ = [("iters", C.c_int), ("rho", C.c_float), ("eps", C.c_float),
                ("reduce_variant", C.c_int), ("flags", C.c_int)]


class _SwParams(C.Structure):
    _fields_ = [("max_evals", C.c_int), ("rho0", C.c_float), ("rho_min", C.c_float),
                ("max_succ", C.c_int), ("max_fail", C.c_int), ("angle_scale", C.c_float),
                ("seed", C.c_ulonglong), ("call", C.c_int), ("reduce_variant", C.c_int),
                ("flags", C.c_int)]


SW_DEFAULTS = dict(max_evals=300, rho0=1.0, rho_min=0.01, max_succ=4, max_fail=4,
                   angle_scale=1.0, seed=2410, call=0, reduce_variant=-1, flags=0)


def sw_params(**kw) -> _SwParams:
    d = dict(SW_DEFAULTS)
    d.update(kw)
    return _SwParams(*[d[f] for f, _ in _SwParams._fields_])


def library_path() -> str:
    return _build.LIB


def load(build: bool = False):
    """Loads libadgb.so (building it first if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libadgb.so is not built; run paper_2410_10447_gb300.build.build()")
    L = C.CDLL(_build.LIB)
    vp = C.c_void_p
    L.adgb_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(_Options)]
    L.adgb_destroy.argtypes = [vp]
    L.adgb_last_error.argtypes = [vp]
    L.adgb_last_error.restype = C.c_char_p
    L.upload_receptor_grids.argtypes = [vp, C.POINTER(_Grid), vp, C.POINTER(C.c_int)]
    L.release_receptor.argtypes = [vp, C.c_int]
    L.upload_ligand_torsion_tree.argtypes = [vp, C.POINTER(_Ligand), C.POINTER(C.c_int)]
    L.release_ligand.argtypes = [vp, C.c_int]
    L.validate_ligand_torsion_tree.argtypes = [C.POINTER(_Ligand), C.c_char_p, C.c_int]
    L.ligand_pair_rounds.argtypes = [C.POINTER(_Ligand), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), vp, C.c_int, vp]
    L.pose_coords_dev.argtypes = [vp, C.c_int, vp, C.c_int, vp, vp]
    L.pose_coords.argtypes = [vp, C.c_int, vp, C.c_int, vp]
    L.score_poses_dev.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp, C.c_int, vp]
    L.score_poses.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp, C.c_int]
    L.local_search_dev.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.POINTER(_LSParams),
                                   vp, vp, vp]
    L.local_search.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.POINTER(_LSParams), vp, vp]
    L.local_search_sw_dev.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.POINTER(_SwParams), vp,
                                      vp, vp, vp]
    L.local_search_sw.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.POINTER(_SwParams), vp, vp,
                                  vp]
    L.reduce4_bench_dev.argtypes = [vp, C.c_int, vp, C.c_int, C.c_int, C.c_int, vp, vp]
    L.dock_dev.argtypes = [vp, C.c_int, C.c_int, C.POINTER(_DockParams), vp, vp, vp, vp]
    L.dock.argtypes = [vp, C.c_int, C.c_int, C.POINTER(_DockParams), vp, vp, vp]
    L.rescore_fp64_dev.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp]
    L.batch_create.argtypes = [vp, C.c_int, vp, vp, vp, C.POINTER(C.c_int)]
    L.batch_autotune.argtypes = [vp, C.c_int, vp, C.c_int, C.POINTER(_Options)]
    L.batch_local_search_dev.argtypes = [vp, C.c_int, vp, C.POINTER(_LSParams), vp, vp]
    L.batch_release.argtypes = [vp, C.c_int]
    L.serve_start.argtypes = [vp, C.POINTER(_ServeOptions), C.POINTER(vp)]
    L.serve_stop.argtypes = [vp]
    L.serve_last_error.argtypes = [vp]
    L.serve_last_error.restype = C.c_char_p
    L.serve_stats.argtypes = [vp, C.POINTER(_ServeStats)]
    L.dock_submit.argtypes = [vp, C.c_int, C.POINTER(_Ligand), C.POINTER(_DockParams),
                              C.POINTER(C.c_longlong)]
    L.dock_poll.argtypes = [vp, C.c_longlong, C.POINTER(_JobInfo)]
    L.dock_wait.argtypes = [vp, C.c_longlong, C.c_int, C.POINTER(_JobInfo)]
    L.dock_result.argtypes = [vp, C.c_longlong, vp, vp, vp]
    L.dock_cancel.argtypes = [vp, C.c_longlong]
    L.dock_forget.argtypes = [vp, C.c_longlong]
    L.dock_noalloc_dev.argtypes = [vp, C.c_int, C.c_int, C.POINTER(_DockParams), vp, vp, vp, vp]
    L.ga_init_population_dev.argtypes = [vp, C.c_int, C.c_int, C.c_ulonglong, C.c_int, C.c_int,
                                         vp, vp]
    L.ga_generation_dev.argtypes = [vp, C.c_int, C.POINTER(_DockParams), C.c_int, vp, vp, vp, vp,
                                    vp]
    L.ga_converged_dev.argtypes = [vp, C.POINTER(_DockParams), vp, vp, vp]
    L.alu_bench_dev.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
    L.philox4x32_10_dev.argtypes = [vp, vp, C.c_int, vp, vp]
    L.device_status.argtypes = [vp]
    L.l2_bench_dev.argtypes = [vp, C.c_int, vp, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_int,
                               vp, vp]
    L.ls_ablation_dev.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.c_int, C.c_int, C.c_int,
                                  vp, vp]
    _lib = L
    return L


def _ptr(x):
    """Raw pointer of a numpy array, a torch tensor, or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check_dev(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)


def _ligand_desc(lig: dict):
    """adgb_ligand_desc over numpy copies of the ligand's arrays; the arrays
    are returned too and must outlive the descriptor."""
    arr = dict(type=_i32(lig["type"]), charge=_f32(lig["charge"]), xyz=_f32(lig["xyz"]),
               tors_bond=_i32(lig["tors_bond"]), mov_off=_i32(lig["mov_off"]),
               mov_atoms=_i32(lig["mov_atoms"]), pairs=_i32(lig["pairs"]),
               R=_f32(lig["R"]), eps=_f32(lig["eps"]), vol=_f32(lig["vol"]),
               solpar=_f32(lig["solpar"]), hb_role=_i32(lig["hb_role"]))
    P = lambda a, t: a.ctypes.data_as(t) if a.size else None
    d = _Ligand(int(lig["n_atoms"]), int(lig["n_types"]), int(lig["n_tors"]),
                int(arr["pairs"].size // 2), P(arr["type"], _i32p), P(arr["charge"], _f32p),
                P(arr["xyz"], _f32p), P(arr["tors_bond"], _i32p), P(arr["mov_off"], _i32p),
                P(arr["mov_atoms"], _i32p), P(arr["pairs"], _i32p), P(arr["R"], _f32p),
                P(arr["eps"], _f32p), P(arr["vol"], _f32p), P(arr["solpar"], _f32p),
                P(arr["hb_role"], _i32p), float(lig["hb_R"]), float(lig["hb_eps"]))
    return d, arr


def validate_ligand_torsion_tree(lig: dict):
    """(status, message) of the library's ligand checks; needs no GPU."""
    d, _keep = _ligand_desc(lig)
    buf = C.create_string_buffer(512)
    rc = load().validate_ligand_torsion_tree(C.byref(d), buf, 512)
    return rc, buf.value.decode()


def ligand_pair_rounds(lig: dict):
    """(n_rounds, lanes, max_degree, words [n_rounds][lanes] uint32, perm
    [n_atoms]) of the pair schedule the library builds; needs no GPU."""
    d, _keep = _ligand_desc(lig)
    nr, nl, md = C.c_int(0), C.c_int(0), C.c_int(0)
    L = load()
    rc = L.ligand_pair_rounds(C.byref(d), C.byref(nr), C.byref(nl), C.byref(md), None, 0, None)
    if rc != ADGB_OK:
        raise AdgbError(rc, "ligand_pair_rounds")
    words = np.zeros((max(nr.value, 1), max(nl.value, 1)), np.uint32)
    perm = np.zeros(int(lig["n_atoms"]), np.int32)
    rc = L.ligand_pair_rounds(C.byref(d), C.byref(nr), C.byref(nl), C.byref(md),
                              words.ctypes.data, words.size, perm.ctypes.data)
    if rc != ADGB_OK:
        raise AdgbError(rc, "ligand_pair_rounds")
    return nr.value, nl.value, md.value, words[:nr.value], perm


class Context:
    """One adgb context on one CUDA device."""

    def __init__(self, device: int = 0, threads_per_pose: int = 0, poses_per_block: int = 0,
                 reduce_variant: int = REDUCE_SHFL, pair_rounds: int = 0,
                 genotypes_per_warp: int = 0):
        self.lib = load()
        self.h = C.c_void_p()
        opts = _Options(threads_per_pose, poses_per_block, reduce_variant, pair_rounds,
                        genotypes_per_warp)
        rc = self.lib.adgb_create(C.byref(self.h), device, C.byref(opts))
        if rc != ADGB_OK:
            raise AdgbError(rc, "adgb_create(device=%d)" % device)
        self._keep = {}

    def close(self):
        if self.h:
            self.lib.adgb_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != ADGB_OK:
            raise AdgbError(rc, self.lib.adgb_last_error(self.h).decode())

    # ------------------------------------------------------------ uploads
    def upload_receptor_grids(self, rec: dict) -> int:
        g = _Grid(int(rec["nx"]), int(rec["ny"]), int(rec["nz"]), float(rec["spacing"]),
                  (C.c_float * 3)(*[float(v) for v in rec["origin"]]), int(rec["n_type_maps"]))
        maps = _f32(rec["maps"])
        rid = C.c_int()
        self._chk(self.lib.upload_receptor_grids(self.h, C.byref(g), maps.ctypes.data, C.byref(rid)))
        return rid.value

    def release_receptor(self, rid: int):
        self._chk(self.lib.release_receptor(self.h, rid))

    def upload_ligand_torsion_tree(self, lig: dict) -> int:
        d, keep = _ligand_desc(lig)
        lid = C.c_int()
        self._chk(self.lib.upload_ligand_torsion_tree(self.h, C.byref(d), C.byref(lid)))
        self._keep[lid.value] = int(lig["n_tors"])
        return lid.value

    def release_ligand(self, lid: int):
        self._chk(self.lib.release_ligand(self.h, lid))

    # ------------------------------------------------------ device calls
    def pose_coords_dev(self, lid, genes, xyz):
        _check_dev(genes, "genes")
        _check_dev(xyz, "xyz")
        self._chk(self.lib.pose_coords_dev(self.h, lid, _ptr(genes), genes.shape[0], _ptr(xyz),
                                           _stream()))

    def score_poses_dev(self, rid, lid, genes, energy, grad=None, variant=-1):
        _check_dev(genes, "genes")
        _check_dev(energy, "energy")
        if grad is not None:
            _check_dev(grad, "grad")
        self._chk(self.lib.score_poses_dev(self.h, rid, lid, _ptr(genes), genes.shape[0],
                                           _ptr(energy), _ptr(grad), variant, _stream()))

    def local_search_dev(self, rid, lid, genes, best_energy, iters, rho=0.8, eps=1e-2,
                         variant=-1, state=None, resume=False):
        _check_dev(genes, "genes")
        _check_dev(best_energy, "best_energy")
        if state is not None:
            _check_dev(state, "state")
        p = _LSParams(int(iters), float(rho), float(eps), int(variant), LS_RESUME if resume else 0)
        self._chk(self.lib.local_search_dev(self.h, rid, lid, _ptr(genes), genes.shape[0],
                                            C.byref(p), _ptr(best_energy), _ptr(state),
                                            _stream()))

    def ls_ablation_dev(self, rid, lid, genes, best_energy, iters, variant, skip_mask):
        """Measurement aid: the two-genotypes-a-warp local search with the steps
        in skip_mask left out (outputs are not energies)."""
        _check_dev(genes, "genes")
        _check_dev(best_energy, "best_energy")
        self._chk(self.lib.ls_ablation_dev(self.h, rid, lid, _ptr(genes), genes.shape[0],
                                           int(iters), int(variant), int(skip_mask),
                                           _ptr(best_energy), _stream()))

    def device_status(self):
        """Raises AdgbError (EDEVICE) once if a tensor-core completion wait gave
        up on the context's device since the last report (after the context's
        stream and torch's current stream have finished)."""
        import torch
        torch.cuda.current_stream().synchronize()
        self._chk(self.lib.device_status(self.h))

    def reduce4_bench_dev(self, variant, x, threads, reps=1, out=None):
        import torch
        _check_dev(x, "x")
        n_blocks = x.numel() // (4 * threads)
        if out is None:
            out = torch.empty_like(x)
        self._chk(self.lib.reduce4_bench_dev(self.h, variant, _ptr(x), threads, n_blocks, reps,
                                             _ptr(out), _stream()))
        return out

    def dock_dev(self, rid, lid, params, best_genes, best_energy, evals=None):
        self._chk(self.lib.dock_dev(self.h, rid, lid, C.byref(params), _ptr(best_genes),
                                    _ptr(best_energy), _ptr(evals), _stream()))

    def dock_noalloc_dev(self, rid, lid, params, best_genes, best_energy, evals=None):
        """dock_dev with the working set in the library's fixed device array
        (no allocation during the call)."""
        self._chk(self.lib.dock_noalloc_dev(self.h, rid, lid, C.byref(params), _ptr(best_genes),
                                            _ptr(best_energy), _ptr(evals), _stream()))

    def batch_create(self, receptor_ids, ligand_ids, n_poses) -> int:
        r, l, n = _i32(receptor_ids), _i32(ligand_ids), _i32(n_poses)
        bid = C.c_int()
        self._chk(self.lib.batch_create(self.h, len(n), r.ctypes.data, l.ctypes.data, n.ctypes.data,
                                        C.byref(bid)))
        return bid.value

    def batch_autotune(self, bid, genes, iters=20):
        _check_dev(genes, "genes")
        import torch
        torch.cuda.current_stream().synchronize()
        o = _Options()
        self._chk(self.lib.batch_autotune(self.h, bid, _ptr(genes), iters, C.byref(o)))
        return dict(threads_per_pose=o.threads_per_pose, poses_per_block=o.poses_per_block,
                    reduce_variant=o.reduce_variant)

    def batch_local_search_dev(self, bid, genes, best_energy, iters, rho=0.8, eps=1e-2, variant=-1):
        _check_dev(genes, "genes")
        _check_dev(best_energy, "best_energy")
        p = _LSParams(int(iters), float(rho), float(eps), int(variant), 0)
        self._chk(self.lib.batch_local_search_dev(self.h, bid, _ptr(genes), C.byref(p),
                                                  _ptr(best_energy), _stream()))

    def batch_release(self, bid):
        self._chk(self.lib.batch_release(self.h, bid))

    def rescore_fp64_dev(self, rid, lid, genes, energy):
        _check_dev(genes, "genes")
        self._chk(self.lib.rescore_fp64_dev(self.h, rid, lid, _ptr(genes), genes.shape[0],
                                            _ptr(energy), _stream()))

    def ga_init_population_dev(self, rid, lid, seed, n_runs, pop, genes):
        _check_dev(genes, "genes")
        self._chk(self.lib.ga_init_population_dev(self.h, rid, lid, seed, n_runs, pop, _ptr(genes),
                                                  _stream()))

    def ga_generation_dev(self, lid, params, gen, genes, energy, genes_out, iters_out):
        self._chk(self.lib.ga_generation_dev(self.h, lid, C.byref(params), gen, _ptr(genes),
                                             _ptr(energy), _ptr(genes_out), _ptr(iters_out),
                                             _stream()))

    def l2_bench_dev(self, kind, buf, n_blocks, threads, reps, out, cell_float4=20):
        """L2 read probe over float32 buf (kind 0 streaming, 1 the grid's 96-byte
        gathers from cells of cell_float4 float4)."""
        _check_dev(buf, "buf")
        _check_dev(out, "out")
        self._chk(self.lib.l2_bench_dev(self.h, int(kind), _ptr(buf), buf.numel() // 4,
                                        int(cell_float4), int(n_blocks), int(threads), int(reps),
                                        _ptr(out), _stream()))

    def alu_bench_dev(self, kind, n_blocks, threads, reps, out):
        """ALU throughput probe (kind 0 FFMA, 1 ex2.approx, 2 rsqrt.approx, 3 packed FFMA2)."""
        self._chk(self.lib.alu_bench_dev(self.h, kind, n_blocks, threads, reps, _ptr(out), _stream()))

    def philox4x32_10_dev(self, ctr_key, out):
        """Philox4x32-10 words: ctr_key [n][6] (counter 0-3, key 0-1) -> out [n][4],
        both int32/uint32-sized CUDA tensors."""
        import torch
        for t, name in ((ctr_key, "ctr_key"), (out, "out")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32
                    and t.is_contiguous()):
                raise TypeError("%s must be a contiguous int32 CUDA tensor" % name)
        if ctr_key.dim() != 2 or ctr_key.shape[1] != 6 or tuple(out.shape) != (ctr_key.shape[0], 4):
            raise ValueError("ctr_key must be [n][6] and out [n][4]")
        self._chk(self.lib.philox4x32_10_dev(self.h, _ptr(ctr_key), ctr_key.shape[0], _ptr(out),
                                             _stream()))

    def ga_converged_dev(self, params, energy, converged):
        """Early-stopping test of params (conv_top, conv_tol) on energy
        [n_runs * pop] -> converged [n_runs] int32 (1 = converged)."""
        self._chk(self.lib.ga_converged_dev(self.h, C.byref(params), _ptr(energy), _ptr(converged),
                                            _stream()))

    # -------------------------------------------------------- host calls
    def dock(self, rid, lid, params):
        """(best genes [runs][G] float32, FP64-rescored best energies [runs],
        evaluations [runs]) of dock() with host buffers."""
        n = params.n_runs
        bg = np.zeros((n, 6 + self._keep[lid]), np.float32)
        be = np.zeros(n, np.float64)
        ev = np.zeros(n, np.int64)
        self._chk(self.lib.dock(self.h, rid, lid, C.byref(params), bg.ctypes.data, be.ctypes.data,
                                ev.ctypes.data))
        return bg, be, ev
    def pose_coords(self, lid, genes, n_atoms):
        g = _f32(genes)
        out = np.zeros((g.shape[0], n_atoms, 3), np.float32)
        self._chk(self.lib.pose_coords(self.h, lid, g.ctypes.data, g.shape[0], out.ctypes.data))
        return out

    def score_poses(self, rid, lid, genes, with_grad=True, variant=-1):
        g = _f32(genes)
        e = np.zeros(g.shape[0], np.float32)
        gr = np.zeros_like(g) if with_grad else None
        self._chk(self.lib.score_poses(self.h, rid, lid, g.ctypes.data, g.shape[0], e.ctypes.data,
                                       _ptr(gr), variant))
        return e, gr

    def local_search(self, rid, lid, genes, iters, rho=0.8, eps=1e-2, variant=-1, state=None,
                     resume=False, want_state=False):
        """Host-buffer local search; genes are updated in place when they
        are a float32 C-contiguous array, and returned either way."""
        g = genes if (isinstance(genes, np.ndarray) and genes.dtype == np.float32
                      and genes.flags.c_contiguous) else _f32(genes)
        n, G = g.shape
        e = np.zeros(n, np.float32)
        st = None
        if resume or want_state:
            # the C call overwrites the state in place: work on a copy
            st = (np.array(state, dtype=np.float32, order="C", copy=True) if state is not None
                  else np.zeros((n, 3, G), np.float32))
        p = _LSParams(int(iters), float(rho), float(eps), int(variant), LS_RESUME if resume else 0)
        self._chk(self.lib.local_search(self.h, rid, lid, g.ctypes.data, n, C.byref(p), e.ctypes.data,
                                        _ptr(st)))
        return e, g, st

    def local_search_sw_dev(self, rid, lid, genes, energy, params, evals=None, state=None):
        """Solis-Wets search of device genotypes in place (energy-only)."""
        _check_dev(genes, "genes")
        _check_dev(energy, "energy")
        self._chk(self.lib.local_search_sw_dev(self.h, rid, lid, _ptr(genes), genes.shape[0],
                                               C.byref(params), _ptr(energy), _ptr(evals),
                                               _ptr(state), _stream()))

    def local_search_sw(self, rid, lid, genes, params, state=None, want_state=False):
        """Host-buffer Solis-Wets search: (energy [n], genes [n][G], evals [n],
        state [n][2G+5] or None); resumes from `state` when params.flags has
        LS_RESUME."""
        g = _f32(genes).copy()
        n, G = g.shape
        e = np.zeros(n, np.float32)
        ev = np.zeros(n, np.int32)
        st = None
        if (params.flags & LS_RESUME) or want_state:
            st = (np.array(state, dtype=np.float32, order="C", copy=True) if state is not None
                  else np.zeros((n, 2 * G + 5), np.float32))
        self._chk(self.lib.local_search_sw(self.h, rid, lid, g.ctypes.data, n, C.byref(params),
                                           e.ctypes.data, ev.ctypes.data, _ptr(st)))
        return e, g, ev, st

    def local_search_host_ptr(self, rid, lid, genes_ptr, n, iters, best_ptr, rho=0.8, eps=1e-2,
                              variant=-1):
        """Host call on raw host pointers (pinned buffers of the caller)."""
        p = _LSParams(int(iters), float(rho), float(eps), int(variant), 0)
        self._chk(self.lib.local_search(self.h, rid, lid, genes_ptr, n, C.byref(p), best_ptr, None))


JOB_DONE, JOB_QUEUED, JOB_RUNNING = 0, 1, 2


class Server:
    """Continuous-batching docking server on a context's device (serve_start)."""

    def __init__(self, ctx: "Context", max_active_jobs=0, mem_budget_bytes=0, threads_per_pose=0,
                 poses_per_block=0, reduce_variant=-1):
        self.ctx, self.lib = ctx, ctx.lib
        self.h = C.c_void_p()
        o = _ServeOptions(max_active_jobs, mem_budget_bytes, threads_per_pose, poses_per_block,
                          reduce_variant)
        rc = self.lib.serve_start(ctx.h, C.byref(o), C.byref(self.h))
        if rc != ADGB_OK:
            raise AdgbError(rc, "serve_start")
        self._genes = {}

    def _chk(self, rc):
        if rc != ADGB_OK:
            raise AdgbError(rc, self.lib.serve_last_error(self.h).decode())

    def submit(self, rid, lig: dict, params) -> int:
        d, keep = _ligand_desc(lig)
        jid = C.c_longlong()
        self._chk(self.lib.dock_submit(self.h, rid, C.byref(d), C.byref(params), C.byref(jid)))
        self._genes[jid.value] = (params.n_runs, 6 + int(lig["n_tors"]))
        return jid.value

    @staticmethod
    def _info(i):
        return dict(status=i.status, n_runs=i.n_runs, n_genes=i.n_genes,
                    generations=i.generations, evals=i.evals, submit_s=i.submit_s,
                    start_s=i.start_s, finish_s=i.finish_s)

    def poll(self, jid):
        i = _JobInfo()
        self._chk(self.lib.dock_poll(self.h, jid, C.byref(i)))
        return self._info(i)

    def wait(self, jid, timeout_ms=-1):
        """Job info once it has finished; None on timeout."""
        i = _JobInfo()
        rc = self.lib.dock_wait(self.h, jid, int(timeout_ms), C.byref(i))
        if rc == -5:
            return None
        self._chk(rc)
        return self._info(i)

    def result(self, jid):
        runs, G = self._genes[jid]
        g = np.zeros((runs, G), np.float32)
        e = np.zeros(runs, np.float64)
        v = np.zeros(runs, np.int64)
        rc = self.lib.dock_result(self.h, jid, g.ctypes.data, e.ctypes.data, v.ctypes.data)
        if rc != ADGB_OK:
            raise AdgbError(rc, "dock_result(job %d)" % jid)
        return g, e, v

    def cancel(self, jid):
        self._chk(self.lib.dock_cancel(self.h, jid))

    def forget(self, jid):
        self._chk(self.lib.dock_forget(self.h, jid))

    def stats(self):
        st = _ServeStats()
        self._chk(self.lib.serve_stats(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServeStats._fields_}

    def stop(self):
        if self.h:
            self.lib.serve_stop(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
