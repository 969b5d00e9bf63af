"""FP64 CPU oracle (test infrastructure only).

Thin ctypes access to ``adgb_oracle.c``, the plain double-precision
reference for the AutoDock4 scoring function, its gene gradient and the
ADADELTA local search (arxiv 2410.10447, Sec. 2.1).  Only the tests, the
smoke check and the benchmark's CPU-baseline leg use it; the CUDA library
never does.  ``build()`` compiles the C file with gcc next to this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adgb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Receptor(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("n_type_maps", C.c_int), ("spacing", C.c_double),
                ("origin", C.c_double * 3), ("maps", _dp)]


class _Ligand(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("n_tors", C.c_int), ("n_pairs", C.c_int),
                ("n_types", C.c_int), ("type", _ip), ("charge", _dp), ("xyz", _dp),
                ("tors_bond", _ip), ("mov_off", _ip), ("mov_atoms", _ip),
                ("pairs", _ip), ("R", _dp), ("eps", _dp), ("vol", _dp),
                ("solpar", _dp), ("hb_role", _ip), ("hb_R", C.c_double),
                ("hb_eps", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE arithmetic, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_sum_naive.restype = C.c_double
        L.orc_sum_neumaier.restype = C.c_double
        L.orc_sum_naive.argtypes = [_dp, C.c_long, C.c_long]
        L.orc_sum_neumaier.argtypes = [_dp, C.c_long, C.c_long]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(_dp)


def _pi(a):
    return a.ctypes.data_as(_ip)


class Receptor:
    """Receptor grid as the oracle sees it (float32 inputs widened to float64)."""

    def __init__(self, rec: dict):
        self.maps = _d(rec["maps"])
        self.c = _Receptor(int(rec["nx"]), int(rec["ny"]), int(rec["nz"]),
                           int(rec["n_type_maps"]), float(np.float32(rec["spacing"])),
                           (C.c_double * 3)(*[float(v) for v in np.asarray(rec["origin"], np.float32)]),
                           _pd(self.maps))


class Ligand:
    def __init__(self, lig: dict):
        self.arrs = dict(
            type=_i(lig["type"]), charge=_d(lig["charge"]), xyz=_d(lig["xyz"]),
            tors_bond=_i(lig["tors_bond"]).reshape(-1), mov_off=_i(lig["mov_off"]),
            mov_atoms=_i(lig["mov_atoms"]), pairs=_i(lig["pairs"]).reshape(-1),
            R=_d(lig["R"]), eps=_d(lig["eps"]), vol=_d(lig["vol"]),
            solpar=_d(lig["solpar"]), hb_role=_i(lig["hb_role"]))
        if len(self.arrs["mov_atoms"]) == 0:
            self.arrs["mov_atoms"] = np.zeros(1, np.int32)
        if len(self.arrs["pairs"]) == 0:
            self.arrs["pairs"] = np.zeros(2, np.int32)
        a = self.arrs
        self.n_atoms = int(lig["n_atoms"])
        self.n_tors = int(lig["n_tors"])
        self.G = 6 + self.n_tors
        self.c = _Ligand(self.n_atoms, self.n_tors, int(len(lig["pairs"])), int(lig["n_types"]),
                         _pi(a["type"]), _pd(a["charge"]), _pd(a["xyz"]), _pi(a["tors_bond"]),
                         _pi(a["mov_off"]), _pi(a["mov_atoms"]), _pi(a["pairs"]),
                         _pd(a["R"]), _pd(a["eps"]), _pd(a["vol"]), _pd(a["solpar"]),
                         _pi(a["hb_role"]), float(np.float32(lig["hb_R"])),
                         float(np.float32(lig["hb_eps"])))


def _lig(x):
    return x if isinstance(x, Ligand) else Ligand(x)


def _rec(x):
    return x if isinstance(x, Receptor) else Receptor(x)


def pose_coords(lig, genes) -> np.ndarray:
    L = _lig(lig)
    g = _d(genes)
    out = np.zeros((L.n_atoms, 3))
    rc = lib().orc_pose_coords(C.byref(L.c), _pd(g), _pd(out))
    if rc:
        raise ValueError("orc_pose_coords failed (%d)" % rc)
    return out


def energy(rec, lig, xyz):
    """(E_inter, E_intra, dE/dx [N][3]) of explicit coordinates."""
    R, L = _rec(rec), _lig(lig)
    x = _d(xyz)
    g = np.zeros((L.n_atoms, 3))
    ei, ea = C.c_double(), C.c_double()
    lib().orc_energy(C.byref(R.c), C.byref(L.c), _pd(x), C.byref(ei), C.byref(ea), _pd(g))
    return ei.value, ea.value, g


def score(rec, lig, genes):
    """(E, dE/dgenes [G], coords [N][3], dE/dx [N][3]) of one genotype."""
    R, L = _rec(rec), _lig(lig)
    g = _d(genes)
    e = C.c_double()
    gg = np.zeros(L.G)
    x = np.zeros((L.n_atoms, 3))
    ag = np.zeros((L.n_atoms, 3))
    rc = lib().orc_score(C.byref(R.c), C.byref(L.c), _pd(g), C.byref(e), _pd(gg), _pd(x), _pd(ag))
    if rc:
        raise ValueError("orc_score failed (%d)" % rc)
    return e.value, gg, x, ag


def score_magnitude(rec, lig, genes, with_positions=False):
    """[G] magnitude of each gene-gradient component: the chain rule over the
    absolute values of every contribution (sets where a relative tolerance on
    a component is meaningful in floating point).  with_positions: also the
    components' sensitivity to rounding the coordinates (a second [G])."""
    R, L = _rec(rec), _lig(lig)
    g = _d(genes)
    m = np.zeros(L.G)
    pm = np.zeros(L.G)
    rc = lib().orc_score_magnitude(C.byref(R.c), C.byref(L.c), _pd(g), _pd(m), _pd(pm))
    if rc:
        raise ValueError("orc_score_magnitude failed (%d)" % rc)
    return (m, pm) if with_positions else m


def adadelta_step(grad, genes, eg2, ed2, rho=0.8, eps=1e-2):
    """One ADADELTA update; returns new (genes, eg2, ed2)."""
    grad = _d(grad)
    g, a, b = _d(genes).copy(), _d(eg2).copy(), _d(ed2).copy()
    lib().orc_adadelta_step(C.c_int(len(g)), _pd(grad), C.c_double(rho), C.c_double(eps),
                            _pd(g), _pd(a), _pd(b))
    return g, a, b


def local_search(rec, lig, genes, iters, rho=0.8, eps=1e-2, state=None):
    """Returns (best_E, best_genes, final_state [3][G]); resumes from state if given."""
    R, L = _rec(rec), _lig(lig)
    g = _d(genes).copy()
    st = np.zeros((3, L.G)) if state is None else _d(state).reshape(3, L.G).copy()
    be = C.c_double()
    rc = lib().orc_local_search(C.byref(R.c), C.byref(L.c), _pd(g), C.c_int(iters),
                                C.c_double(rho), C.c_double(eps),
                                C.c_int(0 if state is None else 1), _pd(st), C.byref(be))
    if rc:
        raise ValueError("orc_local_search failed (%d)" % rc)
    return be.value, g, st


def local_search_batch(rec, lig, genes, iters, rho=0.8, eps=1e-2, nthreads=0):
    R, L = _rec(rec), _lig(lig)
    g = _d(genes).copy()
    n = g.shape[0]
    be = np.zeros(n)
    rc = lib().orc_local_search_batch(C.byref(R.c), C.byref(L.c), C.c_int(n), _pd(g),
                                      C.c_int(iters), C.c_double(rho), C.c_double(eps),
                                      _pd(be), C.c_int(nthreads))
    if rc:
        raise ValueError("orc_local_search_batch failed")
    return be, g


def score_batch(rec, lig, genes, nthreads=0):
    R, L = _rec(rec), _lig(lig)
    g = _d(genes)
    n = g.shape[0]
    e = np.zeros(n)
    gg = np.zeros((n, L.G))
    rc = lib().orc_score_batch(C.byref(R.c), C.byref(L.c), C.c_int(n), _pd(g), _pd(e),
                               _pd(gg), C.c_int(nthreads))
    if rc:
        raise ValueError("orc_score_batch failed")
    return e, gg


class DockParams(C.Structure):
    _fields_ = [("n_runs", C.c_int), ("pop", C.c_int), ("max_gens", C.c_int),
                ("max_evals", C.c_longlong), ("ls_iters", C.c_int), ("ls_rate", C.c_double),
                ("rho", C.c_double), ("eps", C.c_double), ("p_cross", C.c_double),
                ("p_mut", C.c_double), ("mut_trans", C.c_double), ("mut_angle", C.c_double),
                ("seed", C.c_ulonglong), ("conv_every", C.c_int), ("conv_top", C.c_int),
                ("conv_tol", C.c_double), ("ls_method", C.c_int), ("sw_rho0", C.c_double),
                ("sw_rho_min", C.c_double), ("sw_max_succ", C.c_int), ("sw_max_fail", C.c_int),
                ("sw_angle_scale", C.c_double)]


DOCK_DEFAULTS = dict(n_runs=1, pop=150, max_gens=27, max_evals=2500000, ls_iters=300,
                     ls_rate=1.0, rho=0.8, eps=1e-2, p_cross=0.8, p_mut=0.02, mut_trans=2.0,
                     mut_angle=np.pi / 2, seed=2410, conv_every=0, conv_top=15, conv_tol=0.15,
                     ls_method=0, sw_rho0=1.0, sw_rho_min=0.01, sw_max_succ=4, sw_max_fail=4,
                     sw_angle_scale=1.0)


def dock_params(**kw) -> DockParams:
    d = dict(DOCK_DEFAULTS)
    d.update(kw)
    return DockParams(*[d[f] for f, _ in DockParams._fields_])


def philox(ctr, key):
    """Philox4x32-10 of one 128-bit counter and 64-bit key (4 words)."""
    c = (C.c_uint * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def init_individual(rec, n_tors, seed, run, k):
    R = _rec(rec)
    g = np.zeros(6 + n_tors)
    lib().orc_init_individual(C.byref(R.c), C.c_int(n_tors), C.c_ulonglong(seed), C.c_int(run),
                              C.c_int(k), _pd(g))
    return g


def ga_generation(genes, energies, params: DockParams, run, gen):
    """(new genes [pop][G], local-search flags [pop]) of one GA generation."""
    g = _d(genes)
    pop, G = g.shape
    e = _d(energies)
    out = np.zeros_like(g)
    fl = np.zeros(pop, np.int32)
    lib().orc_ga_generation(C.c_int(G), C.c_int(pop), _pd(g), _pd(e), C.byref(params),
                            C.c_int(run), C.c_int(gen), _pd(out), _pi(fl))
    return out, fl


class SwParams(C.Structure):
    _fields_ = [("max_evals", C.c_int), ("max_succ", C.c_int), ("max_fail", C.c_int),
                ("rho0", C.c_double), ("rho_min", C.c_double), ("angle_scale", C.c_double),
                ("seed", C.c_ulonglong), ("call", C.c_int)]


SW_DEFAULTS = dict(max_evals=300, max_succ=4, max_fail=4, rho0=1.0, rho_min=0.01,
                   angle_scale=1.0, seed=2410, call=0)


def sw_params(**kw) -> SwParams:
    d = dict(SW_DEFAULTS)
    d.update(kw)
    return SwParams(*[d[f] for f, _ in SwParams._fields_])


def sw_normal(seed, genotype, step, call, j) -> float:
    f = lib().orc_sw_normal
    f.restype = C.c_double
    return f(C.c_ulonglong(seed), C.c_uint(genotype), C.c_uint(step), C.c_uint(call), C.c_int(j))


def sw_search(rec, lig, genes, params: SwParams, genotype=0, state=None):
    """Solis-Wets search of one genotype: (energy, genes, evals, state
    [2G+5]); resumes from `state` when given."""
    R, L = _rec(rec), _lig(lig)
    g = _d(genes).copy()
    st = np.zeros(2 * L.G + 5) if state is None else _d(state).copy()
    e = C.c_double()
    ev = C.c_int()
    rc = lib().orc_sw_search(C.byref(R.c), C.byref(L.c), _pd(g), C.byref(params), C.c_int(genotype),
                             C.c_int(0 if state is None else 1), _pd(st), C.byref(e), C.byref(ev))
    if rc:
        raise ValueError("orc_sw_search failed")
    return e.value, g, ev.value, st


def converged(energies, top, tol) -> bool:
    """Early-stopping test: population standard deviation of the `top`
    lowest energies below tol (this project's reading)."""
    e = _d(energies).reshape(-1)
    return bool(lib().orc_converged(C.c_int(len(e)), _pd(e), C.c_int(top), C.c_double(tol)))


def dock(rec, lig, params: DockParams, nthreads=0):
    """(best genes [runs][G], best energies [runs], evaluations [runs])."""
    R, L = _rec(rec), _lig(lig)
    bg = np.zeros((params.n_runs, L.G))
    be = np.zeros(params.n_runs)
    ev = np.zeros(params.n_runs, np.int64)
    rc = lib().orc_dock(C.byref(R.c), C.byref(L.c), C.byref(params), _pd(bg), _pd(be),
                        ev.ctypes.data_as(C.POINTER(C.c_longlong)), C.c_int(nthreads))
    if rc:
        raise ValueError("orc_dock failed")
    return bg, be, ev


def sum_naive(x) -> float:
    x = _d(x).reshape(-1)
    return lib().orc_sum_naive(_pd(x), len(x), 1)


def sum_neumaier(x) -> float:
    x = _d(x).reshape(-1)
    return lib().orc_sum_neumaier(_pd(x), len(x), 1)
