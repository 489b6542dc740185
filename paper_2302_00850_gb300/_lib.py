"""ctypes binding of libcola (include/cola.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
torch tensors to device pointers and the current CUDA stream to a
cudaStream_t.  It never computes a result itself and has no CPU path: if the
library is missing it raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# COLA_LIB selects another in-tree build, e.g. the bounds-checking debug build
# (python -m paper_2302_00850_gb300.build --bounds writes _build_bounds/libcola.so)
LIB_PATH = os.environ.get("COLA_LIB") or os.path.join(_PKG, "_build", "libcola.so")

COLA_OK = 0
STATUS_NAMES = {
    0: "COLA_OK", -1: "COLA_ERR_ARG", -2: "COLA_ERR_CUDA", -3: "COLA_ERR_NOMEM",
    -4: "COLA_ERR_NOT_CONVERGED", -5: "COLA_ERR_BREAKDOWN", -6: "COLA_ERR_TIMEOUT",
    -7: "COLA_ERR_UNSUPPORTED",
}
F64, F32, F16 = 0, 1, 2
OP_FULL, OP_EO = 0, 1
SYS_NORMAL, SYS_DIRAC = 0, 1


class ColaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("kappa", ctypes.c_double), ("bc", (ctypes.c_double * 2) * 4)]


class GaugeOpts(ctypes.Structure):
    _fields_ = [("prec_mask", ctypes.c_uint), ("recon", ctypes.c_int * 3)]


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("op", ctypes.c_int),
                ("system", ctypes.c_int), ("inner", ctypes.c_int), ("delta", ctypes.c_double),
                ("nrhs", ctypes.c_int), ("use_graph", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int)]


class HmcParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("tau", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("integrator", ctypes.c_int), ("uniform", ctypes.c_double), ("md", SolverParams),
                ("action_tol", ctypes.c_double)]


class HmcInfo(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
                ("accepted", ctypes.c_int), ("plaquette", ctypes.c_double), ("force_evals", ctypes.c_int),
                ("cg_iters", ctypes.c_int), ("seconds", ctypes.c_double)]


class EigParams(ctypes.Structure):
    _fields_ = [("nev", ctypes.c_int), ("nextra", ctypes.c_int), ("op", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("gamma", ctypes.c_double)]


class EigInfo(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("applications", ctypes.c_int), ("max_rel_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_st = ctypes.c_int

# name: (restype, argtypes), in the order of include/cola.h
SIGNATURES = {
    "cola_gauge_create": (_st, [ctypes.POINTER(Lattice), _vp, ctypes.POINTER(GaugeOpts), _vp, ctypes.POINTER(_vp)]),
    "cola_gauge_destroy": (_st, [_vp]),
    "cola_gauge_update": (_st, [_vp, _vp, _vp]),
    "cola_spinor_bytes": (ctypes.c_size_t, [ctypes.POINTER(Lattice), _i, _i]),
    "cola_spinor_pack": (_st, [_vp, _vp, _vp, _i, _i, _vp]),
    "cola_spinor_unpack": (_st, [_vp, _vp, _vp, _i, _i, _vp]),
    "cola_dslash_apply": (_st, [_vp, _vp, _vp, _vp, _d, _d, _i, _i, _i, _i, _vp]),
    "cola_dirac_apply": (_st, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "cola_mdagm_apply": (_st, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "cola_mdagm_apply_noalloc": (_st, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "cola_clover_attach": (_st, [_vp, _d, _vp]),
    "cola_clover_csw": (_d, [_vp]),
    "cola_clover_apply": (_st, [_vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "cola_cg_solve": (_st, [_vp, _vp, _vp, ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo), _vp]),
    "cola_cg_solve_batched": (_st, [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                     ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo), _vp]),
    "cola_multishift_solve": (_st, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _i, _d,
                                     ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo), _vp]),
    "cola_eig_lowest": (_st, [_vp, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(EigParams),
                               ctypes.POINTER(EigInfo), _vp]),
    "cola_fermion_force": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "cola_dirac_link_grad": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "cola_plaquette": (_st, [_vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "cola_gauge_force": (_st, [_vp, _d, _vp, _vp]),
    "cola_link_update": (_st, [_vp, _vp, _vp, _d, _vp]),
    "cola_hmc_trajectory": (_st, [_vp, _vp, _vp, _vp, ctypes.POINTER(HmcParams), ctypes.POINTER(HmcInfo), _vp]),
    "cola_last_error": (ctypes.c_char_p, []),
    "cola_debug_bounds": (_st, [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(_i), _i]),
    "cola_probe_fp64_fma": (_st, [_vp, _i, _i, _i, _vp, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def load(path: str | None = None):
    """Load libcola.so and declare its signatures (raises if it is not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libcola is not built ({p} missing); run __graft_entry__.build() "
                           "or python -m paper_2302_00850_gb300.build")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status: int):
    if status != COLA_OK:
        msg = load().cola_last_error().decode(errors="replace")
        raise ColaError(status, msg)
    return status
