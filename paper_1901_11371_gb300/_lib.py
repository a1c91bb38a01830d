"""ctypes loader for libhb.so (the C ABI declared in include/hb.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Loading fails loudly if the shared object is missing.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhb.so")

HB_OK, HB_EINVAL, HB_ENOMEM, HB_ECUDA, HB_ENOCONV, HB_ETIMEOUT, HB_ENAN, HB_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
HB_STRIP, HB_SPIRAL, HB_ARC, HB_PARALLEL_STRIPS, HB_POLYLINE = 0, 1, 2, 3, 4
HB_OPT_LEAF_LU = 1
HB_OPT_SWEEP_WINDOW_MIN = 2
HB_C128, HB_C64, HB_SPLIT_BF16 = 0, 1, 2
HB_OP_N, HB_OP_H = 0, 1
ERR_NAMES = {0: "HB_OK", -1: "HB_EINVAL", -2: "HB_ENOMEM", -3: "HB_ECUDA", -4: "HB_ENOCONV", -5: "HB_ETIMEOUT",
             -6: "HB_ENAN", -7: "HB_EUNSUPPORTED"}


class HBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class FactorStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("leaf", C.c_int64), ("depth", C.c_int32), ("form", C.c_int32),
                ("n_butterflies", C.c_int64), ("scale", C.c_double), ("eps", C.c_double),
                ("kmax", C.c_int32), ("sweep_leaf", C.c_int32), ("kavg", C.c_double),
                ("kmax_depth", C.c_int32 * 32), ("kavg_depth", C.c_double * 32),
                ("nnz_leaf", C.c_int64), ("nnz_butterfly", C.c_int64), ("nnz_lu_leaf", C.c_int64),
                ("index_bytes", C.c_int64), ("device_bytes", C.c_int64), ("apply_bytes", C.c_int64),
                ("lower_bytes", C.c_int64), ("upper_bytes", C.c_int64), ("rebuilt_blocks", C.c_int32),
                ("pad1", C.c_int32), ("build_seconds", C.c_double)]


class GmresInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("ir_steps", C.c_int32), ("converged", C.c_int32),
                ("true_rel_res", C.c_double), ("precond_rel_res", C.c_double), ("seconds", C.c_double),
                ("iters_per_rhs", C.POINTER(C.c_int32)), ("res_per_rhs", C.POINTER(C.c_double)),
                ("graph_launches", C.c_int32), ("pad", C.c_int32)]


_VP, _I64, _INT, _DBL = C.c_void_p, C.c_int64, C.c_int, C.c_double

SIGNATURES = {
    "hb_geometry": (_INT, [_INT, C.POINTER(C.c_double), _INT, _I64, C.POINTER(_VP)]),
    "hb_geometry_segments": (_INT, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hb_geometry_polyline": (_INT, [C.POINTER(C.c_double), C.POINTER(C.c_int64), _INT, _I64, C.POINTER(_VP)]),
    "hb_geometry_size": (_I64, [_VP]),
    "hb_geometry_destroy": (None, [_VP]),
    "hb_factor": (_INT, [_VP, _DBL, _DBL, _DBL, _I64, _DBL, _INT, C.c_uint64, _VP, C.POINTER(_VP)]),
    "hb_factor_host": (_INT, [_VP, _DBL, _DBL, _DBL, _I64, _DBL, C.c_uint64, C.POINTER(_VP)]),
    "hb_factor_ex": (_INT, [_VP, _DBL, _DBL, _DBL, _I64, _DBL, _INT, C.c_uint64, _INT, _VP, C.POINTER(_VP)]),
    "hb_factor_host_ex": (_INT, [_VP, _DBL, _DBL, _DBL, _I64, _DBL, C.c_uint64, _INT, C.POINTER(_VP)]),
    "hb_factor_info": (_INT, [_VP, C.POINTER(FactorStats)]),
    "hb_factor_destroy": (None, [_VP]),
    "hb_tree": (_INT, [_VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "hb_apply": (_INT, [_VP, _INT, _VP, _VP, _I64, _I64, _VP]),
    "hb_apply_adjoint": (_INT, [_VP, _VP, _VP, _I64, _I64, _VP]),
    "hb_apply_noalloc": (_INT, [_VP, _INT, _VP, _VP, _I64, _I64, _VP]),
    "hb_precond_solve": (_INT, [_VP, _INT, _VP, _VP, _I64, _I64, _VP]),
    "hb_lower_solve": (_INT, [_VP, _INT, _VP, _VP, _I64, _I64, _VP]),
    "hb_upper_solve": (_INT, [_VP, _INT, _VP, _VP, _I64, _I64, _VP]),
    "hb_residual": (_INT, [_VP, _INT, _VP, _VP, _VP, _I64, _I64, _VP]),
    "hb_gmres": (_INT, [_VP, _INT, _VP, _VP, _I64, _I64, _INT, _DBL, _INT, C.POINTER(GmresInfo), _VP]),
    "hb_tfqmr": (_INT, [_VP, _INT, _VP, _VP, _VP, _I64, _I64, _DBL, _INT, C.POINTER(GmresInfo), _VP]),
    "hb_rhs_plane_wave": (_INT, [_VP, C.POINTER(C.c_double), _I64, _VP, _I64, _VP]),
    "hb_far_field": (_INT, [_VP, _VP, _I64, _I64, C.POINTER(C.c_double), _I64, _VP, _VP]),
    "hb_far_field_adjoint": (_INT, [_VP, _VP, _I64, C.POINTER(C.c_double), _I64, _VP, _I64, _VP]),
    "hb_monostatic": (_INT, [_VP, _VP, _I64, _I64, C.POINTER(C.c_double), _VP, _VP]),
    "hb_set_sweep_grid_min": (_INT, [_VP, _INT]),
    "hb_set_sweep_kernel": (_INT, [_VP, _INT]),
    "hb_set_wait_limit": (_INT, [_VP, C.c_longlong]),
    "hb_set_gmres_graph": (_INT, [_VP, _INT]),
    "hb_autotune": (_INT, [_VP, _I64, _VP, C.POINTER(C.c_int)]),
    "hb_autotune_times": (_INT, [_VP, _I64, C.POINTER(C.c_float), C.POINTER(C.c_int), C.c_int]),
    "hb_status": (_INT, [_VP, _VP]),
    "hb_profile": (_INT, [_VP, _INT]),
    "hb_profile_read": (_INT, [_VP, _INT, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "hb_host_apply": (_INT, [_VP, _INT, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hb_host_sweep": (_INT, [_VP, _INT, C.POINTER(C.c_double)]),
    "hb_host_sweep_sched": (_INT, [_VP, _INT, _INT, _INT, C.POINTER(C.c_double)]),
    "hb_host_apply_plan": (_INT, [_VP, _INT, _INT, _INT, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hb_host_tc_apply": (_INT, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hb_last_error": (C.c_char_p, []),
    "hb_version": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libhb.so once; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhb.so not found at {path}; build it with `python -m paper_1901_11371_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int):
    if code != HB_OK:
        raise HBError(code, load().hb_last_error().decode(errors="replace"))
    return code
