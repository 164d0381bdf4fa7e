"""ctypes binding of libsphgb.so (include/sphgb.h): argument marshalling only.

Every computation runs in the CUDA library; there is no CPU path.  Loading
fails loudly if the library has not been built (``paper_1404_2303_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsphgb.so")

SPH_OK = 0
NOALLOC_MAX_N = 16384  # SPH_NOALLOC_MAX_N of include/sphgb.h
STATUS_NAMES = {
    0: "SPH_OK", -1: "SPH_ERR_INVALID_ARG", -2: "SPH_ERR_CUDA", -3: "SPH_ERR_OOM",
    -4: "SPH_ERR_H_NOT_CONVERGED", -5: "SPH_ERR_CELL_LIMIT", -6: "SPH_ERR_NOT_BUILT",
    -7: "SPH_ERR_TIMEOUT", -8: "SPH_ERR_CAPACITY",
}


class SphParams(C.Structure):
    _fields_ = [
        ("n_ngb", C.c_float), ("gamma", C.c_float), ("split_count", C.c_int32),
        ("split_frac", C.c_float), ("block_max", C.c_int32), ("max_newton", C.c_int32),
        ("max_rebuild", C.c_int32), ("kahan", C.c_int32), ("morton_bits", C.c_int32),
        ("h_tol", C.c_float), ("warps_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32),
        ("h_est_mode", C.c_int32), ("h_est_factor", C.c_float), ("sweep_cap", C.c_int32),
        ("use_graph", C.c_int32), ("sweep_lists", C.c_int32),
        ("pair_list_cap", C.c_int32), ("list_cap", C.c_int32),
        ("sorted_sweep", C.c_int32),
    ]


class SphStats(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("nbox", C.c_int32), ("ncell", C.c_int32), ("nleaf", C.c_int32),
        ("nblock", C.c_int32), ("nself", C.c_int32), ("npair", C.c_int32), ("ndt", C.c_int64),
        ("max_depth", C.c_int32), ("top_level", C.c_int32 * 8), ("newton_iters", C.c_int32),
        ("rebuilds", C.c_int32), ("density_interactions", C.c_int64), ("force_pairs", C.c_int64),
        ("sorted_entries", C.c_int64), ("sweep_ms", C.c_double * 8),
        ("sweep_launches", C.c_int32 * 8), ("sweep_units", C.c_int64 * 8), ("sweep_candidates", C.c_int64 * 8),
        ("newton_active", C.c_int32 * 32), ("unconverged", C.c_int32), ("sweep_grid", C.c_int32), ("sweep_threads", C.c_int32),
        ("build_ms", C.c_double * 8), ("builds", C.c_int32), ("sweep_gathered", C.c_int64 * 8),
        ("pairs_unlisted", C.c_int32), ("pairs_unlisted_cut", C.c_int32),
    ]


class SphError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")


P = C.c_void_p
SIGNATURES = {
    "sph_default_params": (None, [C.POINTER(SphParams)]),
    "sph_create": (C.c_int, [C.POINTER(SphParams), C.POINTER(C.c_void_p)]),
    "sph_destroy": (None, [P]),
    "sph_build": (C.c_int, [P, C.c_int64, P, C.c_double, P, P]),
    "sph_build_batch": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double), P, P, P]),
    "sph_density_fixed_h": (C.c_int, [P, P, P, P, P, P, P, P, P]),
    "sph_density": (C.c_int, [P, P, P, P, P, C.POINTER(C.c_int32), P]),
    "sph_force": (C.c_int, [P, P, P, P, P, P, P]),
    "sph_force_viscous": (C.c_int, [P, P, P, C.c_float, C.c_float, P, P, P, P, P]),
    "sph_verlet_step": (C.c_int, [P, C.c_int64, P, P, P, P, C.c_double, C.c_double, C.c_float,
                                  C.c_float, C.c_float, C.POINTER(C.c_float),
                                  C.POINTER(C.c_int32), P]),
    "sph_force_adjoint": (C.c_int, [P, P, P, P, P, P, P, P, P, P]),
    "sph_density_adjoint": (C.c_int, [P, P, P, P, P, P, P]),
    "sph_adjoint": (C.c_int, [P, P, P, P, P, P, P, P]),
    "sph_pairs_dump": (C.c_int, [P, C.c_int32, C.c_int64, P, P, C.POINTER(C.c_int64), P]),
    "sph_get_stats": (C.c_int, [P, C.POINTER(SphStats)]),
    "sph_profile": (C.c_int, [P, C.c_int32]),
    "sph_set_sweep_config": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32]),
    "sph_launch_count": (C.c_int64, []),
    "sph_state_generation": (C.c_int64, [P]),
    "sph_density_small_noalloc": (C.c_int, [C.c_int32, P, C.c_double, P, P, C.c_float, C.c_int32,
                                            P, P, C.POINTER(C.c_int32), P]),
    "sph_sync_status": (C.c_int, [P, P]),
    "sph_status_string": (C.c_char_p, [C.c_int]),
}

_lib = None


def load(path: str = LIB_PATH):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1404_2303_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str = "") -> None:
    if code != SPH_OK:
        raise SphError(code, where)
