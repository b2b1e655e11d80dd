"""ctypes declarations of the C-ABI in include/pum.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

c_int32, c_int64, c_double, c_void_p = C.c_int32, C.c_int64, C.c_double, C.c_void_p

PUM_OK, PUM_ERR_INVALID_ARG, PUM_ERR_OOM, PUM_ERR_CUDA, PUM_ERR_NOT_SPD = 0, 1, 2, 3, 4
PUM_ERR_BREAKDOWN, PUM_ERR_NOCONV, PUM_ERR_TIMEOUT, PUM_ERR_UNSUPPORTED, PUM_ERR_IO = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_SPD", 5: "BREAKDOWN", 6: "NOCONV",
                7: "TIMEOUT", 8: "UNSUPPORTED", 9: "IO"}
PUM_F64, PUM_F32, PUM_BF16 = 0, 1, 2
PUM_P0_LOWER, PUM_P0_DIAG = 0, 1
PUM_MAT_A, PUM_MAT_P, PUM_MAT_G, PUM_MAT_GT, PUM_MAT_F0, PUM_MAT_G1, PUM_MAT_A1 = range(7)
PUM_TK_COUNT = 7
CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


class BsrView(C.Structure):
    _fields_ = [("n_brows", c_int32), ("n_bcols", c_int32), ("bs", c_int32), ("nnzb", c_int64),
                ("row_ptr", c_void_p), ("col_idx", c_void_p), ("vals", c_void_p), ("on_device", c_int32)]


class BsrHost(C.Structure):
    _fields_ = [("n_brows", c_int32), ("n_bcols", c_int32), ("bs", c_int32), ("nnzb", c_int64),
                ("row_ptr", C.POINTER(c_int32)), ("col_idx", C.POINTER(c_int32)), ("vals", C.POINTER(c_double))]


class Problem(C.Structure):
    _fields_ = [("equation", c_int32), ("p", c_int32), ("finest_m", c_int32), ("n_levels", c_int32),
                ("nitsche_c", c_double * 3), ("quad_pts", c_int32), ("f_coef", c_void_p), ("f_modes", c_int32),
                ("f_decay", c_double), ("aniso", c_double * 3)]


class FsaiParams(C.Structure):
    _fields_ = [("p0", c_int32), ("adaptive", c_int32), ("t_max", c_int32), ("tau", c_double),
                ("nested", c_int32), ("tie_rel", c_double)]


class SmootherParams(C.Structure):
    _fields_ = [("degree_k", c_int32), ("lanczos_its", c_int32), ("lanczos_safety", c_double),
                ("lanczos_seed", C.c_uint64), ("smooth_dt", c_int32), ("g_dt", c_int32), ("mixed_levels", c_int32),
                ("fp32_levels", c_int32), ("smoother", c_int32), ("cycle", c_int32)]


class PcgReport(C.Structure):
    _fields_ = [("rtol", c_double), ("maxit", c_int32), ("flexible", c_int32), ("hist", C.POINTER(c_double)),
                ("iters", c_int32), ("converged", c_int32), ("final_relres", c_double)]


class LevelInfo(C.Structure):
    _fields_ = [("m", c_int32), ("n", c_int32), ("d", c_int32), ("nnzb_A", c_int64), ("nnzb_G", c_int64),
                ("nnzb_GT", c_int64), ("nnzb_P", c_int64), ("nnzb_F0", c_int64), ("nnzb_G1", c_int64),
                ("beta", c_double), ("logdet_S", c_double), ("coarsest", c_int32), ("nested_inner", c_int32),
                ("fused_fsai", c_int32), ("flops_adapt", c_double), ("flops_factor", c_double),
                ("learned", c_int32), ("gate", c_double), ("gg_rows", c_int32), ("gg_parts", c_int32),
                ("gg_ctas", c_int32)]


MLP_FEATURES, MLP_HIDDEN = 12, 64


class Mlp(C.Structure):
    _fields_ = [("w1", C.c_float * (MLP_HIDDEN * MLP_FEATURES)), ("b1", C.c_float * MLP_HIDDEN),
                ("w2", C.c_float * (MLP_HIDDEN * MLP_HIDDEN)), ("b2", C.c_float * MLP_HIDDEN),
                ("w3", C.c_float * MLP_HIDDEN), ("b3", C.c_float)]


class Candidates(C.Structure):
    _fields_ = [("n", c_int64), ("row", c_void_p), ("col", c_void_p), ("x", c_void_p), ("y", c_void_p)]


P = C.POINTER
_SIGNATURES = {
    "pum_create": (c_int32, [P(c_void_p), c_int32, c_void_p]),
    "pum_destroy": (c_int32, [c_void_p]),
    "pum_last_error": (C.c_char_p, [c_void_p]),
    "pum_sync": (c_int32, [c_void_p]),
    "pum_assemble": (c_int32, [c_void_p, P(Problem), P(c_void_p), c_void_p]),
    "pum_hier_from_bsr": (c_int32, [c_void_p, c_int32, P(BsrView), P(BsrView), P(c_void_p)]),
    "bfsai_setup": (c_int32, [c_void_p, c_void_p, P(FsaiParams), P(SmootherParams)]),
    "cheb4_smooth": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_int32]),
    "vcycle_apply": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pcg_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, P(PcgReport)]),
    "bicgstab_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, P(PcgReport)]),
    "pum_convergence_factor": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, P(c_double)]),
    "pum_setup_batch": (c_int32, [P(c_void_p), c_int32, P(c_void_p), c_int32, P(FsaiParams), P(SmootherParams),
                                  P(c_int32)]),
    "pum_solve_batch": (c_int32, [P(c_void_p), c_int32, P(c_void_p), c_int32, P(c_void_p), P(c_void_p),
                                  P(PcgReport), c_int32, P(c_int32)]),
    "pum_residual": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "pum_fsai_apply": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "pum_restrict": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "pum_prolong_add": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "pum_coarse_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pum_hier_levels": (c_int32, [c_void_p, P(c_int32)]),
    "pum_level_info_get": (c_int32, [c_void_p, c_int32, P(LevelInfo)]),
    "pum_hier_export": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, P(BsrHost)]),
    "pum_bsr_free": (None, [P(BsrHost)]),
    "pum_hier_save": (c_int32, [c_void_p, c_void_p, C.c_char_p]),
    "pum_hier_load": (c_int32, [c_void_p, C.c_char_p, P(c_void_p)]),
    "pum_hier_destroy": (c_int32, [c_void_p]),
    "pum_timing_enable": (c_int32, [c_void_p, c_int32]),
    "pum_timing_reset": (c_int32, [c_void_p]),
    "pum_timing_read": (c_int32, [c_void_p, P(c_int64), P(c_double)]),
    "pum_launch_count": (c_int64, [c_void_p]),
    "pum_fsai_apply_noalloc": (c_int32, [c_void_p, P(BsrView), P(BsrView), c_void_p, c_void_p]),
    "pum_fsai_candidates": (c_int32, [c_void_p, c_void_p, c_int32, P(Candidates)]),
    "pum_candidates_free": (None, [P(Candidates)]),
    "pum_candidates_copy": (c_int32, [c_void_p, P(Candidates), c_void_p, c_void_p, c_void_p, c_void_p]),
    "pum_mlp_forward": (c_int32, [c_void_p, P(Mlp), c_void_p, c_int64, c_void_p]),
    "pum_mlp_grad": (c_int32, [c_void_p, P(Mlp), c_void_p, c_void_p, c_int64, P(c_double), P(Mlp)]),
    "pum_mlp_train": (c_int32, [c_void_p, P(Mlp), c_void_p, c_void_p, c_int64, c_int32, c_int32, c_double,
                                C.c_uint64, P(c_double)]),
    "pum_set_pattern_model": (c_int32, [c_void_p, P(Mlp)]),
    "pcg_solve_multi": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, P(PcgReport)]),
    "vcycle_apply_multi": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "pum_solve_batch_multi": (c_int32, [P(c_void_p), c_int32, P(c_void_p), c_int32, c_int32, P(c_void_p),
                                        P(c_void_p), P(PcgReport), P(c_int32)]),
}

_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libpum.so (building it first when missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run paper_2509_06744_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
