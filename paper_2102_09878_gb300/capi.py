"""ctypes binding of the C ABI in include/spaqr.h (argument marshalling only).

Every numerical step runs in the CUDA library libspaqr_gb300.so; this module
only converts arrays and handles.  There is no CPU fallback: loading fails
loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspaqr_gb300.so")

SPAQR_OK = 0
ERRORS = {
    1: "INVALID_ARG",
    2: "RANK_DEFICIENT",
    3: "CAPACITY",
    4: "NOT_CONVERGED",
    5: "TIMEOUT",
    6: "CUDA",
    7: "OOM",
    8: "NO_DEVICE",
}
SPAQR_ERR_INVALID_ARG, SPAQR_ERR_RANK_DEFICIENT, SPAQR_ERR_CAPACITY, SPAQR_ERR_NOT_CONVERGED = 1, 2, 3, 4
SPAQR_ERR_TIMEOUT, SPAQR_ERR_CUDA, SPAQR_ERR_OOM, SPAQR_ERR_NO_DEVICE = 5, 6, 7, 8
PREC = {"fp64": 0, "mixed": 1}
MODE = {"spaqr": 0, "direct": 1, "diag": 2}
ROWS = {"tree": 0, "maxnorm": 1}


class SpaqrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spaqr error {ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Csr(C.Structure):
    _fields_ = [
        ("m", C.c_int64),
        ("n", C.c_int64),
        ("nnz", C.c_int64),
        ("rowptr", C.c_void_p),
        ("colidx", C.c_void_p),
        ("vals", C.c_void_p),
        ("match", C.c_void_p),
    ]


class GridOrdering(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("depth", C.c_int)]


class Options(C.Structure):
    _fields_ = [
        ("eps", C.c_double),
        ("skip", C.c_int),
        ("precision", C.c_int),
        ("mode", C.c_int),
        ("tol", C.c_double),
        ("maxit", C.c_int),
        ("use_graphs", C.c_int),
        ("verbose", C.c_int),
        ("stream", C.c_void_p),
        ("row_rule", C.c_int),
        ("apply_persistent", C.c_int),
        ("step1_qr_width", C.c_int),
    ]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_resid", C.c_double), ("converged", C.c_int), ("seconds", C.c_double)]


class Stats(C.Structure):
    _fields_ = [
        ("t_analyze", C.c_double),
        ("t_factor", C.c_double),
        ("t_solve", C.c_double),
        ("iters", C.c_int),
        ("nnz_W", C.c_int64),
        ("n_ops", C.c_int64),
        ("n_fronts", C.c_int64),
        ("max_front_rows", C.c_int64),
        ("max_front_cols", C.c_int64),
        ("top_cols", C.c_int64),
        ("top_rows", C.c_int64),
        ("flops_front", C.c_double),
        ("flops_sparsify", C.c_double),
        ("t_phase", C.c_double * 6),
        ("launches", C.c_int64),
        ("syncs", C.c_int64),
        ("t_kernel", C.c_double * 6),
        ("n_kernel", C.c_int64 * 6),
        ("bytes_apply", C.c_double),
        ("flops_qrcp", C.c_double),
        ("bytes_qrcp", C.c_double),
    ]


# every exported symbol and its C signature (restype, argtypes)
SIGNATURES = {
    "spaqr_default_options": (None, [C.POINTER(Options)]),
    "spaqr_analyze": (C.c_int, [C.POINTER(GridOrdering), C.POINTER(C.c_void_p)]),
    "spaqr_analysis_destroy": (None, [C.c_void_p]),
    "spaqr_analyze_matrix": (C.c_int, [C.POINTER(Csr), C.c_int, C.POINTER(C.c_void_p)]),
    "spaqr_match": (C.c_int, [C.POINTER(Csr), C.c_void_p]),
    "spaqr_analysis_stage_size": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "spaqr_analysis_stage_clusters": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "spaqr_factor": (C.c_int, [C.POINTER(Csr), C.c_void_p, C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "spaqr_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(SolveInfo)]),
    "spaqr_solve_csne": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(SolveInfo)]),
    "spaqr_factor_batch": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.POINTER(Options), C.c_void_p]),
    "spaqr_apply_Winv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "spaqr_apply_A": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "spaqr_solve_normal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(SolveInfo)]),
    "spaqr_lstsq_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "spaqr_update_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "spaqr_solve_batch": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "spaqr_solve_normal_batch": (
        C.c_int,
        [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p],
    ),
    "spaqr_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "spaqr_num_ops": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "spaqr_op_info": (
        C.c_int,
        [C.c_void_p, C.c_int64, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    ),
    "spaqr_op_copy": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "spaqr_last_error": (C.c_char_p, []),
    "spaqr_destroy": (None, [C.c_void_p]),
    "spaqr_release_cached_memory": (None, []),
    "spaqr_cached_bytes": (C.c_size_t, []),
    "spaqr_dense_front_qr": (
        C.c_int,
        [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    ),
    "spaqr_dense_front_qr_f32": (
        C.c_int,
        [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    ),
    "spaqr_dense_tc_gemm": (
        C.c_int,
        [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p],
    ),
    "spaqr_autotune": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_char_p, C.POINTER(C.c_double)]),
    "spaqr_load_tuning": (C.c_int, [C.c_char_p]),
    "spaqr_dense_qrcp": (
        C.c_int,
        [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
         C.c_void_p],
    ),
    "spaqr_dense_qrcp_route": (
        C.c_int,
        [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
         C.c_int, C.c_void_p],
    ),
    "spaqr_dense_qrcp_f32": (
        C.c_int,
        [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
         C.c_int, C.c_void_p],
    ),
    "spaqr_debug_set_qrcp_wait": (C.c_int, [C.c_longlong, C.c_int]),
    "spaqr_dense_qrcp_static": (
        C.c_int,
        [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
         C.c_void_p],
    ),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (no fallback: raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the spaQR path has no CPU fallback)"
        )
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != SPAQR_OK:
        raise SpaqrError(rc, load().spaqr_last_error().decode())


def ptr(a) -> int:
    """Address of a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def default_options() -> Options:
    o = Options()
    load().spaqr_default_options(C.byref(o))
    return o
