"""ctypes declarations of the libmrcm C ABI (include/mrcm.h).

Loading fails loudly when libmrcm.so has not been built: there is no CPU or
PyTorch fallback for any step of the solve.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrcm.so")

MRCM_OK = 0
STATUS_NAMES = {
    0: "MRCM_OK", 1: "MRCM_ERR_INVALID_ARG", 2: "MRCM_ERR_CUDA", 3: "MRCM_ERR_NOT_SPD",
    4: "MRCM_ERR_NO_CONVERGENCE", 5: "MRCM_ERR_SINGULAR_INTERFACE", 6: "MRCM_ERR_TIMEOUT",
    7: "MRCM_ERR_OOM", 8: "MRCM_ERR_NOT_IMPLEMENTED", 9: "MRCM_ERR_STATE",
}
PRECISIONS = {"fp64": 0, "fp32_ir": 1, "tf32_ir": 2, "learned_pcg": 3}


class mrcm_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
        ("n_cuts", C.c_int * 3),
        ("cuts", C.POINTER(C.c_int) * 3),
        ("patch", (C.c_int * 2) * 3),
        ("beta_mode", C.c_int),
        ("alpha", C.c_double), ("beta_const", C.c_double),
        ("bc_type", (C.c_int * 2) * 3),
        ("bc_value", (C.c_double * 2) * 3),
        ("precision", C.c_int),
        ("ir_max_sweeps", C.c_int),
        ("ir_tol", C.c_double),
        ("wave_bytes", C.c_size_t),
        ("tune_cache", C.c_char_p),
        ("interface_refine", C.c_int),
        ("fallback_cap", C.c_int),
    ]


class mrcm_sizes(C.Structure):
    _fields_ = [
        ("n_cells", C.c_longlong), ("n_sub", C.c_int), ("n_basis", C.c_int),
        ("n_faces", C.c_longlong), ("max_rhs", C.c_int), ("total_rhs", C.c_longlong),
        ("nnz_interface", C.c_longlong), ("n_fronts", C.c_int), ("max_front", C.c_int),
        ("front_flops", C.c_double), ("local_factor_flops", C.c_double),
        ("local_solve_flops", C.c_double), ("max_block", C.c_int),
        ("mbf_entries", C.c_longlong), ("ldl_flops", C.c_double), ("ldl_update_flops", C.c_double),
        ("n_waves", C.c_int),
        ("max_front_ne", C.c_int),
        ("max_front_nb", C.c_int),
        ("ldl_update_tensor_flops", C.c_double),
    ]


# name -> (restype, argtypes)
SIGNATURES = {
    "mrcm_setup": (C.c_int, [C.POINTER(mrcm_config), C.POINTER(C.c_void_p)]),
    "mrcm_query_workspace": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "mrcm_query_sizes": (C.c_int, [C.c_void_p, C.POINTER(mrcm_sizes)]),
    "mrcm_query_local_ldl": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mrcm_query_basis": (C.c_int, [C.c_void_p, C.c_int] + [C.POINTER(C.c_int)] * 4),
    "mrcm_factor_local": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "mrcm_solve_mbf": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrcm_assemble_interface": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrcm_solve_interface": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrcm_reconstruct": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6),
    "mrcm_postprocess_velocity": (C.c_int, [C.c_void_p] * 6),
    "mrcm_transport_query": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "mrcm_impes": (C.c_int, [C.c_void_p] * 4 + [C.c_double] * 3 + [C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                                                   C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p]),
    "mrcm_read_status": (C.c_int, [C.c_void_p, C.c_void_p] + [C.POINTER(C.c_int)] * 4),
    "mrcm_read_fallback": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mrcm_read_work": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_longlong)]),
    "mrcm_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t]),
    "mrcm_solve": (C.c_int, [C.c_void_p] + [C.c_void_p] * 7 + [C.c_size_t, C.c_void_p, C.c_int]),
    "mrcm_solve_host": (C.c_int, [C.c_void_p] + [C.c_void_p] * 7 + [C.c_size_t, C.c_void_p, C.c_int]),
    "mrcm_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mrcm_query_tuning": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int)] * 4),
    "mrcm_read_tuning_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                         C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int),
                                         C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "mrcm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "mrcm_profile_report": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t, C.POINTER(C.c_longlong)]),
    "mrcm_box_solve_noalloc": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int)]
                               + [C.c_void_p] * 6 + [C.c_void_p, C.c_void_p]),
    "mrcm_net_create": (C.c_int, [C.c_int] * 6 + [C.POINTER(C.c_void_p)]),
    "mrcm_net_query": (C.c_int, [C.c_void_p, C.c_int] + [C.POINTER(C.c_size_t)] * 3),
    "mrcm_net_init": (C.c_int, [C.c_void_p, C.c_void_p, C.c_ulonglong, C.c_void_p]),
    "mrcm_net_sync_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrcm_net_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mrcm_net_gradient": (C.c_int, [C.c_void_p] * 5 + [C.c_int] + [C.c_void_p] * 4),
    "mrcm_net_train_step": (C.c_int, [C.c_void_p] * 5 + [C.c_int, C.c_float, C.c_int] + [C.c_void_p] * 3),
    "mrcm_net_flux_weights": (C.c_int, [C.c_void_p] * 4 + [C.c_int, C.c_void_p]),
    "mrcm_net_destroy": (None, [C.c_void_p]),
    "mrcm_net_samples": (C.c_int, [C.c_void_p] * 5 + [C.c_int, C.POINTER(C.c_int), C.c_void_p]),
    "mrcm_solve_mbf_learned": (C.c_int, [C.c_void_p] * 3 + [C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                                               C.c_void_p]),
    "mrcm_read_cg_iterations": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_longlong)]),
    "mrcm_pcg_mbf": (C.c_int, [C.c_void_p] * 4 + [C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "mrcm_measure_fp64_peak": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mrcm_destroy": (None, [C.c_void_p]),
    "mrcm_last_error": (C.c_char_p, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libmrcm.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libmrcm.so not found at {path}: build it with "
            "`python -m paper_2103_08513_gb300.build` (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MRCMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code, handle=None):
    if code != MRCM_OK:
        msg = load().mrcm_last_error(handle)
        raise MRCMError(code, msg.decode() if msg else "")
