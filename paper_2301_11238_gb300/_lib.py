"""ctypes declarations of the C ABI in include/dg_swe.h (argument marshalling only)."""
import ctypes as C
import os

from . import build as _build

(DG_OK, DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_WORKSPACE, DG_ERR_NONFINITE, DG_ERR_NEWTON, DG_ERR_UNSUPPORTED,
 DG_ERR_TIMEOUT) = range(8)
STATUS_NAMES = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_CUDA", 3: "DG_ERR_WORKSPACE",
                4: "DG_ERR_NONFINITE", 5: "DG_ERR_NEWTON", 6: "DG_ERR_UNSUPPORTED", 7: "DG_ERR_TIMEOUT"}
MAX_BC = 8


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int64), ("coords", C.c_void_p),
                ("n_elements", C.c_int64), ("elem_vertices", C.c_void_p), ("face_bc", C.c_void_p),
                ("bed", C.c_void_p)]


class BC(C.Structure):
    _fields_ = [("mode", C.c_int32 * 7), ("value", C.c_double * 7)]


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("rho", C.c_double), ("alpha", C.c_double), ("eta", C.c_double),
                ("sigma0", C.c_double), ("gamma", C.c_double), ("beta", C.c_double),
                ("pap_m", C.c_double), ("h_floor", C.c_double), ("cfl", C.c_double),
                ("precision", C.c_int32), ("n_bc", C.c_int32), ("bc", BC * MAX_BC),
                ("positivity", C.c_int32), ("flow_index", C.c_double), ("rate_floor", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("t", C.c_double), ("dt_last", C.c_double),
                ("dt_min", C.c_double), ("dt_max", C.c_double), ("mass", C.c_double),
                ("mass0", C.c_double), ("status", C.c_int32)]


class ImplicitParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("m3", C.c_int32), ("max_it", C.c_int32),
                ("on_fail_continue", C.c_int32), ("rtol", C.c_double), ("atol", C.c_double),
                ("xtol", C.c_double), ("linear_solver", C.c_int32), ("n_gamma", C.c_int32),
                ("gamma0", C.c_double)]


class ImplicitStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("newton_its", C.c_int64), ("failed_steps", C.c_int64),
                ("t", C.c_double), ("last_res", C.c_double), ("last_its", C.c_int32),
                ("status", C.c_int32)]


_SIGS = {
    "dg_swe_init": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.POINTER(Params), C.POINTER(C.c_void_p)]),
    "dg_swe_workspace_size": (C.c_size_t, [C.c_void_p]),
    "dg_swe_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "dg_swe_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_swe_node_coords": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_swe_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "dg_swe_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_swe_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "dg_swe_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_swe_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "dg_swe_run": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.POINTER(Stats)]),
    "dg_swe_sync": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "dg_swe_advance": (C.c_int, [C.c_void_p, C.c_int64]),
    "dg_swe_time_kernels": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "dg_swe_launches_per_step": (C.c_int32, [C.c_void_p]),
    "dg_swe_residual_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_swe_static_scratch_need": (C.c_size_t, [C.c_void_p]),
    "dg_swe_last_error": (C.c_char_p, [C.c_void_p]),
    "dg_swe_destroy": (None, [C.c_void_p]),
}

class NewtonParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("max_newton", C.c_int32), ("rtol", C.c_double), ("atol", C.c_double),
                ("krylov_dim", C.c_int32), ("krylov_rtol", C.c_double), ("on_fail_continue", C.c_int32)]


class NewtonStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("newton_its", C.c_int64), ("krylov_its", C.c_int64),
                ("failed_steps", C.c_int64), ("t", C.c_double), ("last_res", C.c_double),
                ("last_newton", C.c_int32), ("status", C.c_int32)]


_OPTIONAL_SIGS = {
    "dg_newton_init": (C.c_int, [C.c_void_p, C.POINTER(NewtonParams), C.POINTER(C.c_void_p)]),
    "dg_newton_workspace_size": (C.c_size_t, [C.c_void_p]),
    "dg_newton_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "dg_newton_run": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(NewtonStats)]),
    "dg_newton_last_error": (C.c_char_p, [C.c_void_p]),
    "dg_newton_destroy": (None, [C.c_void_p]),
    "dg_implicit_init": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.POINTER(ImplicitParams),
                                   C.POINTER(C.c_void_p)]),
    "dg_implicit_workspace_size": (C.c_size_t, [C.c_void_p]),
    "dg_implicit_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "dg_implicit_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_implicit_node_coords": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_implicit_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_implicit_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "dg_implicit_run": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(ImplicitStats)]),
    "dg_implicit_active_percent": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "dg_implicit_last_error": (C.c_char_p, [C.c_void_p]),
    "dg_implicit_destroy": (None, [C.c_void_p]),
    "dg_batch_init": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.POINTER(C.c_void_p)]),
    "dg_batch_workspace_size": (C.c_size_t, [C.c_void_p]),
    "dg_batch_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "dg_batch_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_batch_set_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "dg_batch_get_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "dg_batch_run": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "dg_batch_advance": (C.c_int, [C.c_void_p, C.c_int64]),
    "dg_batch_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_batch_autotune": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_batch_time_kernels": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "dg_batch_launches_per_step": (C.c_int32, [C.c_void_p]),
    "dg_batch_tiles": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int32)]),
    "dg_batch_set_tiles": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "dg_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "dg_batch_destroy": (None, [C.c_void_p]),
    "dg_batch_set_persistent": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_probe_fma_rate": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "dg_probe_scratch_bytes": (C.c_size_t, []),
}

_LIB = None


def lib(build_if_missing=True):
    """Load libdgswe.so (building it first if needed).  Raises if it cannot
    be built or loaded: there is no fallback path."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run paper_2301_11238_gb300.build.build()")
    L = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    for name, (res, args) in _OPTIONAL_SIGS.items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
    _LIB = L
    return L
