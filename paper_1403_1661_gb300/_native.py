"""ctypes binding of libswe_gb300.so (argument marshalling only).

Every function declared in include/swe.h is bound here under the same name. The
library is the in-tree build (paper_1403_1661_gb300/_build/libswe_gb300.so); if it
is missing, loading fails with an ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import platform

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", platform.machine(), "libswe_gb300.so")

SWE_OK = 0
SWE_EINVAL = -1
SWE_ENOMEM = -2
SWE_ECUDA = -3
SWE_ENAN = -4
SWE_ETIMEOUT = -5
SWE_EUNSUPPORTED = -6

SWE_FP64 = 0
SWE_FP32 = 1
SWE_FP32_TC = 2

SWE_SCHEME_CUBATURE = 0
SWE_SCHEME_COLLOCATION = 1
SWE_SCHEME_CUBATURE_2N = 2

SWE_RHS_FUSED = 0
SWE_RHS_FUSED_SIMT = 1
SWE_RHS_GLOBAL_OPS = 2
SWE_RHS_SPLIT = 3
SWE_LIM_PP = 1
SWE_LIM_TVB = 2


class swe_params(C.Structure):
    _fields_ = [("g", C.c_double), ("h0", C.c_double), ("eps", C.c_double), ("tvb_M", C.c_double),
                ("tvb_nu", C.c_double), ("cfl", C.c_double), ("N", C.c_int32),
                ("nlevels_max", C.c_int32), ("precision", C.c_int32), ("limiter_mask", C.c_int32),
                ("dry_mode", C.c_int32), ("scheme", C.c_int32), ("compensated", C.c_int32)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_vp = C.c_void_p

# name: (restype, argtypes)
SIGNATURES = {
    "swe_version": (C.c_int, []),
    "swe_strerror": (C.c_char_p, [C.c_int]),
    "swe_last_error": (C.c_char_p, []),
    "swe_ref_sizes": (C.c_int, [C.c_int32, _ip, _ip, _ip]),
    "swe_ref_nodes": (C.c_int, [C.c_int32, _dp, _dp]),
    "swe_ref_operator": (C.c_int, [C.c_int32, C.c_int32, _dp, C.c_size_t]),
    "swe_mesh_create": (C.c_int, [_dp, _dp, C.c_int32, _ip, C.c_int32, C.POINTER(_vp)]),
    "swe_mesh_destroy": (None, [_vp]),
    "swe_mesh_num_elements": (C.c_int, [_vp, _ip]),
    "swe_mesh_connectivity": (C.c_int, [_vp, _ip, _ip]),
    "swe_mesh_node_coords": (C.c_int, [_vp, C.c_int32, _dp, _dp]),
    "swe_mesh_levels": (C.c_int, [_vp, C.c_int32, _dp, _dp, _dp, C.c_double, C.c_double, C.c_int32,
                                  _ip, _dp]),
    "swe_regroup_rule": (C.c_int, [_dp, _ip, C.c_int32, C.c_double, C.c_int64, C.c_int32, _ip, _dp]),
    "swe_workspace_bytes": (C.c_int, [_vp, C.POINTER(swe_params), C.POINTER(C.c_size_t)]),
    "swe_solver_create": (C.c_int, [_vp, C.POINTER(swe_params), _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "swe_solver_destroy": (None, [_vp]),
    "swe_stream_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "swe_stream_destroy": (C.c_int, [_vp]),
    "swe_set_bathymetry": (C.c_int, [_vp, _dp]),
    "swe_set_state": (C.c_int, [_vp, _dp, _dp, _dp]),
    "swe_setup_levels": (C.c_int, [_vp, _ip, _dp]),
    "swe_set_levels": (C.c_int, [_vp, _ip, C.c_double]),
    "swe_regroup": (C.c_int, [_vp, _ip, _ip, _dp]),
    "swe_rhs": (C.c_int, [_vp, _vp]),
    "swe_set_farfield": (C.c_int, [_vp, C.c_int32, C.c_double, C.c_double, C.c_double]),
    "swe_set_open_faces": (C.c_int, [_vp, C.c_void_p]),
    "swe_rhs_scratch_bytes": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_size_t)]),
    "swe_rhs_variant": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_size_t]),
    "swe_substep": (C.c_int, [_vp, C.c_int32]),
    "swe_step": (C.c_int, [_vp, C.c_int32]),
    "swe_limit": (C.c_int, [_vp, C.c_int32]),
    "swe_get_state": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "swe_stats": (C.c_int, [_vp, _dp, _dp, _dp, _i64p]),
    "swe_full_state_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "swe_get_full_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "swe_set_full_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "swe_level_info": (C.c_int, [_vp, _ip, _ip, _dp]),
    "swe_kernel_launches": (C.c_int, [_vp, _i64p]),
    "swe_profile_substeps": (C.c_int, [_vp, C.c_int32, _dp]),
    "swe_batch_workspace_bytes": (C.c_int, [C.POINTER(_vp), C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    "swe_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int32, C.c_int32, _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "swe_batch_step": (C.c_int, [_vp, _ip, _ip]),
    "swe_batch_set_wait_limit": (C.c_int, [_vp, C.c_double]),
    "swe_batch_hold": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "swe_batch_launches": (C.c_int, [_vp, _i64p]),
    "swe_batch_destroy": (None, [_vp]),
    "swe_set_launch_config": (C.c_int, [_vp, C.c_int32]),
    "swe_set_tc_warps": (C.c_int, [_vp, C.c_int32]),
    "swe_mass_hmin_static": (C.c_int, [C.c_int32, C.c_int32, _vp, _vp, _vp, _vp]),
    "swe_tc_projection_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
}

_lib = None


class SWEError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = ""
        if _lib is not None:
            msg = (_lib.swe_last_error() or b"").decode(errors="replace")
            name = (_lib.swe_strerror(code) or b"").decode()
        else:
            name = str(code)
        super().__init__(f"{where}: {name} ({code}): {msg}")


def lib():
    """Load (once) and return the native library with typed signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"native library not built: {LIB_PATH} (run paper_1403_1661_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc, where):
    if rc != SWE_OK:
        raise SWEError(rc, where)
    return rc


def dptr(a):
    """ctypes double* of a C-contiguous float64 numpy array."""
    return a.ctypes.data_as(_dp)


def iptr(a):
    return a.ctypes.data_as(_ip)
