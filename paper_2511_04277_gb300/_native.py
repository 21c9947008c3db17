"""ctypes declarations of the C ABI in include/radgeb.h.

Loading fails loudly (ImportError) when libradgeb.so has not been built: there is
no fallback implementation of any step.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libradgeb.so")

P = ctypes.c_void_p
i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
sz = ctypes.c_size_t
PP = ctypes.POINTER(ctypes.c_void_p)

RG_OK = 0
STATUS = {0: "RG_OK", -1: "RG_ERR_ARG", -2: "RG_ERR_CUDA", -3: "RG_ERR_OOM", -4: "RG_ERR_NOT_CONVERGED",
          -5: "RG_ERR_STACK", -6: "RG_ERR_NUMERIC", -7: "RG_ERR_UNSUPPORTED"}
PREC = {"bf16": 1, "fp16": 2}
WS_KIND = {"gebhart": 1, "gebhart_adjoint": 2, "gebhart_adjoint_factored": 3, "temperatures": 4,
           "temperatures_sets": 5, "enforce_lsq": 6}
KAPPA = {"triangulation": 1, "fractional_variance": 2}


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_faces", i32), ("n_tris", i64), ("bvh_nodes", i32), ("bvh_depth", i32), ("lift", ctypes.c_float),
                ("sah_visits", ctypes.c_float), ("refill", i32)]


# name -> (restype, argtypes), in the order of include/radgeb.h
SIGNATURES = {
    "rg_create": (i32, [PP, ctypes.c_int]),
    "rg_destroy": (None, [P]),
    "rg_last_error": (ctypes.c_char_p, [P]),
    "rg_version": (ctypes.c_char_p, []),
    "rg_launch_count": (i32, [P, ctypes.POINTER(i64)]),
    "rg_workspace_bytes": (i32, [P, ctypes.POINTER(sz)]),
    "rg_solver_workspace": (i32, [i32, i32, i32, ctypes.POINTER(sz)]),
    "rg_gebhart_workspace": (i32, [i32, i32, i32, i32, ctypes.POINTER(sz)]),
    "rg_kernel_timer": (i32, [P, i32]),
    "rg_kernel_timer_read": (i32, [P, i32, ctypes.POINTER(i64), ctypes.POINTER(f64), ctypes.POINTER(f64),
                                    ctypes.POINTER(f64)]),
    "rg_mesh_create": (i32, [P, P, i64, P, i64, P, i32, i32, PP]),
    "rg_mesh_create_gpu_bvh": (i32, [P, P, i64, P, i64, P, i32, i32, PP]),
    "rg_mesh_get_bvh": (i32, [P, P, P]),
    "rg_mesh_destroy": (i32, [P]),
    "rg_mesh_get_info": (i32, [P, ctypes.POINTER(MeshInfo)]),
    "rg_face_areas": (i32, [P, P]),
    "rg_trace": (i32, [P, P, P, u64, u64, i32, P, P]),
    "rg_trace_stats": (i32, [P, P, P, u64, u64, i32, P, P, P]),
    "rg_trace_sided": (i32, [P, P, P, u64, u64, i32, P, P]),
    "rg_counts_to_F": (i32, [P, i32, P, P, P, P]),
    "rg_enforce_iterative": (i32, [P, i32, P, P, f64, i32, P, P]),
    "rg_enforce_iterative_noalloc": (i32, [i32, P, P, f64, i32, P, P]),
    "rg_enforce_iterative_kappa": (i32, [P, i32, P, P, P, f64, i32, P, P]),
    "rg_kappa": (i32, [P, i32, i32, P, P, P, f64, P, P]),
    "rg_trace_reflect": (i32, [P, P, P, P, P, i32, u64, u64, i32, P, P, P]),
    "rg_debug_mbarrier_timeout": (i32, [P, f64, P]),
    "rg_debug_barrier_timeout": (i32, [P, f64, P]),
    "rg_enforce_lsq": (i32, [P, i32, P, P, i32, i32, i32, P, P, sz, P]),
    "rg_aggregate": (i32, [P, i32, P, P, P, i32, P, P, P]),
    "rg_node_view_factors": (i32, [P, i32, P, P, P, P, P]),
    "rg_node_couplings": (i32, [P, i32, P, P, P, P, P, P, P, P]),
    "rg_gebhart": (i32, [P, i32, P, i32, P, P, P, i32, f64, i32, P, P, P, P, sz, P, sz, P]),
    "rg_gebhart_adjoint": (i32, [P, i32, P, i32, P, P, P, P, i32, f64, i32, P, P, P, sz, P, sz, P]),
    "rg_temperatures": (i32, [P, i32, P, P, P, P, f64, f64, i32, f64, P, P, sz, P]),
    "rg_temperatures_adjoint": (i32, [P, i32, P, P, P, f64, f64, P, P, i32, f64, P, P, P, sz, P]),
    "rg_temperatures_sets": (i32, [P, i32, P, i32, P, P, P, P, P, f64, f64, i32, f64, P, P, sz, P]),
    "rg_temperatures_adjoint_sets": (i32, [P, i32, P, i32, P, P, P, P, f64, f64, P, P, i32, f64, P, P, P, P, P, sz, P]),
    "rg_gebhart_adjoint_factored": (i32, [P, i32, P, i32, P, P, P, i32, P, P, i32, f64, i32, P, P, P, sz, P, sz,
                                          P]),
    "rg_tc_gemm": (i32, [P, i32, i32, i32, P, i64, P, i64, i32, P, i64, ctypes.c_float, ctypes.c_float, P]),
    "rg_exact_split": (i32, [P, i32, P, i64, i32, P, P, P, P]),
    "rg_tc_gemm_exact": (i32, [P, i32, i32, i32, i32, P, i64, P, P, P]),
}

_lib = None


def load():
    """The loaded library with every signature declared; ImportError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libradgeb.so not found at {LIB_PATH}: run "
                              "`python -c 'import __graft_entry__ as g; g.build()'` first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class RadgebError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        self.code = STATUS.get(status, str(status))
        super().__init__(f"{self.code}: {message}")
