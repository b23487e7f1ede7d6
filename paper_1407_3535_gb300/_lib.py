"""ctypes declarations of libopta.so's C ABI (include/opta.h, include/opta_debug.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  Loading fails loudly when the shared library is missing.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int32, c_int64, c_size_t, c_uint8, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("OPTA_LIB", os.path.join(PKG, "_build", "libopta.so"))

OPTA_U8, OPTA_F32 = 0, 1

STATUS = {
    0: "OPTA_OK", 1: "OPTA_ERR_INVALID_ARG", 2: "OPTA_ERR_FLAT_TEMPLATE", 3: "OPTA_ERR_OOM",
    4: "OPTA_ERR_CUDA", 5: "OPTA_ERR_TIMEOUT", 6: "OPTA_ERR_BUSY", 7: "OPTA_ERR_UNSUPPORTED",
    8: "OPTA_ERR_TOO_LARGE",
}


class OptaImage(ctypes.Structure):
    _fields_ = [("rows", c_int32), ("cols", c_int32), ("stride_elems", c_int64),
                ("dtype", c_int32), ("on_device", c_int32), ("data", c_void_p)]


class OptaTemplate(ctypes.Structure):
    _fields_ = [("rows", c_int32), ("cols", c_int32), ("stride_elems", c_int64),
                ("on_device", c_int32), ("reserved", c_int32), ("data", c_void_p)]


class OptaResult(ctypes.Structure):
    _fields_ = [("y", c_int32), ("x", c_int32), ("rho", c_double),
                ("n_locations", c_int64), ("n_centres", c_int64), ("n_survivors", c_int64),
                ("n_candidates", c_int64), ("n_evaluated", c_int64), ("rho_threshold", c_double),
                ("group_h", c_int32), ("status", c_int32), ("y_hat", c_int32),
                ("x_hat", c_int32), ("rematch_d", c_int32), ("reserved", c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class OptaParams(ctypes.Structure):
    _fields_ = [("rho_th", c_double), ("rho_max", c_double), ("xi", c_double),
                ("block", c_int32), ("n_levels", c_int32), ("sigma_levels", c_float * 8),
                ("h_max", c_int32), ("fixed_h", c_int32), ("blur", c_int32), ("topk", c_int32),
                ("precision", c_int32), ("literal", c_int32), ("egs_sample", c_int32),
                ("dense", c_int32), ("dense_cut", c_float), ("reserved", c_int32 * 3)]


class OptaServerConfig(ctypes.Structure):
    _fields_ = [("n_workers", c_int32), ("max_batch", c_int32), ("memory_budget", c_int64),
                ("reserved", c_int32 * 8)]


class OptaCompletion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("image_id", c_int32), ("batch_size", c_int32),
                ("worker", c_int32), ("status", c_int32), ("t_submit", c_double),
                ("t_start", c_double), ("t_done", c_double), ("result", OptaResult)]


class OptaSizeInfo(ctypes.Structure):
    _fields_ = [("m", c_int32), ("n", c_int32), ("group_h", c_int32), ("level", c_int32),
                ("cost", c_int64), ("n_groups", c_int64), ("blocks_y", c_int32),
                ("blocks_x", c_int32), ("n_egs_evals", c_int32), ("reserved", c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


# name -> (restype, argtypes); every symbol declared in include/*.h
SIGNATURES = {
    "opta_params_default": (None, [POINTER(OptaParams)]),
    "opta_status_str": (c_char_p, [c_int32]),
    "optA_prepare": (c_int32, [POINTER(OptaImage), POINTER(OptaParams), POINTER(c_int32), c_int32,
                               c_void_p, POINTER(c_void_p)]),
    "optA_ctx_create": (c_int32, [c_void_p, POINTER(c_void_p)]),
    "optA_ctx_destroy": (c_int32, [c_void_p]),
    "optA_ctx_memory_bytes": (c_int32, [c_void_p, POINTER(c_size_t)]),
    "optA_search_ctx": (c_int32, [c_void_p, c_void_p, POINTER(OptaTemplate), c_int32,
                                  POINTER(OptaResult), c_void_p]),
    "optA_ctx_bytes_after": (c_int32, [c_void_p, c_void_p, POINTER(OptaTemplate), c_int32,
                                       POINTER(c_size_t)]),
    "opta_server_config_default": (None, [POINTER(OptaServerConfig)]),
    "opta_server_create": (c_int32, [POINTER(OptaServerConfig), POINTER(c_void_p)]),
    "opta_server_add_image": (c_int32, [c_void_p, POINTER(OptaImage), c_void_p, c_void_p, c_int32,
                                        POINTER(c_int32)]),
    "opta_server_submit": (c_int32, [c_void_p, c_int32, POINTER(OptaTemplate),
                                     POINTER(ctypes.c_uint64)]),
    "opta_server_wait": (c_int32, [c_void_p, POINTER(OptaCompletion), c_int32, c_int32, c_int32,
                                   POINTER(c_int32)]),
    "opta_server_pending": (c_int32, [c_void_p, POINTER(c_int64)]),
    "opta_server_memory": (c_int32, [c_void_p, c_int32, POINTER(c_int64), POINTER(c_int64)]),
    "opta_server_destroy": (c_int32, [c_void_p]),
    "optA_graph_create": (c_int32, [c_void_p, POINTER(OptaTemplate), c_int32, c_void_p,
                                    POINTER(c_void_p)]),
    "optA_graph_set_template": (c_int32, [c_void_p, c_int32, POINTER(OptaTemplate), c_void_p]),
    "optA_graph_launch": (c_int32, [c_void_p, POINTER(OptaResult), c_void_p]),
    "optA_graph_info": (c_int32, [c_void_p, POINTER(c_int64)]),
    "optA_graph_destroy": (c_int32, [c_void_p]),
    "optA_search": (c_int32, [c_void_p, POINTER(OptaTemplate), c_int32, POINTER(OptaResult),
                              c_void_p]),
    "zncc_full": (c_int32, [POINTER(OptaImage), POINTER(OptaTemplate), c_void_p,
                            POINTER(OptaResult), c_void_p]),
    "zncc_full_noalloc": (c_int32, [POINTER(OptaImage), POINTER(OptaTemplate), c_void_p,
                                    POINTER(OptaResult), c_void_p]),
    "optA_debug_bounds": (c_int32, [c_void_p, POINTER(OptaTemplate), c_void_p, c_void_p, c_void_p]),
    "optA_size_info": (c_int32, [c_void_p, c_int32, c_int32, POINTER(OptaSizeInfo)]),
    "optA_memory_bytes": (c_int32, [c_void_p, POINTER(c_size_t)]),
    "optA_destroy": (c_int32, [c_void_p]),
    "opta_dbg_window_stats": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p,
                                        c_void_p]),
    "opta_dbg_blur": (c_int32, [c_void_p, c_int32, c_int32, POINTER(c_float), c_int32, c_void_p,
                                c_void_p]),
    "opta_dbg_blur_corr": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32,
                                     c_void_p, c_float, c_int32, c_void_p, c_void_p]),
    "opta_dbg_rho_co": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                                  c_void_p, c_double, POINTER(c_int64), c_void_p]),
    "optA_debug_maps": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                  POINTER(c_float), c_void_p]),
    "optA_debug_scan1": (c_int32, [c_void_p, POINTER(OptaTemplate), c_int32, c_void_p, c_void_p,
                                   c_void_p]),
    "opta_dbg_i64_to_f32": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p]),
    "opta_dbg_survivors": (c_int32, [c_void_p, POINTER(OptaTemplate), c_void_p, c_int64, c_int32,
                                     c_void_p, c_void_p, c_void_p]),
    "opta_dbg_survivor_lane_min": (c_int32, [c_int32, c_int32, c_int32, POINTER(c_int32), POINTER(c_int32)]),
    "opta_dbg_launch_count": (ctypes.c_uint64, []),
    "opta_dbg_scan1_wait": (None, [ctypes.c_uint64, c_int32]),
    "opta_dbg_profile_enable": (None, [c_int32]),
    "opta_dbg_profile_read": (c_int32, [ctypes.c_char_p, c_int32, POINTER(c_double),
                                        POINTER(c_int64), c_int32]),
}

_LIB = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libopta.so not found at {LIB_PATH}; build it with "
                "`python -m paper_1407_3535_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB
