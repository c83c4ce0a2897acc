"""ctypes loader for libapsp.so: signatures of every entry point in include/apsp.h."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(HERE, "libapsp.so")

APSP_I32, APSP_U16, APSP_F32, APSP_AUTO = 0, 1, 2, 3
INF_I32 = 1073741823
INF_U16 = 0x7FFF
STATES = {0: "QUEUED", 1: "ADMITTED", 2: "RUNNING", 3: "DONE", 4: "ERROR"}
STATUS = {0: "APSP_OK", 1: "APSP_E_INVALID", 2: "APSP_E_CUDA", 3: "APSP_E_NOMEM", 4: "APSP_E_RANGE",
          5: "APSP_E_BUSY", 6: "APSP_E_NOTFOUND", 7: "APSP_E_TIMEOUT", 8: "APSP_E_CANCELLED",
          9: "APSP_E_NOTREADY", 10: "APSP_E_UNSUPPORTED"}


class ApspError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


class apsp_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("dtype", ctypes.c_int), ("block_k", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("queue_depth", ctypes.c_int),
                ("memory_budget", ctypes.c_int64), ("spin_limit", ctypes.c_int64), ("phase3_variant", ctypes.c_int),
                ("symmetric", ctypes.c_int), ("serving_large_n", ctypes.c_int64), ("serving_large_grid", ctypes.c_int)]


class apsp_request(ctypes.Structure):
    _fields_ = [("W", ctypes.c_void_p), ("is_host", ctypes.c_int), ("n", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("dtype", ctypes.c_int)]


def _load():
    if not os.path.exists(lib_path):
        raise ImportError(f"libapsp.so is not built ({lib_path}); run `python -m paper_1902_04446_gb300.build` "
                          "(needs nvcc); there is no CPU fallback")
    L = ctypes.CDLL(lib_path)
    vp, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int
    H = ctypes.c_void_p
    sig = {
        "apsp_config_default": (None, [ctypes.POINTER(apsp_config)]),
        "apsp_create": (st, [ctypes.POINTER(H), ctypes.POINTER(apsp_config)]),
        "apsp_destroy": (st, [H]),
        "apsp_solve": (st, [H, vp, i64, i64, vp, vp]),
        "apsp_solve_t": (st, [H, i32, vp, i64, i64, vp, vp]),
        "apsp_solve_edges": (st, [H, i32, vp, vp, vp, i64, i64, vp, i64, vp]),
        "apsp_last_status": (st, [H, vp]),
        "apsp_int16_bound": (st, [H, vp, i64, i64, ctypes.POINTER(i64), ctypes.POINTER(i32), vp]),
        "apsp_minplus": (st, [H, i32, vp, i64, vp, i64, vp, i64, i64, i64, i64, vp]),
        "apsp_solve_squaring": (st, [H, i32, vp, i64, i64, vp, vp]),
        "apsp_pack_u16": (st, [vp, i64, vp, i64, i64, vp]),
        "apsp_unpack_u16": (st, [vp, i64, vp, i64, i64, vp]),
        "apsp_submit": (st, [H, ctypes.POINTER(apsp_request), ctypes.POINTER(ctypes.c_uint64)]),
        "apsp_poll": (st, [H, ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(vp)]),
        "apsp_wait": (st, [H, ctypes.c_uint64, i64]),
        "apsp_fetch": (st, [H, ctypes.c_uint64, vp, i64, vp]),
        "apsp_release": (st, [H, ctypes.c_uint64]),
        "apsp_cancel": (st, [H, ctypes.c_uint64]),
        "apsp_strerror": (ctypes.c_char_p, [st]),
        "apsp_last_error": (ctypes.c_char_p, [H]),
        "apsp_launch_count": (i64, [H]),
        "apsp_profile": (st, [H, i32]),
        "apsp_solve_batch": (st, [H, i64, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                  ctypes.POINTER(vp), vp]),
        "apsp_check_bounded_wait": (st, [H, i64]),
        "apsp_autotune": (st, [H, i32, i64, ctypes.c_char_p]),
        "apsp_solve_i32_noalloc": (st, [vp, i64, i64, vp, vp]),
        "apsp_noalloc_status": (st, [vp]),
        "apsp_addmin_peak": (st, [i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "apsp_addmin_eval": (st, [i32, vp, vp, vp, vp, i64, vp]),
        "apsp_tri_layout": (st, [i32, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "apsp_tri_from_dense": (st, [H, i32, vp, i64, i64, vp, vp]),
        "apsp_tri_from_edges": (st, [H, i32, vp, vp, vp, i64, i64, vp, vp]),
        "apsp_solve_tri": (st, [H, i32, vp, i64, vp]),
        "apsp_tri_to_dense": (st, [i32, vp, i64, vp, i64, vp]),
        "apsp_tri_rows": (st, [i32, vp, i64, vp, i64, vp, i64, vp]),
        "apsp_tuned_config": (st, [H, i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "apsp_profile_read": (st, [H, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_L = None


def get_lib():
    """The loaded libapsp.so (loaded on first use; raises ImportError when it is not built)."""
    global _L
    if _L is None:
        _L = _load()
    return _L

# every entry point of the header, for the export check
ENTRY_POINTS = sorted(["apsp_config_default", "apsp_create", "apsp_destroy", "apsp_solve", "apsp_solve_t",
                       "apsp_solve_edges", "apsp_last_status", "apsp_int16_bound", "apsp_minplus", "apsp_pack_u16",
                       "apsp_unpack_u16", "apsp_submit", "apsp_poll", "apsp_wait", "apsp_fetch", "apsp_release",
                       "apsp_cancel", "apsp_strerror", "apsp_last_error", "apsp_launch_count",
                       "apsp_profile", "apsp_profile_read", "apsp_solve_batch", "apsp_check_bounded_wait",
                       "apsp_autotune", "apsp_tuned_config", "apsp_solve_i32_noalloc", "apsp_noalloc_status",
                       "apsp_solve_squaring", "apsp_addmin_peak", "apsp_addmin_eval", "apsp_tri_layout",
                       "apsp_tri_from_dense", "apsp_tri_from_edges", "apsp_solve_tri", "apsp_tri_to_dense",
                       "apsp_tri_rows"])
