"""ctypes binding of libldp.so (the C-ABI declared in include/ldp.h).

Argument marshalling only: every step of the extraction runs in the CUDA
kernels behind these entry points.  If the library is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libldp.so")

LDP_OK, LDP_EINVAL, LDP_ECUDA, LDP_ENOMEM, LDP_ETIMEOUT, LDP_ENOTIMPL = range(6)
STATUS_NAMES = {0: "LDP_OK", 1: "LDP_EINVAL", 2: "LDP_ECUDA", 3: "LDP_ENOMEM", 4: "LDP_ETIMEOUT",
                5: "LDP_ENOTIMPL"}
LDP_PLAN_LBP = 1
LDP_PLAN_NO_GRAPH = 2
# readings of Eq. 2-3 (code modes)
LDP_CODE_ABS = 0         # the k largest |m_i|, ties to the lower index
LDP_CODE_RAW = 1         # the k largest signed m_i, ties to the lower index
LDP_CODE_ABS_THRESH = 2  # every i with |m_i| >= the k-th largest |m|
LDP_CODE_RAW_THRESH = 3  # every i with m_i >= the k-th largest m


LDP_DIST_L1, LDP_DIST_INTERSECT, LDP_DIST_CHI2 = 0, 1, 2


def plan_code_mode(m: int) -> int:
    return (int(m) & 3) << 2

# Every function include/ldp.h declares (checked by the CPU test suite).
EXPORTS = [
    "ldp_codes", "ldp_region_hist", "lbp_codes", "lbp_region_hist",
    "ldp_batch_plan_create", "ldp_batch_run", "lbp_batch_run", "ldp_batch_plan_destroy",
    "ldp_batch_plan_set_config", "ldp_num_variants", "ldp_variant_name", "ldp_set_plain_variant",
    "ldp_hist_bins", "ldp_bin_of_code", "ldp_last_error", "ldp_device_status", "ldp_version",
    "ldp_batch_plan_enable_timing", "ldp_batch_plan_kernel_times", "ldp_batch_run_noalloc",
    "ldp_server_create", "ldp_server_submit", "ldp_server_poll", "ldp_server_stats", "ldp_server_destroy",
    "ldp_window_count", "ldp_window_scratch_bytes", "ldp_window_hist", "lbp_window_hist",
    "ldp_batch_window_scratch_bytes", "ldp_batch_window_hist", "ldp_codes_ex", "ldp_region_hist_ex",
    "ldp_resize", "ldp_batch_resize", "ldp_hist_distance", "ldp_pipeline_create", "ldp_pipeline_run",
    "ldp_pipeline_destroy", "ldp_pipeline_set_config", "ldp_test_inject_fault",
]
LDP_FAULT_DEVICE_ALLOC, LDP_FAULT_SERVER_LAUNCH, LDP_FAULT_STAGE_WAIT = 0, 1, 2


class LdpError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class RegionSpec(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("C", ctypes.c_int32), ("compact", ctypes.c_int32)]


class WindowSpec(ctypes.Structure):
    _fields_ = [("wh", ctypes.c_int32), ("ww", ctypes.c_int32), ("sh", ctypes.c_int32), ("sw", ctypes.c_int32),
                ("compact", ctypes.c_int32)]


class ImageDesc(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("pitch", ctypes.c_int32), ("code_pitch", ctypes.c_int32),
                ("codes", ctypes.c_void_p), ("hist_offset", ctypes.c_uint64)]


assert ctypes.sizeof(ImageDesc) == 40


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32), ("arena_bytes", ctypes.c_uint64),
                ("k", ctypes.c_int32), ("rs", RegionSpec), ("variant", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("t_submit_ns", ctypes.c_uint64), ("t_start_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("completed", "pixels", "batches", "pending", "arena_used",
                                                "arena_bytes")]

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Loads libldp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or os.environ.get("LDP_LIBRARY") or LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with `python -m paper_1810_11518_gb300.build` "
                              "(nvcc, sm_103a); there is no fallback path")
        lib = ctypes.CDLL(path)
        vp, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_uint64
        sig = {
            "ldp_codes": [vp, i32, i32, i32, i32, vp, i32, vp],
            "ldp_region_hist": [vp, i32, i32, i32, i32, RegionSpec, vp, vp, i32, vp],
            "lbp_codes": [vp, i32, i32, i32, vp, i32, vp],
            "lbp_region_hist": [vp, i32, i32, i32, i32, i32, vp, vp, i32, vp],
            "ldp_batch_plan_create": [ctypes.POINTER(vp), i32, u64, i32, RegionSpec, u32],
            "ldp_batch_run": [vp, vp, vp, vp, vp],
            "lbp_batch_run": [vp, vp, vp, vp, vp],
            "ldp_batch_plan_destroy": [vp],
            "ldp_batch_plan_set_config": [vp, i32, i32],
            "ldp_num_variants": [],
            "ldp_variant_name": [i32],
            "ldp_set_plain_variant": [i32],
            "ldp_hist_bins": [i32],
            "ldp_bin_of_code": [i32, i32],
            "ldp_last_error": [],
            "ldp_device_status": [vp, ctypes.POINTER(i32)],
            "ldp_version": [],
            "ldp_batch_plan_enable_timing": [vp, i32],
            "ldp_batch_plan_kernel_times": [vp, ctypes.POINTER(ctypes.c_float), i32, ctypes.POINTER(i32)],
            "ldp_batch_run_noalloc": [vp, i32, u64, i32, i32, RegionSpec, vp, vp],
            "ldp_server_create": [ctypes.POINTER(vp), ctypes.POINTER(ServerConfig)],
            "ldp_server_submit": [vp, vp, i32, i32, i32, vp, i32, vp, u64],
            "ldp_server_poll": [vp, ctypes.POINTER(Completion), i32, ctypes.POINTER(i32)],
            "ldp_server_stats": [vp, ctypes.POINTER(ServerStats)],
            "ldp_server_destroy": [vp],
            "ldp_window_count": [i32, i32, i32],
            "ldp_codes_ex": [vp, i32, i32, i32, i32, i32, vp, i32, vp],
            "ldp_resize": [vp, i32, i32, i32, i32, i32, i32, i32, vp, i32, i32, i32, vp],
            "ldp_batch_resize": [vp, i32, i32, i32, vp],
            "ldp_hist_distance": [vp, i32, i32, vp, i32, i32, i32, i32, vp, i32, vp],
            "ldp_pipeline_create": [ctypes.POINTER(vp), i32, u64, i32, RegionSpec, i32, u32],
            "ldp_pipeline_run": [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "ldp_pipeline_destroy": [vp],
            "ldp_pipeline_set_config": [vp, i32, i32],
            "ldp_region_hist_ex": [vp, i32, i32, i32, i32, i32, RegionSpec, vp, vp, i32, vp],
            "ldp_window_scratch_bytes": [i32, i32, i32, WindowSpec, i32],
            "ldp_window_hist": [vp, i32, i32, i32, i32, WindowSpec, vp, vp, i32, vp, u64, vp],
            "lbp_window_hist": [vp, i32, i32, i32, WindowSpec, vp, vp, i32, vp, u64, vp],
            "ldp_batch_window_scratch_bytes": [i32, i32, i32, i32, WindowSpec],
            "ldp_batch_window_hist": [vp, i32, i32, i32, i32, WindowSpec, vp, vp, u64, vp],
            "ldp_test_inject_fault": [i32, i32, i32, vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.ldp_window_scratch_bytes.restype = u64
        lib.ldp_batch_window_scratch_bytes.restype = u64
        lib.ldp_last_error.restype = ctypes.c_char_p
        lib.ldp_variant_name.restype = ctypes.c_char_p
        _lib = lib
        return lib


def check(status: int, fn: str) -> None:
    if status != LDP_OK:
        msg = load().ldp_last_error()
        raise LdpError(status, fn, msg.decode() if msg else "")


def call(fn: str, *args) -> None:
    check(getattr(load(), fn)(*args), fn)
