"""ctypes declarations of libdh (include/dh.h). Argument marshalling only."""

from __future__ import annotations

import ctypes
import os

import torch  # noqa: F401  (loads the CUDA runtime that libdh shares)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdh.so")

DH_OK = 0
STATUS_NAMES = {0: "DH_OK", 1: "DH_ERR_INVALID_ARG", 2: "DH_ERR_UNSUPPORTED_SIZE",
                3: "DH_ERR_OOM", 4: "DH_ERR_CUDA", 5: "DH_ERR_TIMEOUT",
                6: "DH_ERR_FRAME_GAP", 7: "DH_ERR_STATE"}
PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
FLAG_STORE_OVERFLOW, FLAG_NONFINITE_C, FLAG_EIG_NOT_CONVERGED, FLAG_WAIT_TIMEOUT = 1, 2, 4, 8



class BatchItem(ctypes.Structure):
    """dh_batch_item of include/dh.h."""
    _fields_ = [("plan", ctypes.c_void_p), ("frames_dev", ctypes.c_void_p),
                ("frame_stride_elems", ctypes.c_int64), ("n_frames", ctypes.c_int),
                ("render_slot", ctypes.c_int), ("first_slot", ctypes.c_int),
                ("slot_stride", ctypes.c_int), ("n_windows", ctypes.c_int),
                ("k0", ctypes.c_int), ("k1", ctypes.c_int), ("images_dev", ctypes.c_void_p),
                ("eigvals_dev", ctypes.c_void_p)]


class WindowResult(ctypes.Structure):
    """dh_window_result of include/dh.h."""
    _fields_ = [("stream_id", ctypes.c_int), ("window", ctypes.c_int64),
                ("image_host", ctypes.c_void_p), ("eigvals_host", ctypes.c_void_p),
                ("t_ready_s", ctypes.c_double), ("t_done_s", ctypes.c_double)]


# (name, restype, argtypes) for every entry point of include/dh.h
_vp, _i, _i64, _d, _u32p = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, \
    ctypes.POINTER(ctypes.c_uint32)
SIGNATURES = [
    ("dh_plan_create", _i, [ctypes.POINTER(_vp), _i, _i, _d, _d, _d, _i]),
    ("dh_destroy", None, [_vp]),
    ("dh_plan_create_view", _i, [ctypes.POINTER(_vp), _vp, _i]),
    ("dh_plan_set_precision", _i, [_vp, _i]),
    ("dh_plan_reserve", _i, [_vp, _i, _i]),
    ("dh_plan_set_option", _i, [_vp, _i, _i]),
    ("dh_plan_get_option", _i, [_vp, _i, ctypes.POINTER(_i)]),
    ("dh_plan_autotune", _i, [_vp, _i, _vp]),
    ("dh_plan_tune_load", _i, [_vp, ctypes.c_char_p, ctypes.POINTER(_i)]),
    ("dh_plan_tune_save", _i, [_vp, ctypes.c_char_p]),
    ("dh_plan_device_bytes", ctypes.c_size_t, [_vp]),
    ("dh_plan_footprint", ctypes.c_size_t, [_i, _i, _i, _i, _i, _i]),
    ("dh_render_frames", _i, [_vp, _vp, _i64, _i, _i, _vp]),
    ("dh_pca_windows", _i, [_vp, _i, _i, _i, _i, _i, _vp, _vp, _vp]),
    ("dh_fourier_windows", _i, [_vp, _i, _i, _i, _i, _i, _vp, _vp]),
    ("dh_band_gram", _i, [_vp, _i, _i, _vp]),
    ("dh_svd_fourier_windows", _i, [_vp, _i, _i, _i, _i, _i, _i, _i, _vp, _vp, _vp]),
    ("dh_render_stack", _i, [_vp, _vp, _i64, _vp]),
    ("dh_pca_window", _i, [_vp, _i, _i, _vp, _vp, _vp]),
    ("dh_pca_batch", _i, [_vp, _vp, _i64, _i, _i, _i, _i, _vp, _vp, _vp]),
    ("dh_pca_batch_host", _i, [_vp, _vp, _i64, _i, _i, _i, _i, _vp, _vp, _vp]),
    ("dh_pca_batch_host_packed12", _i, [_vp, _vp, _i64, _i, _i, _i, _i, _vp, _vp, _vp]),
    ("dh_unpack_mono12p", _i, [_vp, _i64, _i64, _i, _vp, _i64, _vp]),
    ("dh_normalize_images", _i, [_vp, _i, _i64, _vp, _vp, ctypes.c_float, _vp, _vp]),
    ("dh_debug_hologram", _i, [_vp, _i, _vp, _vp]),
    ("dh_debug_covariance", _i, [_vp, _i, _vp, _vp]),
    ("dh_debug_eigvecs", _i, [_vp, _i, _vp, _vp]),
    ("dh_plan_status", _i, [_vp, _u32p]),
    ("dh_profile_enable", _i, [_vp, _i]),
    ("dh_profile_read", _i, [_vp, _i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_i),
                             ctypes.POINTER(_d)]),
    ("dh_covariance_noalloc", _i, [_vp, _i64, _i, _vp, _vp]),
    ("dh_measure_fma_rate", _i, [_i, _i, _i, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(_d), _vp]),
    ("dh_measure_mma_issue", _i, [_i, _i, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_d),
                                  ctypes.POINTER(_d), _vp]),
    ("dh_batch_run", _i, [ctypes.POINTER(BatchItem), _i, _vp]),
    ("dh_server_create", _i, [ctypes.POINTER(_vp), ctypes.c_size_t]),
    ("dh_server_stream_bytes", ctypes.c_size_t, [_i, _i, _i, _i, _i]),
    ("dh_server_add_stream", _i, [_vp, _i, _i, _d, _d, _d, _i, _i, _i, _i, _i,
                                  ctypes.POINTER(_i)]),
    ("dh_server_remove_stream", _i, [_vp, _i]),
    ("dh_server_set_tune_cache", _i, [_vp, ctypes.c_char_p, _i]),
    ("dh_server_stream_option", _i, [_vp, _i, _i, ctypes.POINTER(_i)]),
    ("dh_server_used_bytes", ctypes.c_size_t, [_vp]),
    ("dh_server_push", _i, [_vp, _i, _vp, _i64, _i]),
    ("dh_server_poll", _i, [_vp, ctypes.POINTER(WindowResult), _i]),
    ("dh_server_release", _i, [_vp, _i, _i64]),
    ("dh_server_clock", _d, [_vp]),
    ("dh_server_drain", _i, [_vp]),
    ("dh_server_destroy", None, [_vp]),
    ("dh_graph_begin", _i, [_vp]),
    ("dh_graph_end", _i, [_vp, ctypes.POINTER(_vp)]),
    ("dh_graph_launch", _i, [_vp, _vp]),
    ("dh_graph_destroy", None, [_vp]),
    ("dh_status_string", ctypes.c_char_p, [_i]),
    ("dh_last_error", ctypes.c_char_p, []),
    ("dh_version", ctypes.c_char_p, []),
]

_lib = None


def load() -> ctypes.CDLL:
    """Load libdh.so; raise (never fall back) if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libdh.so not found at {LIB_PATH}: build it with "
                "`python -m paper_2004_00923_b300.build` (nvcc, sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class DHError(RuntimeError):
    def __init__(self, fn: str, code: int):
        lib = load()
        msg = f"{fn} -> {STATUS_NAMES.get(code, code)} ({lib.dh_status_string(code).decode()})"
        if code == 4:
            msg += f": {lib.dh_last_error().decode()}"
        super().__init__(msg)
        self.code = code


def check(fn: str, code: int) -> None:
    if code != DH_OK:
        raise DHError(fn, code)
