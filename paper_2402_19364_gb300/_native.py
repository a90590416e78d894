"""ctypes declarations of the C-ABI in include/arrow.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
from pathlib import Path

LIB_PATH = Path(__file__).resolve().with_name("libarrow_gb300.so")

ARROW_OK = 0
ARROW_EINVAL = -1
ARROW_ENOMEM = -2
ARROW_ECUDA = -3
ARROW_ETIMEOUT = -4
ARROW_ESTATE = -5
ERROR_NAMES = {ARROW_EINVAL: "EINVAL", ARROW_ENOMEM: "ENOMEM", ARROW_ECUDA: "ECUDA",
               ARROW_ETIMEOUT: "ETIMEOUT", ARROW_ESTATE: "ESTATE"}

ARROW_F32, ARROW_BF16, ARROW_F16 = 0, 1, 2
ARROW_PRED_BLOCK, ARROW_PRED_BAND = 0, 1
ARROW_HOST_ONLY = 0x1
ARROW_DEVICE_DECOMPOSE = 0x2
ARROW_RESCALE = 0x1
ARROW_PROFILE = 0x2
ARROW_GRAPH = 0x4
ARROW_RELU = 0x8
ARROW_ROWNORM = 0x10
ARROW_K_ROWS, ARROW_K_SEGMENTS, ARROW_K_NORM, ARROW_K_PERMUTE, ARROW_K_FUSED = 0, 1, 2, 3, 4


class ArrowError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"arrow {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class ArrowCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class ArrowOpts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("value_dtype", ctypes.c_int32), ("predicate", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("nthreads", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("long_row", ctypes.c_int32), ("segment", ctypes.c_int32), ("device", ctypes.c_int32)]


class ArrowStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("b", ctypes.c_int64),
                ("levels", ctypes.c_int32), ("value_dtype", ctypes.c_int32),
                ("long_rows", ctypes.c_int64), ("segments", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("decompose_seconds", ctypes.c_double)]


class ArrowLevelShape(ctypes.Structure):
    _fields_ = [("n_active", ctypes.c_int64), ("nnz", ctypes.c_int64), ("head_nnz", ctypes.c_int64),
                ("band_nnz", ctypes.c_int64), ("tiles", ctypes.c_int64)]


class ArrowProgram(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_short", ctypes.c_int64), ("n_long_entries", ctypes.c_int64),
                ("n_long_rows", ctypes.c_int64), ("n_segments", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("long_row", ctypes.c_int32)] + [(f, ctypes.POINTER(ctypes.c_int32)) for f in (
                    "rowptr", "col", "src", "lcol", "lsrc", "long_rows", "long_segptr", "seg_begin", "seg_end",
                    "tile_row", "tile_ent")]


class ArrowTuning(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_int32), ("tile_nnz", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("carveout", ctypes.c_int32), ("fold_permute_in", ctypes.c_int32),
                ("fused_small", ctypes.c_int32)]


class ArrowServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("max_active", ctypes.c_int32), ("x_dtype", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("device", ctypes.c_int32)]


class ArrowServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("active", ctypes.c_int64), ("inflight_steps", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("steps", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("peak_bytes", ctypes.c_int64), ("status", ctypes.c_int32), ("host_seconds", ctypes.c_double),
                ("wait_seconds", ctypes.c_double), ("gpu_seconds", ctypes.c_double)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SIZE = ctypes.c_size_t

# name -> (restype, argtypes); every function declared in include/arrow.h
SIGNATURES = {
    "arrow_opts_default": (_I32, [ctypes.POINTER(ArrowOpts)]),
    "arrow_decompose": (_I32, [ctypes.POINTER(ArrowCsr), _I64, ctypes.POINTER(ArrowOpts), ctypes.POINTER(_P)]),
    "arrow_upload": (_I32, [_P]),
    "arrow_free": (None, [_P]),
    "arrow_handle_copy": (_I32, [_P, _I32, ctypes.POINTER(_P)]),
    "arrow_save": (_I32, [_P, ctypes.c_char_p]),
    "arrow_load": (_I32, [ctypes.c_char_p, ctypes.POINTER(ArrowOpts), ctypes.POINTER(_P)]),
    "arrow_batch_create": (_I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P)]),
    "arrow_batch_spmm": (_I32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I64), _I32, _I32, _I32, _P]),
    "arrow_batch_status": (_I32, [_P, ctypes.POINTER(_I32)]),
    "arrow_batch_free": (None, [_P]),
    "arrow_server_create": (_I32, [ctypes.POINTER(ArrowServerOpts), ctypes.POINTER(_P)]),
    "arrow_server_submit": (_I32, [_P, _P, _P, _P, _I64, _I32, ctypes.POINTER(_I64)]),
    "arrow_server_step": (_I32, [_P, _P, ctypes.POINTER(_I32)]),
    "arrow_server_poll": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double), _I32, ctypes.POINTER(_I32)]),
    "arrow_server_drain": (_I32, [_P, _P]),
    "arrow_server_get_stats": (_I32, [_P, ctypes.POINTER(ArrowServerStats)]),
    "arrow_server_free": (None, [_P]),
    "arrow_spmm": (_I32, [_P, _P, _I64, _I32, _P, _I32, _I32, _P]),
    "arrow_workspace_size": (_I32, [_P, _I64, _I32, _I32, ctypes.POINTER(_SIZE)]),
    "arrow_spmm_ws": (_I32, [_P, _P, _I64, _I32, _P, _I32, _I32, _P, _SIZE, _P]),
    "arrow_spmm_static": (_I32, [_P, _P, _I64, _I32, _P, _I32, _I32, _P]),
    "arrow_num_levels": (_I32, [_P, ctypes.POINTER(_I32)]),
    "arrow_level_info": (_I32, [_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "arrow_level_perm": (_I32, [_P, _I32, _P]),
    "arrow_level_csr": (_I32, [_P, _I32, _P, _P, _P]),
    "arrow_get_level_shape": (_I32, [_P, _I32, ctypes.POINTER(ArrowLevelShape)]),
    "arrow_count_tiles": (_I32, [ctypes.POINTER(ArrowCsr), _I64, ctypes.POINTER(_I64)]),
    "arrow_get_program": (_I32, [_P, ctypes.POINTER(ArrowProgram)]),
    "arrow_get_stats": (_I32, [_P, ctypes.POINTER(ArrowStats)]),
    "arrow_profile_get": (_I32, [_P, _I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "arrow_status": (_I32, [_P, ctypes.POINTER(_I32)]),
    "arrow_selftest_timeout": (_I32, [_I64, ctypes.POINTER(_I32)]),
    "arrow_selftest_grid_timeout": (_I32, [_I64, _I32, ctypes.POINTER(_I32)]),
    "arrow_get_tuning": (_I32, [_P, ctypes.POINTER(ArrowTuning)]),
    "arrow_set_tuning": (_I32, [_P, ctypes.POINTER(ArrowTuning)]),
    "arrow_autotune": (_I32, [_P, _P, _P, _I64, _I32, _I32, _I32, _P, ctypes.POINTER(ArrowTuning),
                              ctypes.POINTER(ctypes.c_double)]),
    "arrow_batch_autotune": (_I32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I64), _I32, _I32, _P,
                                    ctypes.POINTER(ArrowTuning), ctypes.POINTER(ctypes.c_double)]),
    "arrow_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise ImportError(f"{LIB_PATH.name} is not built: run `python -m paper_2402_19364_gb300.build` "
                              "(the arrow SpMM has no CPU or library fallback)")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != ARROW_OK:
        msg = lib().arrow_last_error()
        raise ArrowError(rc, msg.decode() if msg else "")
