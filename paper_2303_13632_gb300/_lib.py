"""ctypes binding of the C ABI in include/eri.h (argument marshalling only).

Every function here forwards to the CUDA library ``_build/liberi_gb300.so``; there is
no fallback path.  If the library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

c_double_p = ctypes.POINTER(ctypes.c_double)

ERI_OK = 0
ERI_E_INVALID = 1
ERI_E_UNSUPPORTED = 2
ERI_E_NOMEM = 3
ERI_E_CUDA = 4
ERI_E_NUMERIC = 6

ERI_FP64 = 0
ERI_MIXED = 1
ERI_EXPLICIT = 0
ERI_ALL = 1
ERI_UNIQUE8 = 2
ERI_QUARTETS_ON_DEVICE = 1
ERI_NO_PAIR_TABLE = 2
ERI_NOALLOC_MAX_QUARTETS = 16384
ERI_NUM_CLASS_IDS = 881
ERI_DIGEST_UNIQUE8 = 1
ERI_DIGEST_ACCUMULATE = 2
ERI_DIGEST_SYMMETRIC = 4

STATUS_NAMES = {
    ERI_OK: "ERI_OK", ERI_E_INVALID: "ERI_E_INVALID", ERI_E_UNSUPPORTED: "ERI_E_UNSUPPORTED",
    ERI_E_NOMEM: "ERI_E_NOMEM", ERI_E_CUDA: "ERI_E_CUDA",
    ERI_E_NUMERIC: "ERI_E_NUMERIC",
}

# Every function the header declares, with (restype, argtypes).
_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_szp = ctypes.POINTER(ctypes.c_size_t)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


class eri_shell_t(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 3), ("L", ctypes.c_int32), ("nprim", ctypes.c_int32),
                ("exps", c_double_p), ("coefs", c_double_p)]


class eri_plan_opts_t(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("quartet_mode", ctypes.c_int32),
                ("device", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("schwarz_threshold", ctypes.c_double), ("shard_index", ctypes.c_int64),
                ("shard_count", ctypes.c_int64)]


SIGNATURES = {
    "eri_plan_create": (_i32, [ctypes.POINTER(eri_shell_t), _i32, _p, _i64,
                               ctypes.POINTER(eri_plan_opts_t), ctypes.POINTER(_p)]),
    "eri_plan_destroy": (None, [_p]),
    "eri_plan_update_shells": (_i32, [_p, ctypes.POINTER(eri_shell_t), _i32, _p]),
    "eri_plan_set_precision": (_i32, [_p, _i32]),
    "eri_plan_set_class_precision": (_i32, [_p, _i32, _i32]),
    "eri_plan_calibrate_precision": (_i32, [_p, _i32, _i64, ctypes.c_float, _p]),
    "eri_plan_class_precision": (_i32, [_p, _i32, _i32p, ctypes.POINTER(ctypes.c_float)]),
    "eri_plan_class_launches": (_i32, [_p, _i32, _i32p]),
    "eri_plan_class_kernels": (_i32, [_p, _i32, ctypes.c_char_p, ctypes.c_size_t]),
    "eri_fma_probe": (_i32, [_i32, _i64, _i32, _p, _p]),
    "eri_plan_num_quartets": (_i32, [_p, _i64p]),
    "eri_plan_class_info": (_i32, [_p, _i32, _i64p, _i32p, _i64p, _i64p]),
    "eri_plan_quartet_order": (_i32, [_p, _i64p]),
    "eri_plan_quartets": (_i32, [_p, _p]),
    "eri_plan_screening": (_i32, [_p, _i64p, _i64p]),
    "eri_output_bytes": (_i32, [_p, _i32, _szp, _szp]),
    "eri_packed_class_offset": (_i32, [_p, _i32, _i32, _szp, _szp]),
    "eri_paper512_class_offset": (_i32, [_p, _i32, _i32, _szp, _szp]),
    "eri_pack_paper512": (_i32, [_p, _i32, _p, _p, _p]),
    "eri_pack_paper512_stream": (_i32, [_p, _i64, _i32, _i32, _p, _p]),
    "eri_compute": (_i32, [_p, _p, _p]),
    "eri_compute_class": (_i32, [_p, _i32, _p, _p]),
    "eri_compute_compressed": (_i32, [_p, _i32, _p, _p, _p]),
    "eri_compute_compressed_to_host": (_i32, [_p, _i32, _p, _p, _p, _p, _p]),
    "eri_compute_compressed_class": (_i32, [_p, _i32, _i32, _p, _p, _p]),
    "eri_sync": (_i32, [_p, _p]),
    "eri_backward": (_i32, [_p, _p, _p, _p, _p]),
    "eri_compute_compressed_batched": (_i32, [_p, _i32, _p, _p, _p]),
    "eri_compute_compressed_queue": (_i32, [_p, _i32, _p, _p, _p]),
    "eri_autotune": (_i32, [_p, _i32, _p, _p, ctypes.c_char_p, _p]),
    "eri_status_string": (ctypes.c_char_p, [_i32]),
    "eri_plan_num_basis_functions": (_i32, [_p, _i64p]),
    "eri_digest_jk": (_i32, [_p, _i32, _p, _p, _p, _p, _p, _i32, _p]),
    "eri_compute_class_noalloc": (_i32, [_i32, _i32, _p, _p, _p, _p, _p, _p, _p, _p, _i64, _p, _p, _p]),
    "eri_boys_device": (_i32, [_i32, _p, _i64, _p, _p]),
    "eri_rys_device": (_i32, [_i32, _p, _i64, _p, _p, _p]),
    "eri_rys_device_mixed": (_i32, [_i32, _p, _i64, _p, _p, _p]),
    "eri_convert_device": (_i32, [_p, _i64, _p, _p, _p]),
    "eri_class_id": (_i32, [_i32, _i32, _i32, _i32]),
    "eri_class_shape": (_i32, [_i32, _i32p, _i32p]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Builds (if needed) and loads the CUDA library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or _build.build())
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class EriError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


def check(status: int, where: str = "") -> None:
    if status != ERI_OK:
        raise EriError(status, where)
