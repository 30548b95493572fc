"""ctypes declarations of the C ABI in ``include/dnadfa.h``.

Loads the in-tree ``_build/libdnadfa.so`` (building it first when the sources
are newer).  There is no fallback: if the library cannot be built or loaded,
importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

DFA_OK, DFA_EINVAL, DFA_ETRUNC, DFA_ETIMEOUT, DFA_ECUDA, DFA_EWORKSPACE, DFA_ENOMEM = range(7)
DFA_LOCATE_MAX = 4096
DFA_MAX_M = 64
DFA_COUNT_FAILED = 1 << 63


class dfa_config(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("loader", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32)]


def _declare(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    cfgp = ctypes.POINTER(dfa_config)
    sig = {
        "dfa_build": ([ctypes.c_char_p, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "dfa_free": ([vp], None),
        "dfa_table_bytes": ([i32], i64),
        "dfa_build_into": ([ctypes.c_char_p, i32, vp, i64, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "dfa_pattern_length": ([vp], i32),
        "dfa_export_stt": ([vp, vp, i64], ctypes.c_int),
        "dfa_count": ([vp, i64, vp, vp, cfgp, vp], ctypes.c_int),
        "dfa_find_workspace_bytes": ([i64, cfgp], i64),
        "dfa_find": ([vp, i64, vp, vp, i64, vp, vp, i64, cfgp, vp], ctypes.c_int),
        "dfa_find_status": ([vp, vp, i64, ctypes.POINTER(ctypes.c_uint64), vp], ctypes.c_int),
        "dfa_host_stage_bytes": ([i64, i64], i64),
        "dfa_find_host": ([vp, i64, vp, vp, i64, ctypes.POINTER(ctypes.c_uint64), vp, i64, i64, vp],
                          ctypes.c_int),
        "dfa_find_noalloc": ([vp, i64, vp, vp, i64, vp, cfgp, vp], ctypes.c_int),
        "dfa_find_batched": ([vp, i64, ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(i64), vp,
                              vp, i64, cfgp, vp], ctypes.c_int),
        "dfa_host_stage_bytes_multi": ([i64, ctypes.POINTER(i64), i32], i64),
        "dfa_find_host_multi": ([vp, i64, ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                 ctypes.POINTER(ctypes.c_uint64), vp, i64, i64, vp], ctypes.c_int),
        "dfa_multi_build": ([ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i32), i32, ctypes.POINTER(vp)],
                            ctypes.c_int),
        "dfa_multi_free": ([vp], None),
        "dfa_multi_build_host": ([ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i32), i32,
                                  ctypes.POINTER(vp)], ctypes.c_int),
        "dfa_multi_build_class": ([ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i32), i32,
                                   ctypes.POINTER(vp)], ctypes.c_int),
        "dfa_multi_build_class_host": ([ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i32), i32,
                                        ctypes.POINTER(vp)], ctypes.c_int),
        "dfa_multi_pattern_length": ([vp, i32], i32),
        "dfa_multi_image_bytes": ([vp], i64),
        "dfa_multi_attach": ([vp, vp, i64, vp], ctypes.c_int),
        "dfa_multi_states": ([vp], i32),
        "dfa_multi_export": ([vp, vp, vp, i64], ctypes.c_int),
        "dfa_multi_smem_bytes": ([vp], i64),
        "dfa_multi_count": ([ctypes.POINTER(vp), ctypes.POINTER(i64), i32, vp, vp, cfgp, vp], ctypes.c_int),
        "dfa_debug_wait_timeout": ([vp, i64, i64, vp], ctypes.c_int),
        "dfa_multi_locate_work_bytes": ([i32], i64),
        "dfa_multi_locate": ([vp, i64, vp, ctypes.POINTER(ctypes.c_uint64), vp, i64, vp, i64, vp], ctypes.c_int),
        "dfa_multi_locate_status": ([vp, i32, vp], ctypes.c_int),
        "dfa_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "dfa_version": ([], ctypes.c_char_p),
        "dfa_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def load(path: str | None = None):
    so = path or _build.build()
    if not os.path.exists(so):
        raise ImportError(f"libdnadfa.so not found at {so}")
    return _declare(ctypes.CDLL(so))


lib = load()
LIBRARY_PATH = _build.SO
