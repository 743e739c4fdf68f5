"""ctypes declarations of the oblivgm C ABI (include/oblivgm.h).

The shared library is built in-tree by ``build.py``; there is no fallback:
importing this module on a machine where the library is missing raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_u8p = ctypes.c_void_p
c_u32 = ctypes.c_uint32
c_u64 = ctypes.c_uint64
c_i32 = ctypes.c_int32
c_size = ctypes.c_size_t
c_vp = ctypes.c_void_p

OK, EINVAL, ENOMEM, ECUDA, EARCH, ERANGE, EBUSY, EAGAIN, ETIMEOUT, ENOENT, EFAULT_DEVICE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10)
PRED_EQ, PRED_RANGE = 1, 2
COMBINE_AND, COMBINE_XOR, COMBINE_OR = 0, 1, 2
KEY_DPF, KEY_DCF = 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
ALL_PAIRS = 1
KEYS_DEVICE = 2
SHUFFLE_ADD, SHUFFLE_XOR = 0, 1
AES_TTABLE, AES_BITSLICED = 0, 1
PRG_PARITY = 1
MAX_GROUPS = 64
NOALLOC_SCRATCH_BYTES = 256 * 1024
POLL_LIMIT_DEFAULT_MS = 600000

STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EARCH: "EARCH", ERANGE: "ERANGE",
                EBUSY: "EBUSY", EAGAIN: "EAGAIN", ETIMEOUT: "ETIMEOUT", ENOENT: "ENOENT",
                EFAULT_DEVICE: "EFAULT_DEVICE"}


class Config(ctypes.Structure):
    _fields_ = [("prf_keys", (ctypes.c_uint8 * 16) * 3), ("serve_arena_bytes", c_u64),
                ("serve_max_inflight", c_u32), ("flags", c_u32)]


class Pred(ctypes.Structure):
    _fields_ = [(f, c_u32) for f in ("kind", "table", "attr", "group", "lo", "hi", "combine")]


class Result(ctypes.Structure):
    _fields_ = [("n_groups", c_u32), ("table", c_u32 * MAX_GROUPS), ("n_elems", c_u64 * MAX_GROUPS),
                ("shares", (c_vp * 3) * MAX_GROUPS), ("latency_ms", ctypes.c_double), ("ticket", c_u64)]


_SIGS = {
    "oblivgm_version": ([], c_u32),
    "oblivgm_last_error": ([ctypes.c_char_p, c_size], c_i32),
    "oblivgm_create": ([ctypes.POINTER(c_vp), c_i32, ctypes.POINTER(Config)], c_i32),
    "oblivgm_destroy": ([c_vp], c_i32),
    "oblivgm_sync": ([c_vp, c_vp], c_i32),
    "oblivgm_launch_count": ([c_vp], c_u64),
    "oblivgm_load_shares": ([c_vp, c_u32, c_u64, c_u32, c_u32, ctypes.POINTER(c_vp), c_i32, c_vp], c_i32),
    "oblivgm_unload_shares": ([c_vp, c_u32], c_i32),
    "oblivgm_keygen": ([ctypes.POINTER(Pred), c_u32, c_u32, c_u8p, ctypes.POINTER(c_vp), c_size,
                        ctypes.POINTER(c_size)], c_i32),
    "oblivgm_eval_dpf_batch": ([c_vp, c_u8p, c_u32, c_vp, c_vp, c_u64, c_u32, c_vp, c_u64, c_vp], c_i32),
    "oblivgm_eval_dcf_batch": ([c_vp, c_u8p, c_u32, c_vp, c_vp, c_u64, c_u32, c_vp, c_u64, c_vp], c_i32),
    "oblivgm_filter_and_combine": ([c_vp, c_u32, ctypes.POINTER(c_vp), ctypes.POINTER(c_size), c_u32,
                                    ctypes.POINTER(c_vp), c_vp], c_i32),
    "oblivgm_plan_create": ([c_vp, c_u32, ctypes.POINTER(c_u32), ctypes.POINTER(c_vp), ctypes.POINTER(c_size),
                             ctypes.POINTER(c_u32), ctypes.POINTER(c_vp), ctypes.POINTER(c_vp)], c_i32),
    "oblivgm_plan_launch": ([c_vp, c_vp], c_i32),
    "oblivgm_plan_destroy": ([c_vp], c_i32),
    "oblivgm_keygen_device": ([c_vp, c_u32, c_u32, c_u64, c_vp, c_vp, c_u8p, c_vp, c_u64, c_vp], c_i32),
    "oblivgm_fresh_token_size": ([ctypes.POINTER(Pred), c_u32, c_u32, c_vp, c_u32, ctypes.POINTER(c_u64)], c_i32),
    "oblivgm_keygen_fresh": ([c_vp, ctypes.POINTER(Pred), c_u32, c_u32, c_vp, c_u32, c_u8p, ctypes.POINTER(c_vp),
                              c_u64, c_vp], c_i32),
    "oblivgm_filter_fresh": ([c_vp, c_u32, ctypes.POINTER(c_vp), c_u64, c_u32, ctypes.POINTER(c_vp), c_vp], c_i32),
    "oblivgm_shuffle": ([c_vp, c_u32, c_u64, c_u32, ctypes.POINTER(c_vp), c_u8p, ctypes.POINTER(c_vp), c_vp], c_i32),
    "oblivgm_fetch_multi": ([c_vp, c_u32, ctypes.POINTER(c_vp), c_u32, c_vp, c_u8p, ctypes.POINTER(c_vp), c_u64,
                             ctypes.POINTER(c_u64), c_vp], c_i32),
    "oblivgm_fetch_unique": ([c_vp, c_u32, c_u32, c_u32, ctypes.POINTER(c_vp), c_u32, ctypes.POINTER(c_u32), c_vp,
                              c_vp], c_i32),
    "oblivgm_keygen_onehot": ([ctypes.POINTER(Pred), c_u32, c_u32, c_u8p, ctypes.POINTER(c_vp), c_size,
                               ctypes.POINTER(c_size)], c_i32),
    "oblivgm_load_onehot": ([c_vp, c_u32, c_u64, c_u32, c_u32, ctypes.POINTER(c_vp), c_i32, c_vp], c_i32),
    "oblivgm_filter_onehot": ([c_vp, c_u32, ctypes.POINTER(c_vp), ctypes.POINTER(c_size), c_u32,
                               ctypes.POINTER(c_vp), c_vp], c_i32),
    "oblivgm_filter_plain": ([c_vp, c_u32, ctypes.POINTER(c_vp), ctypes.POINTER(c_size), c_u32,
                              ctypes.POINTER(c_vp), c_vp], c_i32),
    "oblivgm_filter_and_combine_noalloc": ([c_vp, c_u32, ctypes.POINTER(c_vp), ctypes.POINTER(c_size), c_u32,
                                            ctypes.POINTER(c_vp), c_vp], c_i32),
    "oblivgm_filter_batch": ([c_vp, c_u32, ctypes.POINTER(c_u32), ctypes.POINTER(c_vp), ctypes.POINTER(c_size),
                              ctypes.POINTER(c_u32), ctypes.POINTER(c_vp), c_vp], c_i32),
    "oblivgm_submit": ([c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_size), ctypes.POINTER(c_u64)], c_i32),
    "oblivgm_poll": ([c_vp, c_u64, c_i32, ctypes.POINTER(Result)], c_i32),
    "oblivgm_release": ([c_vp, c_u64], c_i32),
    "oblivgm_set_poll_limit": ([c_vp, c_u32, ctypes.POINTER(c_u32)], c_i32),
    "oblivgm_serve_stats": ([c_vp] + [ctypes.POINTER(c_u64)] * 4, c_i32),
    "oblivgm_autotune": ([c_vp, ctypes.POINTER(c_u32), ctypes.POINTER(c_u32)], c_i32),
    "oblivgm_set_schedule": ([c_vp, c_u32, c_u32], c_i32),
    "oblivgm_plan_describe": ([c_vp, ctypes.POINTER(c_u32), ctypes.POINTER(c_u32), ctypes.POINTER(c_u32),
                               ctypes.POINTER(c_u64), ctypes.POINTER(c_u32)], c_i32),
    "oblivgm_set_walk_parallel": ([c_vp, c_u64, ctypes.POINTER(c_u64)], c_i32),
    "oblivgm_set_walk_parallel_tile": ([c_vp, c_u32, ctypes.POINTER(c_u32)], c_i32),
    "oblivgm_test_expire_next_wait": ([c_vp, c_u32], c_i32),
    "oblivgm_test_fail_next_alloc": ([c_vp], c_i32),
    "oblivgm_prg_batch": ([c_vp, c_u32, c_u32, c_u64, c_u64, c_u32, c_vp, c_u64, c_vp], c_i32),
    "oblivgm_autotune_aes_layout": ([c_vp, ctypes.POINTER(c_u32), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)], c_i32),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liboblivgm.so (building it first if allowed); raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"liboblivgm.so is missing at {path}; run build() first")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


class OblivgmError(RuntimeError):
    def __init__(self, status: int, where: str, text: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({text})")
        self.status = status


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    load().oblivgm_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(status: int, where: str) -> int:
    if status != OK:
        raise OblivgmError(status, where, last_error())
    return status
