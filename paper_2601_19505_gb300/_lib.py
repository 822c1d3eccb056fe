"""ctypes declarations of the C ABI in include/fciqmc.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import _build


class FqKey(C.Structure):
    _fields_ = [("lo", C.c_uint64), ("hi", C.c_uint64)]


class FqParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("target", C.c_double), ("zeta", C.c_double),
                ("xi", C.c_double), ("threshold", C.c_double), ("t_rel", C.c_double),
                ("mode", C.c_int32), ("annihilation", C.c_int32), ("seed", C.c_uint64),
                ("run_id", C.c_uint32), ("compression", C.c_int32),
                ("capacity_vec", C.c_size_t), ("capacity_spawn", C.c_size_t)]


class FqStats(C.Structure):
    _fields_ = [("step", C.c_int64), ("len", C.c_int64), ("exact_steps", C.c_int64),
                ("inexact_steps", C.c_int64), ("n_spawns", C.c_int64), ("shift", C.c_double),
                ("norm", C.c_double), ("hproj", C.c_double), ("vproj", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class FqAllocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


SYMBOLS = {
    # name: (restype, argtypes)
    "fq_version": (C.c_char_p, []),
    "fq_strerror": (C.c_char_p, [C.c_int]),
    "fq_params_default": (C.c_int, [C.POINTER(FqParams)]),
    "fq_params_set_zeta": (C.c_int, [C.POINTER(FqParams), C.c_double]),
    "fq_ham_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int,
                                C.c_double, C.c_double]),
    "fq_ham_destroy": (None, [C.c_void_p]),
    "fq_ham_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                              C.POINTER(C.c_int)]),
    "fq_ham_dimension": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "fq_ham_starting_address": (C.c_int, [C.c_void_p, C.POINTER(FqKey)]),
    "fq_encode": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(FqKey)]),
    "fq_decode": (C.c_int, [C.c_void_p, FqKey, C.c_void_p]),
    "fq_ham_column": (C.c_int, [C.c_void_p, FqKey, C.POINTER(C.c_double), C.c_void_p,
                                C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "fq_ham_column_noalloc": (C.c_int, [C.c_void_p, FqKey, C.POINTER(C.c_double), C.c_void_p,
                                        C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "fq_run_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(FqParams),
                                C.c_void_p, C.POINTER(FqAllocator)]),
    "fq_run_destroy": (None, [C.c_void_p]),
    "fq_run_seed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_double,
                              C.c_int64]),
    "fq_run_seed_default": (C.c_int, [C.c_void_p, C.c_double]),
    "fq_run_set_reference": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t]),
    "fq_run_set_dt": (C.c_int, [C.c_void_p, C.c_double]),
    "fq_run_set_shift": (C.c_int, [C.c_void_p, C.c_double]),
    "fq_run_set_target": (C.c_int, [C.c_void_p, C.c_double]),
    "fq_run_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "fq_run_sync": (C.c_int, [C.c_void_p]),
    "fq_run_error_bits": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint)]),
    "fq_run_stats": (C.c_int, [C.c_void_p, C.POINTER(FqStats)]),
    "fq_run_history": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "fq_run_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                C.POINTER(C.c_size_t)]),
    "fq_run_lookup": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "fq_run_sample": (C.c_int, [C.c_void_p, C.c_uint64, C.c_size_t, C.c_void_p, C.c_void_p,
                                C.c_size_t, C.POINTER(C.c_size_t)]),
    "fq_run_spawns": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                C.POINTER(C.c_size_t)]),
    "fq_run_autotune": (C.c_int, [C.c_void_p, C.c_int]),
    "fq_run_reserve": (C.c_int, [C.c_void_p, C.c_size_t, C.c_size_t]),
    "fq_run_capacity": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "fq_run_set_tables": (C.c_int, [C.c_void_p, C.c_uint, C.c_uint]),
    "fq_run_set_spawn_split": (C.c_int, [C.c_void_p, C.c_uint]),
    "fq_run_merge_paths": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "fq_run_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "fq_run_profile": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_float)]),
    "fq_run_arm_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "fq_batch_set_overlaps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "fq_batch_set_spectral": (C.c_int, [C.c_void_p, C.c_int]),
    "fq_batch_overlaps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t),
                                    C.POINTER(C.c_int)]),
    "fq_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int]),
    "fq_batch_destroy": (None, [C.c_void_p]),
    "fq_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "fq_batch_sync": (C.c_int, [C.c_void_p]),
    "fq_batch_autotune": (C.c_int, [C.c_void_p, C.c_int]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfciqmc.so (built in-tree).  Raises when it is missing: there is
    no CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libfciqmc.so is not built; run __graft_entry__.build()")
    L = C.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L
