"""ctypes declarations of the C ABI in include/femnfft.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfemnfft.so")

FS_OK, FS_EINVAL, FS_EDOMAIN, FS_ENOMEM, FS_ECUDA, FS_ETIMEOUT, FS_EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "FS_OK", 1: "FS_EINVAL", 2: "FS_EDOMAIN", 3: "FS_ENOMEM", 4: "FS_ECUDA",
                5: "FS_ETIMEOUT", 6: "FS_EUNSUPPORTED"}
FS_F32, FS_F64 = 32, 64
FS_FLAG_NO_KAHAN, FS_FLAG_TIMING, FS_FLAG_AUTOTUNE, FS_FLAG_SERIAL = 1, 2, 4, 8
FS_FLAG_SPREAD_DIRECT, FS_FLAG_SPREAD_TILES = 16, 32
FS_PROBE_FFMA, FS_PROBE_FFMA2, FS_PROBE_MUFU = 0, 1, 2

EXPORTED = (
    "fs_plan_create", "fs_plan_create_fem", "fs_set_charges", "fs_set_magnetization", "fs_set_magnetization_static",
    "fs_fem_charges", "fs_fem_sources", "fs_eval_potential", "fs_eval_field", "fs_solve_host", "fs_adjoint",
    "fs_sync_status", "fs_plan_info", "fs_stage_times", "fs_plan_destroy", "fs_last_error",
    "fs_version", "fs_batch_create", "fs_batch_eval", "fs_batch_sync_status", "fs_batch_info", "fs_batch_plan",
    "fs_batch_destroy", "fs_wait_selftest", "fs_probe_throughput", "fs3_plan_create", "fs3_set_charges", "fs3_eval_field",
    "fs3_sync_status", "fs3_plan_info", "fs3_plan_destroy", "fs3_plan_create_fem", "fs3_set_magnetization",
    "fs3_fem_charges", "fs3_fem_sources",
)


class FsOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("p", ctypes.c_int), ("eps_B", ctypes.c_double),
                ("cell", ctypes.c_int), ("tile_cells", ctypes.c_int), ("flags", ctypes.c_uint),
                ("stream", ctypes.c_void_p)]


class FsInfo(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("n_tgt", ctypes.c_int64),
                ("n_grid", ctypes.c_int), ("n_os", ctypes.c_int), ("m", ctypes.c_int), ("p", ctypes.c_int),
                ("precision", ctypes.c_int),
                ("eps_I", ctypes.c_double), ("eps_B", ctypes.c_double), ("scale", ctypes.c_double),
                ("window_lo", ctypes.c_int), ("window_n", ctypes.c_int),
                ("cell", ctypes.c_int), ("cells_per_dim", ctypes.c_int),
                ("tile_cells", ctypes.c_int), ("spread_items", ctypes.c_int),
                ("near_pairs", ctypes.c_int64), ("near_pairs_fp64", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("is_fem", ctypes.c_int),
                ("n_nodes", ctypes.c_int64), ("n_tris", ctypes.c_int64), ("n_bedges", ctypes.c_int64),
                ("spread_direct", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class FsInstance(ctypes.Structure):
    _fields_ = [("src_xy", ctypes.c_void_p), ("M", ctypes.c_int64), ("tgt_xy", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("n_grid", ctypes.c_int), ("eps_I", ctypes.c_double)]


class FsBatchFacts(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("nrhs", ctypes.c_int), ("precision", ctypes.c_int),
                ("total_src", ctypes.c_int64), ("total_tgt", ctypes.c_int64),
                ("spread_items", ctypes.c_int), ("fft_units", ctypes.c_int), ("fft_blocks", ctypes.c_int),
                ("near_items", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class NativeLibraryMissing(RuntimeError):
    pass


_lib = None


def load(path: str = LIB_PATH):
    """Load libfemnfft.so; raises NativeLibraryMissing when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise NativeLibraryMissing(
            f"{path} not found: build it with `python -m paper_0807_2387_gb300.build` "
            "(there is no fallback implementation)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I64, I32, D = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "fs_plan_create": [P, I64, P, I64, I32, D, I32, D, ctypes.POINTER(FsOpts), PP],
        "fs_plan_create_fem": [P, I64, P, I64, I32, D, I32, D, ctypes.POINTER(FsOpts), PP],
        "fs_set_charges": [P, P, I32, I32],
        "fs_set_magnetization": [P, P, I32],
        "fs_set_magnetization_static": [P, P, I32],
        "fs_fem_charges": [P, P, P, I32],
        "fs_fem_sources": [P, P],
        "fs_eval_potential": [P, P, I32],
        "fs_eval_field": [P, P, P, I32],
        "fs_solve_host": [P, P, I32, I32, P, P, I32],
        "fs_adjoint": [P, P, P, I32, P, P, P, I32],
        "fs_sync_status": [P],
        "fs_plan_info": [P, ctypes.POINTER(FsInfo)],
        "fs_stage_times": [P, ctypes.POINTER(ctypes.c_double), I32],
        "fs_plan_destroy": [P],
        "fs_batch_create": [ctypes.POINTER(FsInstance), I32, D, I32, I32, ctypes.POINTER(FsOpts), PP],
        "fs_batch_eval": [P, PP, I32, PP, PP, I32],
        "fs_batch_sync_status": [P],
        "fs_batch_info": [P, ctypes.POINTER(FsBatchFacts)],
        "fs_batch_plan": [P, I32, PP],
        "fs_batch_destroy": [P],
        "fs_wait_selftest": [I32],
        "fs_probe_throughput": [I32, I32, I32, ctypes.POINTER(D), ctypes.POINTER(D)],
        "fs3_plan_create": [P, I64, P, I64, I32, D, I32, D, ctypes.POINTER(FsOpts), PP],
        "fs3_set_charges": [P, P, I32, I32],
        "fs3_eval_field": [P, P, P, I32],
        "fs3_sync_status": [P],
        "fs3_plan_info": [P, ctypes.POINTER(FsInfo)],
        "fs3_plan_destroy": [P],
        "fs3_plan_create_fem": [P, I64, P, I64, I32, D, I32, D, ctypes.POINTER(FsOpts), PP],
        "fs3_set_magnetization": [P, P, I32],
        "fs3_fem_charges": [P, P, P, I32],
        "fs3_fem_sources": [P, P],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.fs_last_error.argtypes = []
    lib.fs_last_error.restype = ctypes.c_char_p
    lib.fs_version.argtypes = []
    lib.fs_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


class FastSumError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int, where: str):
    if status != FS_OK:
        msg = load().fs_last_error().decode(errors="replace")
        raise FastSumError(status, where, msg)
