"""Oracle O1 loader: builds ``direct.c`` with gcc (+OpenMP) and calls it via ctypes.

Test infrastructure only (see ``oracle/__init__``).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_direct.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile the direct-sum oracle (gcc -O2, OpenMP if available); returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.o1_direct.argtypes = [dp, ctypes.c_long, dp, ctypes.c_long, dp, dp, dp, dp]
            lib.o1_direct.restype = None
            lib.o1_threads.restype = ctypes.c_int
            lib.o1_adjoint.argtypes = [dp, ctypes.c_long, dp, ctypes.c_long, dp, dp, dp, dp, dp, dp]
            lib.o1_adjoint.restype = None
            _handle = lib
    return _handle


def _ptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    """OpenMP threads the direct sum uses (OMP_NUM_THREADS, else all cores)."""
    return int(_lib().o1_threads())


def direct_sum(tgt, src, q, field: bool = True, hessian: bool = False):
    """phi (N,), H (N,2) and optionally the Hessian of phi (N,3: xx, xy, yy), physical units."""
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n_t, n_s = len(tgt), len(src)
    phi = np.zeros(n_t)
    fld = np.zeros((n_t, 2)) if field else None
    hes = np.zeros((n_t, 3)) if hessian else None
    _lib().o1_direct(_ptr(tgt), n_t, _ptr(src), n_s, _ptr(q), _ptr(phi), _ptr(fld), _ptr(hes))
    out = [phi]
    if field:
        out.append(fld)
    if hessian:
        out.append(hes)
    return tuple(out) if len(out) > 1 else phi


def direct_adjoint(tgt, src, q, gphi, gH):
    """Gradients of L(phi, H) through the direct sum: (dL/dq (M,), dL/dy (M,2), dL/dx (N,2))."""
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    gphi = np.ascontiguousarray(gphi, dtype=np.float64)
    gH = np.ascontiguousarray(gH, dtype=np.float64)
    dq = np.zeros(len(src))
    dy = np.zeros((len(src), 2))
    dx = np.zeros((len(tgt), 2))
    _lib().o1_adjoint(_ptr(tgt), len(tgt), _ptr(src), len(src), _ptr(q), _ptr(gphi), _ptr(gH),
                      _ptr(dq), _ptr(dy), _ptr(dx))
    return dq, dy, dx
