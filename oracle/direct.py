"""ctypes loader for the FP64 direct sum in direct.c (built with gcc -fopenmp).

TEST INFRASTRUCTURE (CPU oracle): only the tests, the smoke check and the
benchmark's CPU-baseline leg may use it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_direct.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile direct.c into a shared library next to it (plain gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        _lib.oracle_direct.argtypes = [p, p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, p,
                                       ctypes.c_int64, p, ctypes.c_int]
        _lib.oracle_direct_grad.argtypes = _lib.oracle_direct.argtypes
        _lib.oracle_max_threads.restype = ctypes.c_int
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _prep(points, q):
    pts = np.ascontiguousarray(points, dtype=np.float64)
    qq = np.ascontiguousarray(np.atleast_2d(q), dtype=np.complex128)
    return pts, qq


def direct(points, q, k: float, targets=None, nthreads: int = 0) -> np.ndarray:
    """phi at ``targets`` (default: all points); q [n] or [nrhs][n]; returns [nrhs][nt] (or [nt])."""
    pts, qq = _prep(points, q)
    n = pts.shape[0]
    tg = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    out = np.zeros((qq.shape[0], tg.shape[0]), dtype=np.complex128)
    _load().oracle_direct(pts.ctypes.data, qq.ctypes.data, n, qq.shape[0], float(k), tg.ctypes.data,
                          tg.shape[0], out.ctypes.data, int(nthreads))
    return out[0] if np.ndim(q) == 1 else out


def direct_grad(points, q, k: float, targets=None, nthreads: int = 0) -> np.ndarray:
    """grad phi at ``targets``: [nt, 3] (or [nrhs][nt][3]) complex."""
    pts, qq = _prep(points, q)
    n = pts.shape[0]
    tg = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    out = np.zeros((qq.shape[0], tg.shape[0], 3), dtype=np.complex128)
    _load().oracle_direct_grad(pts.ctypes.data, qq.ctypes.data, n, qq.shape[0], float(k), tg.ctypes.data,
                               tg.shape[0], out.ctypes.data, int(nthreads))
    return out[0] if np.ndim(q) == 1 else out
