"""CPU oracle for exact DBSCAN — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never calls it, and it shares
no code with the CUDA library.

``dbscan`` wraps the plain brute-force C implementation in ``dbscan_oracle.c``
(Section II's definitions, the serial three-step outline of Section II, and the
``<= eps^2`` test of Section IV-B).  ``bfs.py`` holds a second, independent
implementation (classic expand-cluster) used only to cross-check this one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dbscan_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERR_ARG = 1
ERR_NOT_QUANTISED = 2
ERR_OOM = 3

MUT_STRICT_LESS = 1
MUT_NO_SELF = 2
MUT_BORDER_MAX = 4
MUT_NO_UNION = 8


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP over rows)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
            lib.oracle_quantise.argtypes = [p, i64, i32, p]
            lib.oracle_quantise.restype = ctypes.c_int
            lib.oracle_threshold.argtypes = [ctypes.c_float]
            lib.oracle_threshold.restype = i64
            lib.oracle_counts.argtypes = [p, i64, i32, i64, i64, i64, p, i32, i32]
            lib.oracle_counts.restype = ctypes.c_int
            lib.oracle_dbscan.argtypes = [p, i64, i32, ctypes.c_float, i32, i32, p, p, p, i32, i32]
            lib.oracle_dbscan.restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status}")
        self.status = status


def threshold(eps: float) -> int:
    """T = floor(eps^2 * 2^20), eps taken as float32."""
    return int(_load().oracle_threshold(ctypes.c_float(eps)))


def quantise(points: np.ndarray) -> np.ndarray:
    """Integer grid units u = 1024 x; raises OracleError(2) off the 2^-10 grid."""
    x = np.ascontiguousarray(points, dtype=np.float32)
    n, d = x.shape
    u = np.empty((n, d), dtype=np.int32)
    st = _load().oracle_quantise(x.ctypes.data, n, d, u.ctypes.data)
    if st:
        raise OracleError(st)
    return u


def counts(points: np.ndarray, eps: float, rows: slice | None = None, nthreads: int = 0,
           mutation: int = 0) -> np.ndarray:
    """Neighbour counts (self included) of ``rows`` against all points."""
    u = quantise(points)
    n, d = u.shape
    r0, r1, _ = (rows or slice(0, n)).indices(n)
    out = np.empty(max(r1 - r0, 0), dtype=np.int32)
    st = _load().oracle_counts(u.ctypes.data, n, d, threshold(eps), r0, r1, out.ctypes.data,
                               nthreads, mutation)
    if st:
        raise OracleError(st)
    return out


def dbscan(points: np.ndarray, eps: float, min_pts: int, label_mode: int = 0, nthreads: int = 0,
           mutation: int = 0):
    """Exact DBSCAN. Returns (labels int32[n], counts int32[n], core bool[n]).

    label_mode 0: a cluster's id is its smallest core index; 1: ids 0..k-1 in
    that order.  Noise is -1.
    """
    x = np.ascontiguousarray(points, dtype=np.float32)
    n, d = x.shape
    labels = np.empty(n, dtype=np.int32)
    cnt = np.empty(n, dtype=np.int32)
    core = np.empty(n, dtype=np.uint8)
    st = _load().oracle_dbscan(x.ctypes.data, n, d, ctypes.c_float(eps), int(min_pts), int(label_mode),
                               labels.ctypes.data, cnt.ctypes.data, core.ctypes.data, int(nthreads),
                               int(mutation))
    if st:
        raise OracleError(st)
    return labels, cnt, core.astype(bool)
