"""CPU oracle for the Lu-Lin DIST method (arXiv 2309.09072) -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
(and ``--impl reference``) arm may import this package.  The GPU library does
not load it, and it shares no code with the GPU library: the arithmetic lives
in ``lcs_oracle.c`` (plain C, compiled with gcc by :func:`build`), and this
module only marshals numpy arrays into it.

Conventions: ``a`` (length m) labels the grid rows, ``b`` (length n) the
columns; ``DIST(i, j) = LCS(a, b[i:j])`` for ``j >= i`` and ``INT32_MIN``
below the diagonal; breakout (D-form) matrices use ``INF = 2**63 - 1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcs_oracle.c")
_LIB = os.path.join(_HERE, "liblcs_oracle.so")
_lock = threading.Lock()
_lib = None

NEG_INF = np.iinfo(np.int32).min
INF = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    """Compile ``lcs_oracle.c`` into ``liblcs_oracle.so`` (gcc, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i64 = ctypes.c_int64
            lib.oracle_lcs_length.argtypes = [u8p, i64, u8p, i64]
            lib.oracle_lcs_length.restype = i64
            lib.oracle_dist_row.argtypes = [u8p, i64, u8p, i64, i64, i32p]
            lib.oracle_dist_row.restype = ctypes.c_int
            lib.oracle_dist.argtypes = [u8p, i64, u8p, i64, i32p, i64, ctypes.c_int]
            lib.oracle_dist.restype = ctypes.c_int
            lib.oracle_dist_rows.argtypes = [u8p, i64, u8p, i64, i64p, i64, i32p, ctypes.c_int]
            lib.oracle_dist_rows.restype = ctypes.c_int
            lib.oracle_merge.argtypes = [i32p, i32p, i64, i64, i32p, i32p]
            lib.oracle_merge.restype = None
            lib.oracle_traceback.argtypes = [u8p, i64, u8p, i64, u8p, i64p]
            lib.oracle_traceback.restype = i64
            lib.oracle_path.argtypes = [u8p, i64, u8p, i64, i64p, i64p]
            lib.oracle_path.restype = i64
            lib.oracle_dform.argtypes = [i32p, i64, i64, i64, i64p]
            lib.oracle_dform.restype = None
            lib.oracle_leaf_dform.argtypes = [ctypes.c_uint8, u8p, i64, i64p, i64p]
            lib.oracle_leaf_dform.restype = None
            lib.oracle_dform_combine.argtypes = [i64p, i64, i64p, i64, i64, i64p]
            lib.oracle_dform_combine.restype = None
            _lib = lib
    return _lib


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        x = np.frombuffer(bytes(x), dtype=np.uint8)
    elif isinstance(x, str):
        x = np.frombuffer(x.encode("latin-1"), dtype=np.uint8)
    return np.ascontiguousarray(x, dtype=np.uint8)


def _p(arr, ctype):
    if arr is None:
        return None
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def lcs_length(a, b) -> int:
    """Textbook two-row DP length (Sec. I)."""
    a, b = _u8(a), _u8(b)
    r = _load().oracle_lcs_length(_p(a, ctypes.c_uint8), len(a), _p(b, ctypes.c_uint8), len(b))
    if r < 0:
        raise MemoryError("oracle_lcs_length")
    return int(r)


def dist(a, b, nthreads: int = 0) -> np.ndarray:
    """Full (n+1) x (n+1) int32 DIST by the per-source DP."""
    a, b = _u8(a), _u8(b)
    n = len(b)
    out = np.empty((n + 1, n + 1), dtype=np.int32)
    r = _load().oracle_dist(_p(a, ctypes.c_uint8), len(a), _p(b, ctypes.c_uint8), n,
                            _p(out, ctypes.c_int32), n + 1, int(nthreads))
    if r < 0:
        raise MemoryError("oracle_dist")
    return out


def dist_rows(a, b, rows, nthreads: int = 0) -> np.ndarray:
    """Rows ``rows`` of DIST, shape (len(rows), n+1)."""
    a, b = _u8(a), _u8(b)
    n = len(b)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() > n):
        raise ValueError("row out of range")
    out = np.empty((len(rows), n + 1), dtype=np.int32)
    if len(rows) == 0:
        return out
    r = _load().oracle_dist_rows(_p(a, ctypes.c_uint8), len(a), _p(b, ctypes.c_uint8), n,
                                 _p(rows, ctypes.c_int64), len(rows), _p(out, ctypes.c_int32),
                                 int(nthreads))
    if r < 0:
        raise MemoryError("oracle_dist_rows")
    return out


def merge(U: np.ndarray, L: np.ndarray):
    """Brute-force (max,+) merge with leftmost argmax; returns (D, K)."""
    U = np.ascontiguousarray(U, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.int32)
    if U.shape != L.shape or U.shape[0] != U.shape[1]:
        raise ValueError("U and L must be equal square matrices")
    n = U.shape[0] - 1
    D = np.empty_like(U)
    K = np.empty_like(U)
    _load().oracle_merge(_p(U, ctypes.c_int32), _p(L, ctypes.c_int32), n, n + 1,
                         _p(D, ctypes.c_int32), _p(K, ctypes.c_int32))
    return D, K


def traceback(a, b):
    """Leftmost-path LCS; returns (lcs_bytes, v) with v the cross vertices."""
    a, b = _u8(a), _u8(b)
    m = len(a)
    out = np.zeros(max(1, min(m, len(b))), dtype=np.uint8)
    v = np.zeros(m + 1, dtype=np.int64)
    r = _load().oracle_traceback(_p(a, ctypes.c_uint8), m, _p(b, ctypes.c_uint8), len(b),
                                 _p(out, ctypes.c_uint8), _p(v, ctypes.c_int64))
    if r < 0:
        raise MemoryError("oracle_traceback")
    return bytes(out[:r]), v


def path(a, b) -> np.ndarray:
    """Vertices (row, col) of the leftmost heaviest path, (0, 0) to (m, n)."""
    a, b = _u8(a), _u8(b)
    m, n = len(a), len(b)
    rows = np.zeros(m + n + 1, dtype=np.int64)
    cols = np.zeros(m + n + 1, dtype=np.int64)
    r = _load().oracle_path(_p(a, ctypes.c_uint8), m, _p(b, ctypes.c_uint8), n,
                            _p(rows, ctypes.c_int64), _p(cols, ctypes.c_int64))
    if r < 0:
        raise MemoryError("oracle_path")
    return np.stack([rows[:r], cols[:r]], axis=1)


def dform(D: np.ndarray, wmax: int) -> np.ndarray:
    """DIST -> breakout matrix (n+1) x (wmax+1), INF where unreachable."""
    D = np.ascontiguousarray(D, dtype=np.int32)
    n = D.shape[0] - 1
    out = np.empty((n + 1, wmax + 1), dtype=np.int64)
    _load().oracle_dform(_p(D, ctypes.c_int32), n, D.shape[1], int(wmax), _p(out, ctypes.c_int64))
    return out


def leaf_dform(ah: int, b):
    """Two-row leaf by the paper's construction; returns (D_1based, gaps)."""
    b = _u8(b)
    n = len(b)
    out = np.empty(n, dtype=np.int64)
    gaps = np.empty(n, dtype=np.int64)
    _load().oracle_leaf_dform(int(ah) & 0xFF, _p(b, ctypes.c_uint8), n,
                              _p(out, ctypes.c_int64), _p(gaps, ctypes.c_int64))
    return out, gaps


def dform_combine(DU: np.ndarray, DL: np.ndarray) -> np.ndarray:
    """The paper's breakout-matrix combination of an upper and a lower half."""
    DU = np.ascontiguousarray(DU, dtype=np.int64)
    DL = np.ascontiguousarray(DL, dtype=np.int64)
    n = DU.shape[0] - 1
    wu, wl = DU.shape[1] - 1, DL.shape[1] - 1
    out = np.empty((n + 1, wu + wl + 1), dtype=np.int64)
    _load().oracle_dform_combine(_p(DU, ctypes.c_int64), wu, _p(DL, ctypes.c_int64), wl, n,
                                 _p(out, ctypes.c_int64))
    return out
