"""CPU oracle for batched X-drop seed extension -- TEST INFRASTRUCTURE ONLY.

Loads ``xdrop_oracle.c`` (linear gaps, the paper's method),
``xdrop_affine_oracle.c`` (the same extension with affine gaps),
``xdrop_traceback_oracle.c`` (alignment paths) and ``xdrop_matrix_oracle.c``
(any alphabet scored by a substitution matrix, affine gaps), compiled
with the host C compiler into ``oracle/_build/liboracle.so`` through ctypes.  Only the tests, the smoke
check and the CPU-baseline leg of ``bench.py`` may use it; the library and
its Python binding never import it.  It shares no code with the CUDA path.

Every function follows the passages and readings listed at the top of
``xdrop_oracle.c`` (``affine_*``: of ``xdrop_affine_oracle.c``).  Parity
status: pinned (brute-force full DP at X = inf, closed forms, invariants
and hand-derived worked examples in tests/; the affine extension also
against the linear one at gap_open = 0).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xdrop_oracle.c")
_SRC_AFFINE = os.path.join(_HERE, "xdrop_affine_oracle.c")
_SRC_TRACE = os.path.join(_HERE, "xdrop_traceback_oracle.c")
_SRC_MATRIX = os.path.join(_HERE, "xdrop_matrix_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OK, INVALID, NOMEM = 0, 1, 2

PAIR_DTYPE = np.dtype([("score", "<i8"), ("left", "<i8"), ("right", "<i8"),
                       ("begA", "<i8"), ("begB", "<i8"), ("endA", "<i8"),
                       ("endB", "<i8"), ("cells", "<i8"), ("status", "<i8")])


class _Ext(ctypes.Structure):
    _fields_ = [("best", ctypes.c_int64), ("bi", ctypes.c_int64),
                ("bj", ctypes.c_int64), ("cells", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (gcc -O2, no -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                              os.path.getmtime(_SRC_AFFINE),
                                              os.path.getmtime(_SRC_TRACE),
                                              os.path.getmtime(_SRC_MATRIX)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, _SRC_AFFINE, _SRC_TRACE, _SRC_MATRIX])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        L.oracle_xdrop_extend.argtypes = [p, i64, p, i64, i64, i64, i64, i64,
                                          ctypes.POINTER(_Ext)]
        L.oracle_xdrop_extend.restype = ctypes.c_int
        L.oracle_pair.argtypes = [p, i64, p, i64, i64, i64, i64, i64, i64, i64, i64, p]
        L.oracle_pair.restype = ctypes.c_int
        L.oracle_batch.argtypes = [p, p, p, ctypes.c_uint32, p, p, p, ctypes.c_uint32,
                                   p, i64, i64, i64, i64, i64, p, ctypes.c_int, p]
        L.oracle_batch.restype = ctypes.c_int
        L.oracle_params_valid.argtypes = [i64, i64, i64, i64]
        L.oracle_params_valid.restype = ctypes.c_int
        L.oracle_affine_extend.argtypes = [p, i64, p, i64, i64, i64, i64, i64, i64,
                                           ctypes.POINTER(_Ext)]
        L.oracle_affine_extend.restype = ctypes.c_int
        L.oracle_affine_pair.argtypes = [p, i64, p, i64, i64, i64, i64, i64, i64, i64, i64,
                                         i64, p]
        L.oracle_affine_pair.restype = ctypes.c_int
        L.oracle_affine_batch.argtypes = [p, p, p, ctypes.c_uint32, p, p, p, ctypes.c_uint32,
                                          p, i64, i64, i64, i64, i64, i64, p, ctypes.c_int, p]
        L.oracle_affine_batch.restype = ctypes.c_int
        L.oracle_affine_params_valid.argtypes = [i64, i64, i64, i64, i64]
        L.oracle_affine_params_valid.restype = ctypes.c_int
        pi64 = ctypes.POINTER(i64)
        L.oracle_xdrop_traceback.argtypes = [p, i64, p, i64, i64, i64, i64, i64, pi64, pi64, pi64,
                                             pi64, p, pi64]
        L.oracle_xdrop_traceback.restype = ctypes.c_int
        L.oracle_pair_traceback.argtypes = [p, i64, p, i64, i64, i64, i64, i64, i64, i64, i64, p,
                                            pi64]
        L.oracle_pair_traceback.restype = ctypes.c_int
        L.oracle_matrix_extend.argtypes = [p, i64, p, i64, p, i64, i64, i64, i64,
                                           ctypes.POINTER(_Ext)]
        L.oracle_matrix_extend.restype = ctypes.c_int
        L.oracle_matrix_pair.argtypes = [p, i64, p, i64, i64, i64, i64, p, i64, i64, i64, i64, p]
        L.oracle_matrix_pair.restype = ctypes.c_int
        L.oracle_matrix_batch.argtypes = [p, p, p, ctypes.c_uint32, p, p, p, ctypes.c_uint32,
                                          p, i64, p, i64, i64, i64, i64, p, ctypes.c_int, p]
        L.oracle_matrix_batch.restype = ctypes.c_int
        L.oracle_matrix_params_valid.argtypes = [p, i64, i64, i64, i64]
        L.oracle_matrix_params_valid.restype = ctypes.c_int
        _lib = L
    return _lib


def _buf(x: bytes):
    return ctypes.c_char_p(x) if x else ctypes.c_char_p(b"")


def extend(a: bytes, b: bytes, match: int = 1, mismatch: int = -1, gap: int = -1,
           X: int = 50):
    """One X-drop extension of a against b (both read forwards from cell (0,0)).

    Returns (best, bi, bj, cells): best score >= 0, the number of bases of a and
    b consumed at the best cell, and the computed-cell count.
    """
    out = _Ext()
    rc = lib().oracle_xdrop_extend(_buf(a), len(a), _buf(b), len(b), match, mismatch,
                                   gap, X, ctypes.byref(out))
    if rc:
        raise MemoryError("oracle extension could not allocate")
    return out.best, out.bi, out.bj, out.cells


def pair(A: bytes, B: bytes, posA: int, posB: int, k: int, match: int = 1,
         mismatch: int = -1, gap: int = -1, X: int = 50) -> np.void:
    """One seeded pair: left extension + seed + right extension (PAIR_DTYPE)."""
    r = np.zeros(1, dtype=PAIR_DTYPE)
    lib().oracle_pair(_buf(A), len(A), _buf(B), len(B), posA, posB, k, match, mismatch,
                      gap, X, r.ctypes.data)
    return r[0]


def params_valid(match: int, mismatch: int, gap: int, X: int) -> bool:
    return bool(lib().oracle_params_valid(match, mismatch, gap, X))


def batch(poolA: np.ndarray, offA: np.ndarray, lenA: np.ndarray,
          poolB: np.ndarray, offB: np.ndarray, lenB: np.ndarray,
          seeds: np.ndarray, match: int, mismatch: int, gap: int, X: int,
          Xs: Optional[np.ndarray] = None, threads: Optional[int] = None):
    """Every pair of a batch, one pair per task over `threads` host threads.

    seeds: structured array of (idxA, idxB, posA, posB, len) uint32 records.
    Returns (results as PAIR_DTYPE array, threads used).
    """
    poolA = np.ascontiguousarray(poolA, dtype=np.uint8)
    poolB = np.ascontiguousarray(poolB, dtype=np.uint8)
    offA = np.ascontiguousarray(offA, dtype=np.uint64)
    offB = np.ascontiguousarray(offB, dtype=np.uint64)
    lenA = np.ascontiguousarray(lenA, dtype=np.uint32)
    lenB = np.ascontiguousarray(lenB, dtype=np.uint32)
    sd = np.ascontiguousarray(
        np.stack([seeds[f] for f in ("idxA", "idxB", "posA", "posB", "len")], axis=1)
        .astype(np.uint32))
    n = sd.shape[0]
    out = np.zeros(n, dtype=PAIR_DTYPE)
    xs = None if Xs is None else np.ascontiguousarray(Xs, dtype=np.int32)
    if threads is None:
        threads = os.cpu_count() or 1
    used = lib().oracle_batch(poolA.ctypes.data, offA.ctypes.data, lenA.ctypes.data,
                              lenA.size, poolB.ctypes.data, offB.ctypes.data,
                              lenB.ctypes.data, lenB.size, sd.ctypes.data, n,
                              match, mismatch, gap, X,
                              None if xs is None else xs.ctypes.data, int(threads),
                              out.ctypes.data)
    return out, used


def run_batch(b, threads: Optional[int] = None):
    """Convenience wrapper for a synth.Batch-like object (ASCII pools; take
    a subset of a packed batch first)."""
    if getattr(b, "packed", False):
        raise ValueError("the oracle reads ASCII pools: use b.subset(...) of a packed batch")
    return batch(b.poolA, b.offA, b.lenA, b.poolB, b.offB, b.lenB, b.seeds, b.match,
                 b.mismatch, b.gap, b.X, b.Xs, threads)


# ---- affine gaps (xdrop_affine_oracle.c) ----

def affine_extend(a: bytes, b: bytes, match: int = 1, mismatch: int = -1, gap_open: int = -2,
                  gap_extend: int = -1, X: int = 50):
    """One affine-gap X-drop extension (a gap of length L scores
    gap_open + L * gap_extend).  Returns (best, bi, bj, cells)."""
    out = _Ext()
    rc = lib().oracle_affine_extend(_buf(a), len(a), _buf(b), len(b), match, mismatch,
                                    gap_open, gap_extend, X, ctypes.byref(out))
    if rc:
        raise MemoryError("oracle extension could not allocate")
    return out.best, out.bi, out.bj, out.cells


def affine_pair(A: bytes, B: bytes, posA: int, posB: int, k: int, match: int = 1,
                mismatch: int = -1, gap_open: int = -2, gap_extend: int = -1,
                X: int = 50) -> np.void:
    r = np.zeros(1, dtype=PAIR_DTYPE)
    lib().oracle_affine_pair(_buf(A), len(A), _buf(B), len(B), posA, posB, k, match, mismatch,
                             gap_open, gap_extend, X, r.ctypes.data)
    return r[0]


def affine_params_valid(match: int, mismatch: int, gap_open: int, gap_extend: int,
                        X: int) -> bool:
    return bool(lib().oracle_affine_params_valid(match, mismatch, gap_open, gap_extend, X))


def run_batch_affine(b, gap_open: int, gap_extend: int, threads: Optional[int] = None):
    """Every pair of a synth.Batch-like object (ASCII pools) with affine gaps
    (b.gap is ignored).  Returns (PAIR_DTYPE results, threads used)."""
    if getattr(b, "packed", False):
        raise ValueError("the oracle reads ASCII pools: use b.subset(...) of a packed batch")
    poolA = np.ascontiguousarray(b.poolA, dtype=np.uint8)
    poolB = np.ascontiguousarray(b.poolB, dtype=np.uint8)
    offA = np.ascontiguousarray(b.offA, dtype=np.uint64)
    offB = np.ascontiguousarray(b.offB, dtype=np.uint64)
    lenA = np.ascontiguousarray(b.lenA, dtype=np.uint32)
    lenB = np.ascontiguousarray(b.lenB, dtype=np.uint32)
    sd = np.ascontiguousarray(
        np.stack([b.seeds[f] for f in ("idxA", "idxB", "posA", "posB", "len")], axis=1)
        .astype(np.uint32))
    n = sd.shape[0]
    out = np.zeros(n, dtype=PAIR_DTYPE)
    xs = None if b.Xs is None else np.ascontiguousarray(b.Xs, dtype=np.int32)
    if threads is None:
        threads = os.cpu_count() or 1
    used = lib().oracle_affine_batch(poolA.ctypes.data, offA.ctypes.data, lenA.ctypes.data,
                                     lenA.size, poolB.ctypes.data, offB.ctypes.data,
                                     lenB.ctypes.data, lenB.size, sd.ctypes.data, n,
                                     b.match, b.mismatch, gap_open, gap_extend, b.X,
                                     None if xs is None else xs.ctypes.data, int(threads),
                                     out.ctypes.data)
    return out, used


# ---- alignment paths (xdrop_traceback_oracle.c) ----

def traceback(a: bytes, b: bytes, match: int = 1, mismatch: int = -1, gap: int = -1,
              X: int = 50):
    """One extension with its path: (best, bi, bj, cells, ops) where ops is a
    string of 'M' / 'I' / 'D' from (0,0) to the best cell."""
    v = [ctypes.c_int64() for _ in range(5)]
    buf = ctypes.create_string_buffer(len(a) + len(b) + 1)
    rc = lib().oracle_xdrop_traceback(_buf(a), len(a), _buf(b), len(b), match, mismatch, gap, X,
                                      *[ctypes.byref(x) for x in v[:4]], buf, ctypes.byref(v[4]))
    if rc:
        raise MemoryError("oracle traceback could not allocate")
    return v[0].value, v[1].value, v[2].value, v[3].value, buf.raw[:v[4].value].decode()


def pair_traceback(A: bytes, B: bytes, posA: int, posB: int, k: int, match: int = 1,
                   mismatch: int = -1, gap: int = -1, X: int = 50) -> str:
    """A seeded pair's alignment as 'M' / 'I' / 'D' operations from
    (begA, begB) to (endA, endB)."""
    n = ctypes.c_int64()
    buf = ctypes.create_string_buffer(len(A) + len(B) + 1)
    rc = lib().oracle_pair_traceback(_buf(A), len(A), _buf(B), len(B), posA, posB, k, match,
                                     mismatch, gap, X, buf, ctypes.byref(n))
    if rc:
        raise ValueError("invalid pair or allocation failure")
    return buf.raw[:n.value].decode()


# ---- substitution matrix, any alphabet (xdrop_matrix_oracle.c) ----

def _matrix(M):
    M = np.ascontiguousarray(M, dtype=np.int32)
    if M.ndim != 2 or M.shape[0] != M.shape[1]:
        raise ValueError("the substitution matrix must be K x K")
    return M, M.shape[0]


def matrix_extend(a: bytes, b: bytes, M, gap_open: int = 0, gap_extend: int = -1, X: int = 50):
    """One X-drop extension of letter codes a against b (bytes of values
    0..K-1), scored by the K x K matrix M and affine gaps.
    Returns (best, bi, bj, cells)."""
    M, K = _matrix(M)
    out = _Ext()
    rc = lib().oracle_matrix_extend(_buf(a), len(a), _buf(b), len(b), M.ctypes.data, K,
                                    gap_open, gap_extend, X, ctypes.byref(out))
    if rc:
        raise MemoryError("oracle extension could not allocate")
    return out.best, out.bi, out.bj, out.cells


def matrix_pair(A: bytes, B: bytes, posA: int, posB: int, k: int, M, gap_open: int = 0,
                gap_extend: int = -1, X: int = 50) -> np.void:
    M, K = _matrix(M)
    r = np.zeros(1, dtype=PAIR_DTYPE)
    lib().oracle_matrix_pair(_buf(A), len(A), _buf(B), len(B), posA, posB, k, M.ctypes.data, K,
                             gap_open, gap_extend, X, r.ctypes.data)
    return r[0]


def matrix_params_valid(M, gap_open: int, gap_extend: int, X: int) -> bool:
    M, K = _matrix(M)
    return bool(lib().oracle_matrix_params_valid(M.ctypes.data, K, gap_open, gap_extend, X))


def run_batch_matrix(b, M, gap_open: int, gap_extend: int, threads: Optional[int] = None):
    """Every pair of a synth.Batch-like object whose pools hold letter codes
    (one byte each, values < K), scored by M with affine gaps (b.match,
    b.mismatch and b.gap are ignored).  Returns (PAIR_DTYPE results, threads)."""
    M, K = _matrix(M)
    poolA = np.ascontiguousarray(b.poolA, dtype=np.uint8)
    poolB = np.ascontiguousarray(b.poolB, dtype=np.uint8)
    offA = np.ascontiguousarray(b.offA, dtype=np.uint64)
    offB = np.ascontiguousarray(b.offB, dtype=np.uint64)
    lenA = np.ascontiguousarray(b.lenA, dtype=np.uint32)
    lenB = np.ascontiguousarray(b.lenB, dtype=np.uint32)
    sd = np.ascontiguousarray(
        np.stack([b.seeds[f] for f in ("idxA", "idxB", "posA", "posB", "len")], axis=1)
        .astype(np.uint32))
    n = sd.shape[0]
    out = np.zeros(n, dtype=PAIR_DTYPE)
    xs = None if b.Xs is None else np.ascontiguousarray(b.Xs, dtype=np.int32)
    if threads is None:
        threads = os.cpu_count() or 1
    used = lib().oracle_matrix_batch(poolA.ctypes.data, offA.ctypes.data, lenA.ctypes.data,
                                     lenA.size, poolB.ctypes.data, offB.ctypes.data,
                                     lenB.ctypes.data, lenB.size, sd.ctypes.data, n,
                                     M.ctypes.data, K, gap_open, gap_extend, b.X,
                                     None if xs is None else xs.ctypes.data, int(threads),
                                     out.ctypes.data)
    return out, used
