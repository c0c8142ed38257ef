"""CPU oracle for the sparse-vector KNN join -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library and never imports
it; inputs come from the caller as CSR arrays (any object with ``indptr``,
``indices``, ``values`` and ``dim``).

Functions (all return ``ids`` int32 [n, k], ``scores`` float64 [n, k], ``stats``):

* :func:`bf_join`   -- the plain definition (Section 3, eq. 1): every dot(r, s) by the
  two-pointer merge of Algorithm 2, positive scores ordered by (score desc, id asc),
  first k, padded with (-1, 0).
* :func:`iib_join`  -- Algorithm 3 inside the block nested loop of Algorithm 1.
* :func:`iiib_join` -- Algorithm 4 inside the block nested loop of Algorithm 1.

uint8 scores are exact integers held in float64 (every partial sum is below 2^53);
float32 inputs give fp64 reference scores.

Parity status: every function is pinned by ``tests/test_oracle_pins.py`` (hand-worked
examples, dense int64 matmul + stable sort, brute force on tiny inputs, Theorem 1
equivalences, the exact posting count of eq. 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _CSR(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("dim", ctypes.c_int32),
                ("indptr", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("postings_touched", ctypes.c_int64), ("postings_indexed", ctypes.c_int64),
                ("merge_steps", ctypes.c_int64), ("residual_dots", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            lib.oracle_bf_join.argtypes = [P(_CSR), P(_CSR), ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, P(_Stats)]
            for name in ("oracle_iib_join", "oracle_iiib_join"):
                getattr(lib, name).argtypes = [P(_CSR), P(_CSR), ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p, P(_Stats)]
            _lib = lib
    return _lib


def _as_csr(x, keep):
    indptr = np.ascontiguousarray(x.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(x.indices, dtype=np.int32)
    values = np.ascontiguousarray(x.values)
    if values.dtype == np.uint8:
        dt = 0
    elif values.dtype == np.float32:
        dt = 1
    else:
        raise TypeError("values must be uint8 or float32")
    keep.extend([indptr, indices, values])
    return _CSR(indptr.shape[0] - 1, int(x.dim), indptr.ctypes.data, indices.ctypes.data,
                values.ctypes.data, dt)


def _run(fn, R, S, k, *extra):
    if k < 1:
        raise ValueError("k must be >= 1")
    keep = []
    cr, cs = _as_csr(R, keep), _as_csr(S, keep)
    n = cr.n_rows
    ids = np.full((n, k), -1, dtype=np.int32)
    sc = np.zeros((n, k), dtype=np.float64)
    st = _Stats()
    rc = fn(ctypes.byref(cr), ctypes.byref(cs), k, *extra, ids.ctypes.data, sc.ctypes.data,
            ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"oracle returned {rc}")
    stats = {f: int(getattr(st, f)) for f, _ in _Stats._fields_}
    return ids, sc, stats


def bf_join(R, S, k: int, threads: int = 1):
    """Plain definition: merge-dot every (r, s), sort positive scores, first k."""
    return _run(_load().oracle_bf_join, R, S, k, int(threads))


def iib_join(R, S, k: int, rblock: int = 0, sblock: int = 0, threads: int = 0):
    """Algorithm 3 (IIB) in the block nested loop join; 0 block size = whole set."""
    return _run(_load().oracle_iib_join, R, S, k, int(rblock), int(sblock), int(threads))


def iiib_join(R, S, k: int, rblock: int = 0, sblock: int = 0, threads: int = 0):
    """Algorithm 4 (IIIB) in the block nested loop join; 0 block size = whole set."""
    return _run(_load().oracle_iiib_join, R, S, k, int(rblock), int(sblock), int(threads))
