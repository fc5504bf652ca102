"""Oracle: ctypes front of ``degrid.c`` (FP64 degridding sums).

Test infrastructure only (see ``oracle/__init__``).  ``build()`` compiles the
oracle's C files (``degrid.c``, ``exact.c``) with the host gcc (portable C99,
no intrinsics) into one library in ``oracle/_bin``; the first call builds it
if it is missing or older than a source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "degrid.c"), os.path.join(_HERE, "exact.c")]
_BIN = os.path.join(_HERE, "_bin")
_SO = os.path.join(_BIN, "liboracle_degrid.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BIN, exist_ok=True)
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(f) for f in _SRCS):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.oracle_degrid.argtypes = [ctypes.c_long, d, d, d, d, i, d, lp, i, ctypes.c_int,
                                      d, ctypes.c_int, ctypes.c_double, ctypes.c_int, d, d, d]
        lib.oracle_degrid.restype = None
        lib.oracle_exact_overlap.argtypes = [ctypes.c_long, d, d, d, ctypes.c_double, d, d, d]
        lib.oracle_exact_overlap.restype = None
        lib.oracle_exact_degrid.argtypes = [ctypes.c_long, d, d, d, d, d, d, d, i, ctypes.c_int, d,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int, d, d, d, d, d]
        lib.oracle_exact_degrid.restype = None
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def degrid_sums(u, v, L, M, tab_id, tables, grid, du, support, ov):
    """Per-visibility (T0, Tu, Tv), complex128 arrays shaped like ``u``.

    ``tables`` is a list of FP64 radial tables; ``tab_id`` picks one per visibility.
    """
    lib = _load()
    shape = np.shape(u)
    u = np.ascontiguousarray(np.ravel(u), dtype=np.float64)
    v = np.ascontiguousarray(np.ravel(v), dtype=np.float64)
    L = np.ascontiguousarray(np.ravel(L), dtype=np.float64)
    M = np.ascontiguousarray(np.ravel(M), dtype=np.float64)
    tid = np.ascontiguousarray(np.ravel(tab_id), dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate(tables), dtype=np.float64)
    lens = np.asarray([len(t) for t in tables], dtype=np.int32)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    g = np.ascontiguousarray(grid, dtype=np.complex128)
    n = u.size
    t0 = np.zeros(n, dtype=np.complex128)
    tu = np.zeros(n, dtype=np.complex128)
    tv = np.zeros(n, dtype=np.complex128)
    dp, ip, lp = ctypes.c_double, ctypes.c_int, ctypes.c_long
    lib.oracle_degrid(n, _p(u, dp), _p(v, dp), _p(L, dp), _p(M, dp), _p(tid, ip), _p(flat, dp),
                      _p(offs, lp), _p(lens, ip), int(ov), _p(g.view(np.float64), dp), g.shape[0],
                      float(du), int(support), _p(t0.view(np.float64), dp),
                      _p(tu.view(np.float64), dp), _p(tv.view(np.float64), dp))
    return t0.reshape(shape), tu.reshape(shape), tv.reshape(shape)
