"""The paper's own CPU method (§2.3, in the threaded form of §3), from ``paper_method.c``.

TEST AND BASELINE INFRASTRUCTURE (same rule as the rest of ``oracle/``):
the tests cross-check it against the sort-based oracle, and the benchmark's
CPU leg times it on the host cores.  Built with ``-fopenmp`` when gcc
accepts it; without OpenMP the threaded routine runs on one thread.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

from . import ERR_NOMEM, OK, Result, _BUILD, _HERE, _f64, _i32, _p, dims

_SRC = os.path.join(_HERE, "paper_method.c")
_SO = os.path.join(_BUILD, "libpaper_method.so")
_lib = None
openmp = None   # True / False once built


def build(force: bool = False) -> str:
    """Compile ``paper_method.c`` (with OpenMP when available)."""
    global openmp
    os.makedirs(_BUILD, exist_ok=True)
    stamp = _SO + ".openmp"
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
            openmp = True
        except (subprocess.CalledProcessError, OSError):
            subprocess.check_call(base)
            openmp = False
        os.replace(tmp, _SO)
        with open(stamp, "w") as f:
            f.write("1" if openmp else "0")
    elif openmp is None:
        openmp = os.path.exists(stamp) and open(stamp).read().strip() == "1"
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.paper_max_threads.argtypes = []
        lib.paper_max_threads.restype = ctypes.c_int
        lib.paper_sparse_omp.argtypes = [i32p, i32p, f64p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int, i32p, i32p, i32p, f64p,
                                         ctypes.POINTER(ctypes.c_int)]
        lib.paper_sparse_omp.restype = ctypes.c_int64
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().paper_max_threads())


def assemble(ii, jj, s=None, m: int = 0, n: int = 0, threads: Optional[int] = None,
             want_irank: bool = True):
    """``sparse(i, j, s, m, n)`` by the paper's method -> (Result, threads used).

    ``threads=None`` runs the method on one thread (the serial method of
    §2.3); an integer runs the threaded form (§3) on that many threads
    (0 = all available).
    """
    ii, jj = _i32(ii), _i32(jj)
    if s is not None:
        s = _f64(s)
    st, m, n = dims(ii, jj, m, n)
    if st != OK:
        return Result(st), 0
    L = ii.size
    irank = np.empty(max(L, 1), np.int32) if want_irank else None
    jcS = np.empty(n + 1, np.int32)
    irS = np.empty(max(L, 1), np.int32)
    prS = np.empty(max(L, 1), np.float64) if s is not None else None
    lib = _load()
    t = ctypes.c_int(0)
    nnz = lib.paper_sparse_omp(_p(ii, ctypes.c_int32), _p(jj, ctypes.c_int32),
                               _p(s, ctypes.c_double), L, m, n, 1 if threads is None else int(threads),
                               _p(irank, ctypes.c_int32), _p(jcS, ctypes.c_int32),
                               _p(irS, ctypes.c_int32), _p(prS, ctypes.c_double), ctypes.byref(t))
    used = t.value
    if nnz < 0:
        return Result(ERR_NOMEM), used
    nnz = int(nnz)
    return Result(OK, m, n, nnz, nnz, irank[:L] if irank is not None else None, jcS,
                  irS[:nnz].copy(), prS[:nnz].copy() if prS is not None else None), used
