"""CPU oracle for Matlab-compatible sparse assembly ``S = sparse(i,j,s,m,n,nzmax)``.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU library never
loads it and shares no code with it.

The arithmetic lives in ``oracle.c`` (the definition of the paper's result:
sort (j, i, k), sweep once, fold each run in ascending k from +0.0).  This
module compiles it with gcc, loads it with ctypes and adds the boundary
rules that the paper leaves to the caller:

* §2.2 (text before the input listing): a zero dimension is implicit, the
  largest index; App. A pre-processing rejects indices below 1.
* App. A pre-processing of Matlab's double index arrays (``getix``,
  ``assemble_f64``): a value below 1.0 or different from its ceiling is a
  bad index.  Reading for values the paper's ``int`` cannot hold: above
  2^31 - 1 is a bad index too.
* ``nzmax`` appears only in the call signature of §1.  Reading used here:
  0 means "exactly nnz"; nzmax >= nnz gives that capacity with the unused
  tail zero-filled (irS = 0, prS = +0.0); 0 < nzmax < nnz is an error.
* No value-based dropping: the paper defines every slot from the index
  pattern alone (Eqs. (2.2)-(2.3), nnz = 1 + max irank), so explicit zeros
  and sums that cancel to zero are kept.

Status codes (same numbering as the library's public header, restated):
OK 0, ERR_ARG 1, ERR_INDEX 2, ERR_NZMAX 3, ERR_SIZE 4, ERR_NOMEM 5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

OK, ERR_ARG, ERR_INDEX, ERR_NZMAX, ERR_SIZE, ERR_NOMEM = 0, 1, 2, 3, 4, 5
INT32_MAX = 2**31 - 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``oracle/_build/liboracle.so`` (plain gcc -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_dims.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    i32p, i32p]
        lib.oracle_dims.restype = ctypes.c_int
        lib.oracle_assemble.argtypes = [i32p, i32p, f64p, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_int32, i32p, i32p, i32p, f64p]
        lib.oracle_assemble.restype = ctypes.c_int64
        lib.oracle_numeric.argtypes = [i32p, f64p, ctypes.c_int64, ctypes.c_int64, f64p]
        lib.oracle_numeric.restype = None
        lib.oracle_adjoint.argtypes = [i32p, f64p, ctypes.c_int64, f64p]
        lib.oracle_adjoint.restype = None
        lib.oracle_getix.argtypes = [f64p, ctypes.c_int64, i32p]
        lib.oracle_getix.restype = ctypes.c_int64
        lib.oracle_set_mutation.argtypes = [ctypes.c_int]
        lib.oracle_set_mutation.restype = ctypes.c_int
        _lib = lib
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Result:
    """Outcome of one oracle assembly.  Arrays are None unless status == OK."""

    status: int
    m: int = 0
    n: int = 0
    nnz: int = 0
    cap: int = 0          # length of irS / prS (nnz, or nzmax when larger)
    irank: Optional[np.ndarray] = None   # int32[len], 0-based slot of triplet k
    jcS: Optional[np.ndarray] = None     # int32[n+1]
    irS: Optional[np.ndarray] = None     # int32[cap], 0-based rows
    prS: Optional[np.ndarray] = None     # float64[cap] (None for symbolic-only)


def getix(ival):
    """Double index array -> (number of bad values, int32 indices)."""
    ival = _f64(ival)
    out = np.empty(max(ival.size, 1), np.int32)
    bad = _load().oracle_getix(_p(ival, ctypes.c_double), ival.size, _p(out, ctypes.c_int32))
    return int(bad), out[: ival.size]


def assemble_f64(ii, jj, s=None, m: int = 0, n: int = 0, nzmax: int = 0) -> Result:
    """``sparse(i, j, s, m, n, nzmax)`` with Matlab's double index arrays."""
    ii, jj = _f64(ii), _f64(jj)
    if ii.shape != jj.shape:
        return Result(ERR_ARG)
    bi, i32 = getix(ii)
    bj, j32 = getix(jj)
    if bi or bj:
        return Result(ERR_INDEX)
    return assemble(i32, j32, s, m, n, nzmax)


def dims(ii, jj, m: int = 0, n: int = 0):
    """Validate indices and resolve implicit dimensions -> (status, m, n)."""
    ii, jj = _i32(ii), _i32(jj)
    if ii.shape != jj.shape:
        return ERR_ARG, 0, 0
    if ii.size > INT32_MAX:
        return ERR_SIZE, 0, 0
    mo, no = ctypes.c_int32(0), ctypes.c_int32(0)
    st = _load().oracle_dims(_p(ii, ctypes.c_int32), _p(jj, ctypes.c_int32), ii.size,
                             int(m), int(n), ctypes.byref(mo), ctypes.byref(no))
    return st, mo.value, no.value


def assemble(ii, jj, s=None, m: int = 0, n: int = 0, nzmax: int = 0) -> Result:
    """``S = sparse(i, j, s, m, n, nzmax)`` by definition (unit-offset i, j).

    With ``s is None`` only the symbolic part (irank, jcS, irS) is formed.
    """
    ii, jj = _i32(ii), _i32(jj)
    if nzmax < 0:
        return Result(ERR_ARG)
    if s is not None:
        s = _f64(s)
        if s.shape != ii.shape:
            return Result(ERR_ARG)
    st, m, n = dims(ii, jj, m, n)
    if st != OK:
        return Result(st)
    L = ii.size
    irank = np.empty(L, np.int32)
    jcS = np.empty(n + 1, np.int32)
    irS = np.empty(max(L, 1), np.int32)
    prS = np.empty(max(L, 1), np.float64) if s is not None else None
    nnz = _load().oracle_assemble(_p(ii, ctypes.c_int32), _p(jj, ctypes.c_int32),
                                  _p(s, ctypes.c_double), L, m, n, _p(irank, ctypes.c_int32),
                                  _p(jcS, ctypes.c_int32), _p(irS, ctypes.c_int32),
                                  _p(prS, ctypes.c_double))
    if nnz < 0:
        return Result(ERR_NOMEM)
    if nzmax and nzmax < nnz:
        return Result(ERR_NZMAX, m, n, nnz)
    cap = max(nnz, nzmax)
    irS_out = np.zeros(cap, np.int32)
    irS_out[:nnz] = irS[:nnz]
    prS_out = None
    if prS is not None:
        prS_out = np.zeros(cap, np.float64)
        prS_out[:nnz] = prS[:nnz]
    return Result(OK, m, n, int(nnz), int(cap), irank, jcS, irS_out, prS_out)


def numeric(irank, s, nnz: int) -> np.ndarray:
    """prS from a symbolic map: +0.0, then prS[irank[k]] += s[k] for ascending k."""
    irank, s = _i32(irank), _f64(s)
    prS = np.empty(max(nnz, 1), np.float64)
    _load().oracle_numeric(_p(irank, ctypes.c_int32), _p(s, ctypes.c_double), irank.size,
                           int(nnz), _p(prS, ctypes.c_double))
    return prS[:nnz]


def adjoint(irank, dprS) -> np.ndarray:
    """ds[k] = dprS[irank[k]]: the transpose of the numeric scatter."""
    irank, dprS = _i32(irank), _f64(dprS)
    ds = np.empty(max(irank.size, 1), np.float64)
    _load().oracle_adjoint(_p(irank, ctypes.c_int32), _p(dprS, ctypes.c_double), irank.size,
                           _p(ds, ctypes.c_double))
    return ds[: irank.size]


def set_mutation(k: int) -> int:
    """Tests only: plant mistake number ``k`` in the oracle (0 restores it)."""
    return _load().oracle_set_mutation(int(k))
