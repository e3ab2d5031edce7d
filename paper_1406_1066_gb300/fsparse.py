"""Thin ctypes binding of libfsparse (the C ABI in include/fsparse.h).

Argument marshalling only: every step of the assembly runs in the CUDA
kernels of the library.  Two layers:

* ``fsparse_*`` functions with the C names take raw device pointers
  (ints), sizes and a stream handle, and return plain Python values; a
  non-OK status raises :class:`FsparseError`.
* Torch-level helpers (``symbolic``, ``numeric``, ``assemble``,
  ``Assemble``, ``Batch`` ...) check dtypes/devices, pass
  ``tensor.data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``,
  and wrap plan-owned device arrays as zero-copy tensors.

There is no CPU fallback: if the library is not built or cannot be loaded,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfsparse.so")

OK, ERR_ARG, ERR_INDEX, ERR_NZMAX, ERR_SIZE, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_INTERNAL = range(9)
SORT_AUTO, SORT_ONESWEEP, SORT_BUCKET, SORT_BUCKET_RADIX = 0, 1, 2, 3
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_INDEX", "ERR_NZMAX", "ERR_SIZE", "ERR_NOMEM", "ERR_CUDA",
                "ERR_TIMEOUT", "ERR_INTERNAL"]


class FsparseError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: FSPARSE_{name}: {message}")


class Config(ctypes.Structure):
    """Launch configuration (``fsparse_config``)."""

    _fields_ = [("strategy", ctypes.c_int32), ("radix_bits", ctypes.c_int32),
                ("sweep_items", ctypes.c_int32), ("sweep_threads", ctypes.c_int32),
                ("bucket_target", ctypes.c_int32), ("numeric_tile", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


def lib() -> ctypes.CDLL:
    """Load libfsparse.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1406_1066_gb300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "fsparse_symbolic": [_P, _P, _I64, _I32, _I32, _I64, _P, ctypes.POINTER(_P)],
        "fsparse_plan_info": [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I64),
                              ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
        "fsparse_plan_arrays": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)],
        "fsparse_plan_destroy": [_P],
        "fsparse_plan_release": [_P, _P],
        "fsparse_numeric": [_P, _P, _P, _P],
        "fsparse_numeric_adjoint": [_P, _P, _P, _P],
        "fsparse_assemble": [_P, _P, _P, _I64, _I32, _I32, _I64, _P, _I64, _P, ctypes.POINTER(_P)],
        "fsparse_symbolic_f64": [_P, _P, _I64, _I32, _I32, _I64, _P, ctypes.POINTER(_P)],
        "fsparse_plan_append": [_P, _P, _P, _I64, _P, ctypes.POINTER(_P)],
        "fsparse_plan_export": [_P, _P, _I64, ctypes.POINTER(_I64)],
        "fsparse_plan_import": [_P, _I64, _P, ctypes.POINTER(_P)],
        "fsparse_assemble_f64": [_P, _P, _P, _I64, _I32, _I32, _I64, _P, _I64, _P, ctypes.POINTER(_P)],
        "fsparse_batch_create": [_I32, ctypes.POINTER(_P), _P, ctypes.POINTER(_P)],
        "fsparse_batch_info": [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
        "fsparse_batch_symbolic": [_I32, _P, _P, ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                                   ctypes.POINTER(_I32), _P, ctypes.POINTER(_P)],
        "fsparse_batch_arrays": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                 ctypes.POINTER(_I32), ctypes.POINTER(_I32)],
        "fsparse_batch_numeric": [_P, _P, _P, _P],
        "fsparse_batch_destroy": [_P],
        "fsparse_batch_release": [_P, _P],
        "fsparse_get_config": [_I64, _I32, _I32, ctypes.POINTER(Config)],
        "fsparse_set_config": [ctypes.POINTER(Config)],
        "fsparse_autotune": [_P, _P, _P, _I64, _I32, _I32, _I32, _P, ctypes.POINTER(Config)],
        "fsparse_tune_save": [ctypes.c_char_p],
        "fsparse_tune_load": [ctypes.c_char_p],
        "fsparse_tune_clear": [],
        "fsparse_assemble_noalloc": [_P, _P, _P, _I64, _I32, _I32, _P, _P, _P, _P,
                                     ctypes.POINTER(_I64), _P],
        "fsparse_shard_route": [_P, _P, _P, _I64, _I32, _I32, _I32, ctypes.POINTER(_I64), _P, _P, _P, _P,
                                ctypes.POINTER(_I64), _P],
        "fsparse_shard_unroute": [_P, _P, _I64, _P, _P],
        "fsparse_shard_gather": [_P, _P, _I64, _P, _P],
        "fsparse_shard_offset": [_P, _I64, _I64, _P, _P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.fsparse_last_error_string.argtypes = []
    L.fsparse_last_error_string.restype = ctypes.c_char_p
    L.fsparse_status_string.argtypes = [ctypes.c_int]
    L.fsparse_status_string.restype = ctypes.c_char_p
    L.fsparse_last_timings.argtypes = [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double), _I32]
    L.fsparse_last_timings.restype = _I32
    L.fsparse_kernel_launches.argtypes = []
    L.fsparse_kernel_launches.restype = _I64
    _lib = L
    return L


def _check(st: int, where: str) -> None:
    if st != OK:
        msg = lib().fsparse_last_error_string().decode(errors="replace")
        raise FsparseError(st, where, msg)


# --------------------------------------------------------------------------- C names
def fsparse_symbolic(ii: int, jj: int, length: int, m: int, n: int, nzmax: int, stream: int) -> int:
    out = _P()
    _check(lib().fsparse_symbolic(ii, jj, length, m, n, nzmax, stream, ctypes.byref(out)),
           "fsparse_symbolic")
    return out.value


def fsparse_plan_info(plan: int) -> Tuple[int, int, int, int, int]:
    m, n, L, nnz, cap = _I32(), _I32(), _I64(), _I64(), _I64()
    _check(lib().fsparse_plan_info(plan, ctypes.byref(m), ctypes.byref(n), ctypes.byref(L),
                                   ctypes.byref(nnz), ctypes.byref(cap)), "fsparse_plan_info")
    return m.value, n.value, L.value, nnz.value, cap.value


def fsparse_plan_arrays(plan: int, irank: bool = True, jcS: bool = True,
                        irS: bool = True) -> Tuple[int, int, int]:
    """Device pointers (0 where not requested); asking for irank may derive it."""
    a, b, c = _P(), _P(), _P()
    _check(lib().fsparse_plan_arrays(plan, ctypes.byref(a) if irank else None,
                                     ctypes.byref(b) if jcS else None,
                                     ctypes.byref(c) if irS else None), "fsparse_plan_arrays")
    return a.value or 0, b.value or 0, c.value or 0


def fsparse_plan_destroy(plan: int) -> None:
    _check(lib().fsparse_plan_destroy(plan), "fsparse_plan_destroy")


def fsparse_plan_release(plan: int, stream: int) -> None:
    _check(lib().fsparse_plan_release(plan, stream), "fsparse_plan_release")


def fsparse_numeric(plan: int, sr: int, prS: int, stream: int) -> None:
    _check(lib().fsparse_numeric(plan, sr, prS, stream), "fsparse_numeric")


def fsparse_numeric_adjoint(plan: int, dprS: int, ds: int, stream: int) -> None:
    _check(lib().fsparse_numeric_adjoint(plan, dprS, ds, stream), "fsparse_numeric_adjoint")


def fsparse_assemble(ii: int, jj: int, sr: int, length: int, m: int, n: int, nzmax: int, prS: int,
                     capacity: int, stream: int) -> int:
    out = _P()
    st = lib().fsparse_assemble(ii, jj, sr, length, m, n, nzmax, prS, capacity, stream,
                                ctypes.byref(out))
    if st != OK and out.value:
        lib().fsparse_plan_destroy(out.value)
    _check(st, "fsparse_assemble")
    return out.value


def fsparse_plan_export(plan: int) -> bytes:
    size = _I64()
    _check(lib().fsparse_plan_export(plan, None, 0, ctypes.byref(size)), "fsparse_plan_export")
    buf = ctypes.create_string_buffer(size.value)
    _check(lib().fsparse_plan_export(plan, buf, size.value, ctypes.byref(size)), "fsparse_plan_export")
    return buf.raw


def fsparse_plan_import(image: bytes, stream: int) -> int:
    out = _P()
    _check(lib().fsparse_plan_import(image, len(image), stream, ctypes.byref(out)), "fsparse_plan_import")
    return out.value


def fsparse_plan_append(plan: int, ii: int, jj: int, length: int, stream: int) -> int:
    out = _P()
    _check(lib().fsparse_plan_append(plan, ii, jj, length, stream, ctypes.byref(out)),
           "fsparse_plan_append")
    return out.value


def fsparse_symbolic_f64(ii: int, jj: int, length: int, m: int, n: int, nzmax: int, stream: int) -> int:
    out = _P()
    _check(lib().fsparse_symbolic_f64(ii, jj, length, m, n, nzmax, stream, ctypes.byref(out)),
           "fsparse_symbolic_f64")
    return out.value


def fsparse_assemble_f64(ii: int, jj: int, sr: int, length: int, m: int, n: int, nzmax: int, prS: int,
                         capacity: int, stream: int) -> int:
    out = _P()
    st = lib().fsparse_assemble_f64(ii, jj, sr, length, m, n, nzmax, prS, capacity, stream,
                                    ctypes.byref(out))
    if st != OK and out.value:
        lib().fsparse_plan_destroy(out.value)
    _check(st, "fsparse_assemble_f64")
    return out.value


def fsparse_batch_create(plans: Sequence[int], stream: int) -> int:
    arr = (_P * max(len(plans), 1))(*plans)
    out = _P()
    _check(lib().fsparse_batch_create(len(plans), arr, stream, ctypes.byref(out)),
           "fsparse_batch_create")
    return out.value


def fsparse_batch_symbolic(ii: int, jj: int, len_off: Sequence[int], m: Sequence[int],
                           n: Sequence[int], stream: int) -> int:
    count = len(m)
    lo = (_I64 * (count + 1))(*len_off)
    mm = (_I32 * max(count, 1))(*m)
    nn = (_I32 * max(count, 1))(*n)
    out = _P()
    _check(lib().fsparse_batch_symbolic(count, ii, jj, lo, mm, nn, stream, ctypes.byref(out)),
           "fsparse_batch_symbolic")
    return out.value


def fsparse_batch_arrays(batch: int, count: int, irank: bool = True):
    """(irank, jcS, irS) device pointers (irank 0 unless asked) and the instances' m, n."""
    a, b, c = _P(), _P(), _P()
    mm = (_I32 * max(count, 1))()
    nn = (_I32 * max(count, 1))()
    _check(lib().fsparse_batch_arrays(batch, ctypes.byref(a) if irank else None, ctypes.byref(b),
                                      ctypes.byref(c), mm, nn), "fsparse_batch_arrays")
    return a.value or 0, b.value or 0, c.value or 0, list(mm)[:count], list(nn)[:count]


def fsparse_batch_info(batch: int) -> Tuple[List[int], List[int]]:
    cnt = _I32()
    _check(lib().fsparse_batch_info(batch, ctypes.byref(cnt), None, None), "fsparse_batch_info")
    lo = (_I64 * (cnt.value + 1))()
    no = (_I64 * (cnt.value + 1))()
    _check(lib().fsparse_batch_info(batch, None, lo, no), "fsparse_batch_info")
    return list(lo), list(no)


def fsparse_batch_numeric(batch: int, sr: int, prS: int, stream: int) -> None:
    _check(lib().fsparse_batch_numeric(batch, sr, prS, stream), "fsparse_batch_numeric")


def fsparse_batch_destroy(batch: int) -> None:
    _check(lib().fsparse_batch_destroy(batch), "fsparse_batch_destroy")


def fsparse_batch_release(batch: int, stream: int) -> None:
    _check(lib().fsparse_batch_release(batch, stream), "fsparse_batch_release")


def fsparse_shard_route(ii: int, jj: int, sr: int, length: int, m: int, n: int,
                        col_split: Sequence[int], send_i: int, send_j: int, send_s: int, send_k: int,
                        stream: int) -> List[int]:
    """Route a slice to the owners of its columns; returns the group sizes."""
    R = len(col_split) - 1
    split = (_I64 * (R + 1))(*[int(x) for x in col_split])
    counts = (_I64 * max(R, 1))()
    _check(lib().fsparse_shard_route(ii, jj, sr, length, m, n, R, split, send_i, send_j, send_s, send_k,
                                     counts, stream), "fsparse_shard_route")
    return list(counts)[:R]


def fsparse_shard_unroute(back: int, send_k: int, length: int, out: int, stream: int) -> None:
    _check(lib().fsparse_shard_unroute(back, send_k, length, out, stream), "fsparse_shard_unroute")


def fsparse_shard_gather(sr: int, send_k: int, length: int, send_s: int, stream: int) -> None:
    _check(lib().fsparse_shard_gather(sr, send_k, length, send_s, stream), "fsparse_shard_gather")


def fsparse_shard_offset(src: int, length: int, add: int, out: int, stream: int) -> None:
    _check(lib().fsparse_shard_offset(src, length, add, out, stream), "fsparse_shard_offset")


def fsparse_get_config(length: int, m: int, n: int) -> dict:
    c = Config()
    _check(lib().fsparse_get_config(length, m, n, ctypes.byref(c)), "fsparse_get_config")
    return c.as_dict()


def fsparse_set_config(cfg: Optional[dict]) -> None:
    if cfg is None:
        _check(lib().fsparse_set_config(None), "fsparse_set_config")
        return
    c = Config(**{k: int(v) for k, v in cfg.items()})
    _check(lib().fsparse_set_config(ctypes.byref(c)), "fsparse_set_config")


def fsparse_autotune(ii: int, jj: int, sr: int, length: int, m: int, n: int, reps: int,
                     stream: int) -> dict:
    c = Config()
    _check(lib().fsparse_autotune(ii, jj, sr, length, m, n, reps, stream, ctypes.byref(c)),
           "fsparse_autotune")
    return c.as_dict()


def fsparse_tune_save(path: str) -> None:
    _check(lib().fsparse_tune_save(path.encode()), "fsparse_tune_save")


def fsparse_tune_load(path: str) -> None:
    _check(lib().fsparse_tune_load(path.encode()), "fsparse_tune_load")


def fsparse_tune_clear() -> None:
    _check(lib().fsparse_tune_clear(), "fsparse_tune_clear")


def fsparse_last_timings() -> List[Tuple[str, float]]:
    """(phase, ms) of this thread's last symbolic/assemble call run with FSPARSE_TIMING=1."""
    names = (ctypes.c_char_p * 32)()
    ms = (ctypes.c_double * 32)()
    n = lib().fsparse_last_timings(names, ms, 32)
    return [(names[i].decode(), ms[i]) for i in range(min(n, 32))]


def fsparse_kernel_launches() -> int:
    return int(lib().fsparse_kernel_launches())


def fsparse_status_string(st: int) -> str:
    return lib().fsparse_status_string(st).decode()


# --------------------------------------------------------------------------- torch level
def _torch():
    import torch
    return torch


def _stream() -> int:
    return _torch().cuda.current_stream().cuda_stream


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")
    return t


class _DeviceView:
    """Zero-copy view of plan-owned device memory; keeps the owner alive."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


class Plan:
    """Owner of one ``fsparse_plan`` (symbolic result, reusable for numerics)."""

    def __init__(self, handle: int, device):
        self.handle = handle
        self.device = device
        self.m, self.n, self.len, self.nnz, self.cap = fsparse_plan_info(handle)

    def _view(self, ptr: int, n: int):
        torch = _torch()
        if n == 0:
            return torch.empty(0, dtype=torch.int32, device=self.device)
        return torch.as_tensor(_DeviceView(ptr, n, "<i4", self), device=self.device)

    @property
    def irank(self):
        return self._view(fsparse_plan_arrays(self.handle, True, False, False)[0], self.len)

    @property
    def jcS(self):
        return self._view(fsparse_plan_arrays(self.handle, False, True, False)[1], self.n + 1)

    @property
    def irS(self):
        return self._view(fsparse_plan_arrays(self.handle, False, False, True)[2], self.cap)

    def numeric(self, s, out=None):
        return numeric(self, s, out)

    def export(self) -> bytes:
        """Host image of the plan (checkpoint); see ``import_plan``."""
        return fsparse_plan_export(self.handle)

    def close(self) -> None:
        """Release the plan after the work queued so far on the current stream."""
        if self.handle:
            torch = _torch()
            with torch.cuda.device(self.device):
                fsparse_plan_release(self.handle, _stream())
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _index_dtype(ii, jj):
    """int32 indices, or float64 ones (Matlab's double arrays, App. A)."""
    torch = _torch()
    dt = ii.dtype if isinstance(ii, torch.Tensor) else None
    if dt not in (torch.int32, torch.float64):
        raise TypeError(f"ii must be int32 or float64, got {dt}")
    _dev(ii, dt, "ii")
    _dev(jj, dt, "jj")
    return dt == torch.float64


def symbolic(ii, jj, m: int = 0, n: int = 0, nzmax: int = 0) -> Plan:
    torch = _torch()
    f64 = _index_dtype(ii, jj)
    if ii.numel() != jj.numel():
        raise ValueError("ii and jj differ in length")
    call = fsparse_symbolic_f64 if f64 else fsparse_symbolic
    with torch.cuda.device(ii.device):
        h = call(ii.data_ptr(), jj.data_ptr(), ii.numel(), m, n, nzmax, _stream())
    return Plan(h, ii.device)


def append(plan: Plan, ii, jj) -> Plan:
    """Delayed assembly: a new plan for the plan's triplets followed by (ii, jj)."""
    torch = _torch()
    _dev(ii, torch.int32, "ii")
    _dev(jj, torch.int32, "jj")
    if ii.numel() != jj.numel():
        raise ValueError("ii and jj differ in length")
    with torch.cuda.device(plan.device):
        h = fsparse_plan_append(plan.handle, ii.data_ptr(), jj.data_ptr(), ii.numel(), _stream())
    return Plan(h, plan.device)


def import_plan(image: bytes, device=None) -> Plan:
    """Rebuild a plan from ``Plan.export()`` on the current (or given) device."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        h = fsparse_plan_import(image, _stream())
    return Plan(h, dev)


def numeric(plan: Plan, s, out=None):
    torch = _torch()
    _dev(s, torch.float64, "s")
    if s.numel() != plan.len:
        raise ValueError("s has the wrong length for this plan")
    if out is None:
        out = torch.empty(plan.cap, dtype=torch.float64, device=plan.device)
    _dev(out, torch.float64, "out")
    if out.numel() < plan.cap:
        raise ValueError("out is shorter than the plan's capacity")
    with torch.cuda.device(plan.device):
        fsparse_numeric(plan.handle, s.data_ptr(), out.data_ptr(), _stream())
    return out


def numeric_adjoint(plan: Plan, dprS, out=None):
    torch = _torch()
    _dev(dprS, torch.float64, "dprS")
    if dprS.numel() < plan.nnz:
        raise ValueError("dprS is shorter than nnz")
    if out is None:
        out = torch.empty(plan.len, dtype=torch.float64, device=plan.device)
    _dev(out, torch.float64, "out")
    with torch.cuda.device(plan.device):
        fsparse_numeric_adjoint(plan.handle, dprS.data_ptr(), out.data_ptr(), _stream())
    return out


def assemble(ii, jj, s, m: int = 0, n: int = 0, nzmax: int = 0, prS=None):
    """``S = sparse(i, j, s, m, n, nzmax)`` -> (jcS, irS, prS, plan).

    ii and jj are int32, or float64 as Matlab passes them (App. A
    pre-processing: non-integer or < 1 values are bad indices).  jcS and irS
    are views of the plan's arrays; prS has the plan's capacity.
    """
    torch = _torch()
    f64 = _index_dtype(ii, jj)
    _dev(s, torch.float64, "s")
    L = ii.numel()
    if jj.numel() != L or s.numel() != L:
        raise ValueError("ii, jj and s differ in length")
    if prS is None:
        prS = torch.empty(max(L, nzmax, 1), dtype=torch.float64, device=ii.device)
    _dev(prS, torch.float64, "prS")
    call = fsparse_assemble_f64 if f64 else fsparse_assemble
    with torch.cuda.device(ii.device):
        h = call(ii.data_ptr(), jj.data_ptr(), s.data_ptr(), L, m, n, nzmax,
                 prS.data_ptr(), prS.numel(), _stream())
    plan = Plan(h, ii.device)
    return plan.jcS, plan.irS, prS[: plan.cap], plan


def _assemble_fn():
    torch = _torch()

    class Assemble(torch.autograd.Function):
        """prS = A(plan) s, differentiable in s; backward is ds = dprS[irank]."""

        @staticmethod
        def forward(ctx, s, plan):
            ctx.plan = plan
            return numeric(plan, s.contiguous())

        @staticmethod
        def backward(ctx, dprS):
            plan = ctx.plan
            return numeric_adjoint(plan, dprS.contiguous()), None

    return Assemble


_ASSEMBLE = None


def __getattr__(name):
    global _ASSEMBLE
    if name == "Assemble":
        if _ASSEMBLE is None:
            _ASSEMBLE = _assemble_fn()
        return _ASSEMBLE
    raise AttributeError(name)


class Batch:
    """Many instances' numerics in one launch (``fsparse_batch_*``).

    ``Batch(plans)`` concatenates existing plans; ``batch_symbolic(...)``
    assembles many instances in one symbolic pass.
    """

    def __init__(self, plans: Optional[Sequence[Plan]] = None, handle: int = 0, device=None):
        torch = _torch()
        if handle:
            self.device = device
            self.handle = handle
        else:
            self.device = plans[0].device if plans else None
            with torch.cuda.device(self.device):
                self.handle = fsparse_batch_create([p.handle for p in plans], _stream())
        self.len_off, self.nnz_off = fsparse_batch_info(self.handle)
        self.count = len(self.len_off) - 1

    def _view(self, ptr: int, n: int):
        torch = _torch()
        if n == 0:
            return torch.empty(0, dtype=torch.int32, device=self.device)
        return torch.as_tensor(_DeviceView(ptr, n, "<i4", self), device=self.device)

    def arrays(self, irank: bool = True):
        """(irank, jcS, irS, m, n) of a batch made by ``batch_symbolic`` (see
        ``fsparse_batch_arrays`` for the layout); zero-copy device views."""
        a, b, c, m, n = fsparse_batch_arrays(self.handle, self.count, irank)
        jcs_len = sum(x + 1 for x in n)
        ir = self._view(a, self.len_off[-1]) if irank else None
        return ir, self._view(b, jcs_len), self._view(c, self.nnz_off[-1]), m, n

    def instance(self, b: int, irank: bool = True):
        """Instance b's (irank, jcS, irS) as views (``batch_symbolic`` batches)."""
        ir, jc, rs, m, n = self.arrays(irank)
        c0 = sum(x + 1 for x in n[:b])
        return (ir[self.len_off[b]:self.len_off[b + 1]] if irank else None,
                jc[c0:c0 + n[b] + 1], rs[self.nnz_off[b]:self.nnz_off[b + 1]])

    def numeric(self, s_cat, out=None):
        torch = _torch()
        _dev(s_cat, torch.float64, "s_cat")
        if s_cat.numel() != self.len_off[-1]:
            raise ValueError("s_cat has the wrong length")
        if out is None:
            out = torch.empty(max(self.nnz_off[-1], 1), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            fsparse_batch_numeric(self.handle, s_cat.data_ptr(), out.data_ptr(), _stream())
        return out

    def close(self) -> None:
        """Release the batch after the work queued so far on the current stream."""
        if self.handle:
            torch = _torch()
            with torch.cuda.device(self.device):
                fsparse_batch_release(self.handle, _stream())
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_symbolic(ii, jj, len_off: Sequence[int], m: Sequence[int], n: Sequence[int]) -> Batch:
    """Many instances (concatenated int32 triplets, host offsets and
    dimensions) in one symbolic pass -> a :class:`Batch`."""
    torch = _torch()
    _dev(ii, torch.int32, "ii")
    _dev(jj, torch.int32, "jj")
    if ii.numel() != jj.numel() or ii.numel() != int(len_off[-1]):
        raise ValueError("ii, jj and len_off disagree in length")
    with torch.cuda.device(ii.device):
        h = fsparse_batch_symbolic(ii.data_ptr(), jj.data_ptr(), [int(x) for x in len_off],
                                   [int(x) for x in m], [int(x) for x in n], _stream())
    return Batch(handle=h, device=ii.device)


def autotune(ii, jj, s, m: int, n: int, reps: int = 3) -> dict:
    torch = _torch()
    _dev(ii, torch.int32, "ii")
    _dev(jj, torch.int32, "jj")
    _dev(s, torch.float64, "s")
    with torch.cuda.device(ii.device):
        return fsparse_autotune(ii.data_ptr(), jj.data_ptr(), s.data_ptr(), ii.numel(), m, n, reps,
                                _stream())
