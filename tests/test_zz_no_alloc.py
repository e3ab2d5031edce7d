"""fsparse_assemble_noalloc, the entry point for callers that may not allocate
device memory (its working memory is a static array inside the library),
called through the C ABI and compared with fsparse_assemble and with the CPU
oracle.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
MAX_LEN = 131072
MAX_COLS = 131072


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def noalloc_status(t):
    """Call the entry point; return (status, nnz, irank, jcS, irS, prS)."""
    L = t.L
    ii, jj, s = _dev(t.ii), _dev(t.jj), _dev(t.s)
    irank = torch.full((max(L, 1),), -7, dtype=torch.int32, device=DEV)
    jcS = torch.full((t.n + 1,), -7, dtype=torch.int32, device=DEV)
    irS = torch.full((max(L, 1),), -7, dtype=torch.int32, device=DEV)
    prS = torch.full((max(L, 1),), np.nan, dtype=torch.float64, device=DEV)
    nnz = ctypes.c_int64(-1)
    st = fsparse.lib().fsparse_assemble_noalloc(
        ii.data_ptr(), jj.data_ptr(), s.data_ptr(), L, t.m, t.n, irank.data_ptr(), jcS.data_ptr(),
        irS.data_ptr(), prS.data_ptr(), ctypes.byref(nnz), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    n = max(nnz.value, 0)
    return st, n, irank[:L].cpu().numpy(), jcS.cpu().numpy(), irS[:n].cpu().numpy(), prS[:n].cpu().numpy()


def noalloc(t):
    st, *out = noalloc_status(t)
    assert st == fsparse.OK, fsparse.lib().fsparse_last_error_string()
    return tuple(out)


def reference(t):
    jcS, irS, prS, plan = fsparse.assemble(_dev(t.ii), _dev(t.jj), _dev(t.s), t.m, t.n)
    torch.cuda.synchronize()
    out = (plan.nnz, plan.irank.cpu().numpy(), jcS.cpu().numpy(), irS[: plan.nnz].cpu().numpy(),
           prS[: plan.nnz].cpu().numpy())
    plan.close()
    return out


def from_oracle(t):
    r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
    assert r.status == oracle.OK
    return r.nnz, r.irank, r.jcS, r.irS[: r.nnz], r.prS[: r.nnz]


def same(a, b):
    assert a[0] == b[0]
    for x, y in zip(a[1:4], b[1:4]):
        np.testing.assert_array_equal(x, y)
    assert np.array_equal(np.asarray(a[4]).view(np.int64), np.asarray(b[4]).view(np.int64))   # bit for bit


def test_noalloc_matches_assemble_and_oracle_on_consecutive_calls():
    problems = [inputs.mesh3d(12, 5),                                     # 116,160 triplets
                inputs.random_small(MAX_LEN, 3000, 4000, 9, dup=0.4),    # the size limit
                inputs.random_small(MAX_LEN, MAX_LEN, MAX_LEN, 12, dup=0.4),  # widest keys (64-bit)
                inputs.random_small(1000, 50, MAX_COLS, 13, dup=0.3),    # most columns, few triplets
                inputs.random_small(333, 7, 5, 10, dup=0.6)]             # small after large
    for t in problems:
        ref = reference(t)
        exact = from_oracle(t)
        first = noalloc(t)
        second = noalloc(t)          # the shared array keeps the previous call's contents
        same(first, exact)
        same(second, exact)
        same(first, ref)


def test_noalloc_empty_input():
    t = inputs.random_small(0, 9, 17, 14)
    nnz, irank, jcS, irS, prS = noalloc(t)
    assert nnz == 0 and irank.size == 0
    np.testing.assert_array_equal(jcS, np.zeros(18, np.int32))


def test_noalloc_bad_index_then_exact_call():
    t = inputs.random_small(5000, 40, 30, 15, dup=0.3)
    bad = t.ii.copy()
    bad[1234] = 41                       # above m
    st, *_ = noalloc_status(inputs.Triplets(bad, t.jj, t.s, t.m, t.n))
    assert st == fsparse.ERR_INDEX
    bad = t.jj.copy()
    bad[7] = 0                           # below 1
    st, *_ = noalloc_status(inputs.Triplets(t.ii, bad, t.s, t.m, t.n))
    assert st == fsparse.ERR_INDEX
    same(noalloc(t), from_oracle(t))


def test_noalloc_withheld_digit_pass_times_out_then_exact_call(monkeypatch):
    """The first digit pass's tile 0 withholds its counts (injected on the
    host): that pass leaves positions unwritten, so the kernels after it read
    whatever the shared array holds -- here a previous call's 64-bit keys,
    whose columns lie far beyond this problem's n.  The call must return
    FSPARSE_ERR_TIMEOUT (its bounded waits give up, every write stays in
    bounds), and the next call must be exact."""
    wide = inputs.random_small(MAX_LEN, MAX_LEN, MAX_LEN, 16, dup=0.2)
    same(noalloc(wide), from_oracle(wide))
    t = inputs.random_small(60_000, 300, 200, 17, dup=0.4)
    monkeypatch.setenv("FSPARSE_FAULT", "timeout_sort")
    t0 = time.perf_counter()
    st, *_ = noalloc_status(t)
    waited = time.perf_counter() - t0
    monkeypatch.delenv("FSPARSE_FAULT")
    assert st == fsparse.ERR_TIMEOUT
    assert waited < 60.0
    same(noalloc(t), from_oracle(t))


def test_noalloc_rejects_sizes_beyond_its_limits():
    lib = fsparse.lib()
    nnz = ctypes.c_int64(0)
    assert lib.fsparse_assemble_noalloc(None, None, None, MAX_LEN + 1, 10, 10, None, None, None,
                                        None, ctypes.byref(nnz), None) == fsparse.ERR_SIZE
    assert lib.fsparse_assemble_noalloc(None, None, None, 10, 10, MAX_COLS + 1, None, None, None,
                                        None, ctypes.byref(nnz), None) == fsparse.ERR_SIZE
    assert lib.fsparse_assemble_noalloc(None, None, None, 10, 0, 10, None, None, None,
                                        None, ctypes.byref(nnz), None) == fsparse.ERR_ARG
