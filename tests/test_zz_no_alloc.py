"""fsparse_assemble_noalloc, the entry point for callers that may not allocate
device memory (its working memory is a static array inside the library),
called through the C ABI and compared with fsparse_assemble.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
MAX_LEN = 131072


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def noalloc(t):
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
    assert st == fsparse.OK, fsparse.lib().fsparse_last_error_string()
    torch.cuda.synchronize()
    n = nnz.value
    return n, irank[:L].cpu().numpy(), jcS.cpu().numpy(), irS[:n].cpu().numpy(), prS[:n].cpu().numpy()


def reference(t):
    jcS, irS, prS, plan = fsparse.assemble(_dev(t.ii), _dev(t.jj), _dev(t.s), t.m, t.n)
    torch.cuda.synchronize()
    out = (plan.nnz, plan.irank.cpu().numpy(), jcS.cpu().numpy(), irS[: plan.nnz].cpu().numpy(),
           prS[: plan.nnz].cpu().numpy())
    plan.close()
    return out


def same(a, b):
    assert a[0] == b[0]
    for x, y in zip(a[1:4], b[1:4]):
        np.testing.assert_array_equal(x, y)
    assert np.array_equal(a[4].view(np.int64), b[4].view(np.int64))   # prS bit for bit


def test_noalloc_matches_assemble_on_consecutive_calls():
    problems = [inputs.mesh3d(12, 5),                                     # 116,160 triplets
                inputs.random_small(MAX_LEN, 3000, 4000, 9, dup=0.4),    # the size limit
                inputs.random_small(MAX_LEN, MAX_LEN, MAX_LEN, 12, dup=0.4),  # widest keys (64-bit)
                inputs.random_small(333, 7, 5, 10, dup=0.6)]             # small after large
    for t in problems:
        ref = reference(t)
        first = noalloc(t)
        second = noalloc(t)          # the shared array keeps the previous call's contents
        same(first, ref)
        same(second, ref)


def test_noalloc_rejects_sizes_beyond_its_limits():
    lib = fsparse.lib()
    nnz = ctypes.c_int64(0)
    assert lib.fsparse_assemble_noalloc(None, None, None, MAX_LEN + 1, 10, 10, None, None, None,
                                        None, ctypes.byref(nnz), None) == fsparse.ERR_SIZE
    assert lib.fsparse_assemble_noalloc(None, None, None, 10, 10, MAX_LEN + 1, None, None, None,
                                        None, ctypes.byref(nnz), None) == fsparse.ERR_SIZE
    assert lib.fsparse_assemble_noalloc(None, None, None, 10, 0, 10, None, None, None,
                                        None, ctypes.byref(nnz), None) == fsparse.ERR_ARG
