"""Helpers for the GPU parity tests: run the CUDA path, compare with the oracle."""
from __future__ import annotations

import contextlib

import numpy as np
import torch

import oracle
from paper_1406_1066_gb300 import fsparse

DEV = torch.device("cuda:0")


def bits(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@contextlib.contextmanager
def config(**kw):
    """Force a launch configuration for the duration of a block."""
    base = {"strategy": 0, "radix_bits": 0, "sweep_items": 0, "sweep_threads": 0,
            "bucket_target": 0, "numeric_tile": 0}
    base.update(kw)
    fsparse.fsparse_set_config(base)
    try:
        yield
    finally:
        fsparse.fsparse_set_config(None)


def gpu_assemble(ii, jj, s, m=0, n=0, nzmax=0):
    """Full assembly on the GPU; numpy results."""
    jcS, irS, prS, plan = fsparse.assemble(to_dev(ii), to_dev(jj), to_dev(s), m, n, nzmax)
    torch.cuda.synchronize()
    out = dict(nnz=plan.nnz, cap=plan.cap, m=plan.m, n=plan.n, irank=plan.irank.cpu().numpy(),
               jcS=jcS.cpu().numpy(), irS=irS.cpu().numpy(), prS=prS.cpu().numpy(), plan=plan)
    return out


def assert_same(g: dict, r: oracle.Result, values: bool = True):
    assert r.status == oracle.OK
    assert (g["m"], g["n"]) == (r.m, r.n)
    assert g["nnz"] == r.nnz, (g["nnz"], r.nnz)
    assert g["cap"] == r.cap
    np.testing.assert_array_equal(g["irank"], r.irank)
    np.testing.assert_array_equal(g["jcS"], r.jcS)
    np.testing.assert_array_equal(g["irS"][: r.cap], r.irS)
    if values:
        gb, rb = bits(g["prS"][: r.cap]), bits(r.prS)
        if not np.array_equal(gb, rb):
            bad = np.nonzero(gb != rb)[0]
            raise AssertionError(f"prS differs at {bad.size} slots, first {bad[:5]}: "
                                 f"{g['prS'][bad[:5]]} vs {r.prS[bad[:5]]}")


def check_against_oracle(t, nzmax=0):
    g = gpu_assemble(t.ii, t.jj, t.s, t.m, t.n, nzmax)
    r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n, nzmax)
    assert_same(g, r)
    return g, r


def check_properties(ii_d, jj_d, plan, expect_nnz=None):
    """Invariants that hold at any size (computed on the GPU with torch)."""
    irank = plan.irank.long()
    jcS = plan.jcS.long()
    irS = plan.irS[: plan.nnz].long()
    nnz = plan.nnz
    if expect_nnz is not None:
        assert nnz == expect_nnz
    assert int(jcS[0]) == 0 and int(jcS[-1]) == nnz
    assert bool((jcS[1:] >= jcS[:-1]).all())
    assert int(irank.max()) + 1 == nnz
    assert bool((irS[irank] == ii_d.long() - 1).all()), "irS[irank[k]] = ii[k]-1"
    col_of_slot = torch.searchsorted(jcS, torch.arange(nnz, device=DEV), right=True) - 1
    assert bool((col_of_slot[irank] == jj_d.long() - 1).all()), "slot lies in column jj[k]"
    hit = torch.zeros(nnz, dtype=torch.bool, device=DEV)
    hit[irank] = True
    assert bool(hit.all()), "every slot hit"
    same_col = col_of_slot[1:] == col_of_slot[:-1]
    assert bool((irS[1:][same_col] > irS[:-1][same_col]).all()), "rows ascend in a column"
