"""The paper's own CPU method (serial §2.3, threaded §3) against the printed
example and the sort-based oracle: a third, independent route to the same
irank / jcS / irS / prS."""
import numpy as np
import pytest

import oracle
import pins
from oracle import paper_method
from paper_1406_1066_gb300 import inputs


def same(a: oracle.Result, b: oracle.Result):
    assert a.status == b.status == oracle.OK
    assert a.nnz == b.nnz
    np.testing.assert_array_equal(a.irank, b.irank)
    np.testing.assert_array_equal(a.jcS, b.jcS)
    np.testing.assert_array_equal(a.irS[: a.nnz], b.irS[: b.nnz])
    np.testing.assert_array_equal(pins.bits(a.prS[: a.nnz]), pins.bits(b.prS[: b.nnz]))


@pytest.mark.parametrize("threads", [None, 1, 2, 3, 4])
def test_running_example_gives_printed_arrays(threads):
    g = pins.golden()
    t, e = g["running_example"], g["matrix_eq_2_1"]
    r, _ = paper_method.assemble(t["ii"], t["jj"], t["s"], threads=threads)
    assert r.irank.tolist() == g["part4"]["irank"]
    assert r.jcS.tolist() == e["jcS"] and r.irS.tolist() == e["irS"] and r.prS.tolist() == e["prS"]


CASES = [
    ("random", lambda: inputs.random_small(30_000, 400, 300, 41, dup=0.5)),
    ("random_wide", lambda: inputs.random_small(20_000, 50_000, 70_000, 42, dup=0.2)),
    ("pooled", lambda: inputs.pooled(2_000, 1_500, 60_000, 5_000, 43)),
    ("mesh2d", lambda: inputs.mesh2d(30, 44)),
    ("mesh3d", lambda: inputs.mesh3d(9, 45)),
    ("tall", lambda: inputs.random_small(5_000, 3, 900, 46, dup=0.6)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("threads", [None, 1, 3, 8])
def test_agrees_with_oracle(name, make, threads):
    t = make()
    ref = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
    r, used = paper_method.assemble(t.ii, t.jj, t.s, t.m, t.n, threads=threads)
    same(r, ref)
    if threads is not None and paper_method.openmp:
        assert used == threads


def test_more_threads_than_rows_and_empty():
    r, _ = paper_method.assemble([2, 1, 2], [1, 1, 1], [1.0, 2.0, 3.0], 2, 1, threads=8)
    assert r.jcS.tolist() == [0, 2] and r.irS.tolist() == [0, 1] and r.prS.tolist() == [2.0, 4.0]
    r, _ = paper_method.assemble([], [], [], 3, 4, threads=4)
    assert r.nnz == 0 and r.jcS.tolist() == [0] * 5
