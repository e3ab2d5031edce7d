"""Matlab-style double index arrays (App. A pre-processing) on the GPU,
against the oracle's ``assemble_f64`` / ``getix``."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DEV, assert_same, bits, gpu_assemble, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu


def as_f64(t):
    return t.ii.astype(np.float64), t.jj.astype(np.float64)


@pytest.mark.parametrize("case", ["mesh2d_40", "mesh3d_14", "random_implicit", "random_explicit"])
def test_double_indices_match_oracle(case):
    if case == "mesh2d_40":
        t = inputs.mesh2d(40, 31)
    elif case == "mesh3d_14":
        t = inputs.mesh3d(14, 32)
    else:
        t = inputs.random_small(50_000, 700, 900, 33, dup=0.4)
    m, n = (0, 0) if case == "random_implicit" else (t.m, t.n)
    fi, fj = as_f64(t)
    g = gpu_assemble(fi, fj, t.s, m, n)
    r = oracle.assemble_f64(fi, fj, t.s, m, n)
    assert_same(g, r)


def test_double_indices_nzmax_and_symbolic():
    t = inputs.random_small(20_000, 300, 200, 34, dup=0.5)
    fi, fj = as_f64(t)
    r = oracle.assemble_f64(fi, fj, t.s, t.m, t.n, 30_000)
    g = gpu_assemble(fi, fj, t.s, t.m, t.n, 30_000)
    assert_same(g, r)
    plan = fsparse.symbolic(to_dev(fi), to_dev(fj), t.m, t.n)
    prS = fsparse.numeric(plan, to_dev(t.s)).cpu().numpy()
    r0 = oracle.assemble_f64(fi, fj, t.s, t.m, t.n)
    assert plan.nnz == r0.nnz
    assert np.array_equal(plan.irank.cpu().numpy(), r0.irank)
    assert np.array_equal(bits(prS[: r0.nnz]), bits(r0.prS))


BAD = [0.0, -0.0, -3.0, 0.5, 1.5, np.nextafter(2.0, 1.0), np.nextafter(7.0, 8.0),
       float("nan"), float("inf"), float("-inf"), 2.0**31, 1e300, 5e-324]


@pytest.mark.parametrize("where", ["ii", "jj"])
@pytest.mark.parametrize("value", BAD, ids=[repr(float(v)) for v in BAD])
def test_bad_double_index_is_rejected(where, value):
    t = inputs.random_small(5000, 40, 30, 35)
    fi, fj = as_f64(t)
    k = 1234
    (fi if where == "ii" else fj)[k] = value
    assert oracle.assemble_f64(fi, fj, t.s, 0, 0).status == oracle.ERR_INDEX
    for m, n in ((0, 0), (t.m, t.n)):
        with pytest.raises(fsparse.FsparseError) as e:
            fsparse.assemble(to_dev(fi), to_dev(fj), to_dev(t.s), m, n)
        assert e.value.status == fsparse.ERR_INDEX
        with pytest.raises(fsparse.FsparseError) as e:
            fsparse.symbolic(to_dev(fi), to_dev(fj), m, n)
        assert e.value.status == fsparse.ERR_INDEX


def test_double_index_beyond_explicit_dimension():
    fi = np.array([1.0, 5.0, 2.0])
    fj = np.array([1.0, 1.0, 2.0])
    assert oracle.assemble_f64(fi, fj, np.ones(3), 4, 2).status == oracle.ERR_INDEX
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.assemble(to_dev(fi), to_dev(fj), to_dev(np.ones(3)), 4, 2)
    assert e.value.status == fsparse.ERR_INDEX
    # the largest int index is accepted when the dimension allows it
    big = float(2**31 - 1)
    r = oracle.assemble_f64([big], [1.0], [2.5], 0, 1)
    assert r.status == oracle.OK and r.m == 2**31 - 1


def test_empty_double_input():
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    jcS, irS, prS, plan = fsparse.assemble(e, e, e, 3, 4)
    assert plan.nnz == 0 and jcS.cpu().tolist() == [0] * 5


def test_int_and_double_paths_agree_on_mesh3d_40():
    """Sizes that take the bucket path; compared with the oracle element by element."""
    t = inputs.mesh3d(40, 36)
    fi, fj = as_f64(t)
    g = gpu_assemble(fi, fj, t.s, t.m, t.n)
    r = oracle.assemble_f64(fi, fj, t.s, t.m, t.n)
    assert_same(g, r)
