"""Delayed assembly: appending triplets to a plan equals assembling the
concatenation (triplet numbers continue), checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DEV, bits, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu


def check_plan(plan, ii, jj, s, m, n):
    r = oracle.assemble(ii, jj, s, m, n)
    assert r.status == oracle.OK
    assert (plan.m, plan.n, plan.len, plan.nnz, plan.cap) == (m, n, len(ii), r.nnz, r.nnz)
    np.testing.assert_array_equal(plan.irank.cpu().numpy(), r.irank)
    np.testing.assert_array_equal(plan.jcS.cpu().numpy(), r.jcS)
    np.testing.assert_array_equal(plan.irS.cpu().numpy()[: r.nnz], r.irS)
    prS = fsparse.numeric(plan, to_dev(s)).cpu().numpy()
    assert np.array_equal(bits(prS[: r.nnz]), bits(r.prS))


def append_parts(t, cuts):
    """Symbolic on the first part, then append the others one by one."""
    edges = [0] + list(cuts) + [t.L]
    plan = fsparse.symbolic(to_dev(t.ii[: edges[1]]), to_dev(t.jj[: edges[1]]), t.m, t.n)
    for a, b in zip(edges[1:-1], edges[2:]):
        nxt = fsparse.append(plan, to_dev(t.ii[a:b]), to_dev(t.jj[a:b]))
        plan.close()
        plan = nxt
    return plan


@pytest.mark.parametrize("split", [0.0, 0.01, 0.5, 0.93, 0.995, 1.0])
def test_append_random(split):
    t = inputs.random_small(40_000, 500, 400, 51, dup=0.5)
    plan = append_parts(t, [int(t.L * split)])
    check_plan(plan, t.ii, t.jj, t.s, t.m, t.n)


@pytest.mark.parametrize("frac", [0.01, 0.002])
def test_append_small_part_of_a_mesh(frac):
    """A small appended part: the old plan's run starts are looked up where
    the new runs need them instead of being listed (fewer new runs than 1/64
    of the old ones)."""
    t = inputs.mesh3d(20, 56)
    cut = t.L - int(t.L * frac)
    plan = append_parts(t, [cut])
    check_plan(plan, t.ii, t.jj, t.s, t.m, t.n)


def test_append_mesh_in_three_parts():
    t = inputs.mesh3d(12, 52)
    plan = append_parts(t, [t.L // 3, 2 * t.L // 3 + 5])
    check_plan(plan, t.ii, t.jj, t.s, t.m, t.n)


def test_append_same_triplets_again_and_disjoint_columns():
    t = inputs.random_small(5_000, 80, 60, 53, dup=0.3)
    ii = np.concatenate([t.ii, t.ii])
    jj = np.concatenate([t.jj, t.jj])
    s = np.concatenate([t.s, t.s[::-1].copy()])
    plan = fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), t.m, t.n)
    plan2 = fsparse.append(plan, to_dev(t.ii), to_dev(t.jj))
    check_plan(plan2, ii, jj, s, t.m, t.n)
    check_plan(plan, t.ii, t.jj, t.s, t.m, t.n)   # the old plan is unchanged
    # new triplets only in columns the old plan never touched
    a = inputs.random_small(3_000, 50, 20, 54)
    b = inputs.random_small(3_000, 50, 20, 55)
    jb = b.jj + 20
    p1 = fsparse.symbolic(to_dev(a.ii), to_dev(a.jj), 50, 40)
    p2 = fsparse.append(p1, to_dev(b.ii), to_dev(jb))
    check_plan(p2, np.concatenate([a.ii, b.ii]), np.concatenate([a.jj, jb]),
               np.concatenate([a.s, b.s]), 50, 40)


def test_append_checks_indices_against_the_plan():
    t = inputs.random_small(1_000, 30, 30, 56)
    plan = fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), 30, 30)
    for bi, bj in (([31], [1]), ([1], [31]), ([0], [1])):
        with pytest.raises(fsparse.FsparseError) as e:
            fsparse.append(plan, to_dev(np.array(bi, np.int32)), to_dev(np.array(bj, np.int32)))
        assert e.value.status == fsparse.ERR_INDEX


def test_append_to_empty_plan_and_adjoint():
    e = torch.empty(0, dtype=torch.int32, device=DEV)
    plan = fsparse.symbolic(e, e, 40, 30)
    t = inputs.random_small(6_000, 40, 30, 57, dup=0.4)
    p2 = fsparse.append(plan, to_dev(t.ii), to_dev(t.jj))
    check_plan(p2, t.ii, t.jj, t.s, 40, 30)
    r = oracle.assemble(t.ii, t.jj, t.s, 40, 30)
    dprS = np.random.Generator(np.random.PCG64(58)).standard_normal(r.nnz)
    ds = fsparse.numeric_adjoint(p2, to_dev(dprS)).cpu().numpy()
    assert np.array_equal(bits(ds), bits(oracle.adjoint(r.irank, dprS)))


def test_append_large_mesh_halves():
    """Both halves large enough for the bucket path."""
    t = inputs.mesh3d(36, 59)
    plan = append_parts(t, [t.L // 2])
    check_plan(plan, t.ii, t.jj, t.s, t.m, t.n)
