"""Seeded random problems of many shapes, through every sort strategy, the
numeric re-assembly and delayed assembly, each against the oracle.

The shapes mix what the directed tests take one at a time: lengths from 0 to
a few hundred thousand, dimensions from 1 to 2^21, columns filled evenly,
half of them empty, or a few very dense ones, and duplicate rates from none
to most.  Every case is fixed by its seed."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, bits, config, gpu_assemble, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu

CASES = 200


def make_case(seed):
    g = np.random.Generator(np.random.PCG64(90_000 + seed))
    L = int(np.exp(g.uniform(0, np.log(300_000)))) if g.random() > 0.05 else 0
    m = int(np.exp(g.uniform(0, np.log(1 << 21))))
    n = int(np.exp(g.uniform(0, np.log(1 << 21))))
    shape = g.integers(0, 3)
    ii = g.integers(1, m + 1, L, dtype=np.int32)
    if shape == 0:                    # columns filled evenly
        jj = g.integers(1, n + 1, L, dtype=np.int32)
    elif shape == 1:                  # the upper half of the columns empty
        jj = g.integers(1, max(1, n // 2) + 1, L, dtype=np.int32)
    else:                             # a few dense columns among sparse ones
        dense = g.integers(1, n + 1, 3, dtype=np.int32)
        jj = np.where(g.random(L) < 0.5, dense[g.integers(0, 3, L)], g.integers(1, n + 1, L)).astype(np.int32)
    dup = float(g.choice([0.0, 0.3, 0.8]))
    if L > 1 and dup > 0:
        src = g.integers(0, L, L)
        take = g.random(L) < dup
        ii = np.where(take, ii[src], ii).astype(np.int32)
        jj = np.where(take, jj[src], jj).astype(np.int32)
    s = g.standard_normal(L)
    s[g.random(L) < 0.02] = -0.0
    strategy = int(g.integers(0, 4))   # 0 = automatic, 1 = onesweep, 2 = bucket, 3 = bucket radix only
    split = int(L * g.random()) if L else 0
    return inputs.Triplets(ii, jj, s, m, n, 0, f"fuzz_{seed}"), strategy, split, g.standard_normal(L)


@pytest.mark.parametrize("seed", range(CASES))
def test_fuzz_assemble_numeric_append(seed):
    t, strategy, split, s2 = make_case(seed)
    r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
    with config(strategy=strategy):
        g = gpu_assemble(t.ii, t.jj, t.s, t.m, t.n)
        assert_same(g, r)
        # re-assembly with other values through the same plan
        pr2 = fsparse.numeric(g["plan"], to_dev(s2)).cpu().numpy()
        assert np.array_equal(bits(pr2[: r.nnz]), bits(oracle.numeric(r.irank, s2, r.nnz)[: r.nnz]))
        g["plan"].close()
        # the same triplets as a plan of a prefix plus an appended rest
        base = fsparse.symbolic(to_dev(t.ii[:split]), to_dev(t.jj[:split]), t.m, t.n)
        plan = fsparse.append(base, to_dev(t.ii[split:]), to_dev(t.jj[split:]))
        base.close()
        assert (plan.nnz, plan.len) == (r.nnz, t.L)
        np.testing.assert_array_equal(plan.jcS.cpu().numpy(), r.jcS)
        np.testing.assert_array_equal(plan.irS.cpu().numpy()[: r.nnz], r.irS)
        np.testing.assert_array_equal(plan.irank.cpu().numpy(), r.irank)
        pr3 = fsparse.numeric(plan, to_dev(t.s)).cpu().numpy()
        assert np.array_equal(bits(pr3[: r.nnz]), bits(r.prS))
        plan.close()
