"""The paper's benchmark data sets (§4.2: ransparse(siz, nnz_row, nrep), the table of
data sets; 25,000,000 triplets each, values all ones) through the GPU path, checked
against the oracle element by element."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, gpu_assemble
from paper_1406_1066_gb300 import inputs

pytestmark = pytest.mark.gpu

DATA = {"data1": (10000, 50, 50), "data2": (50000, 50, 10), "data3": (50000, 10, 50)}


@pytest.mark.parametrize("name", sorted(DATA))
def test_paper_data_set(name):
    siz, nnz_row, nrep = DATA[name]
    t = inputs.ransparse(siz, nnz_row, nrep, seed=1100 + int(name[-1]))
    assert t.L == 25_000_000
    g = gpu_assemble(t.ii, t.jj, t.s, t.m, t.n)
    r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
    assert_same(g, r)
    # values are ones: every slot holds the multiplicity of its pair (>= nrep)
    assert np.all(r.prS >= nrep) and r.prS.sum() == t.L
