"""Adjoint / autograd: ds = dprS[irank], against the oracle, finite differences and gradcheck."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DEV, bits, config, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mesh60():
    t = inputs.workload("mesh3d_60")
    plan = fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), t.m, t.n)
    r = oracle.assemble(t.ii, t.jj, None, t.m, t.n)
    return t, plan, r


def test_backward_matches_oracle_transpose(mesh60):
    t, plan, r = mesh60
    assert np.array_equal(plan.irank.cpu().numpy(), r.irank)
    dprS = np.random.Generator(np.random.PCG64(1414)).standard_normal(plan.nnz)
    s = to_dev(t.s).requires_grad_(True)
    prS = fsparse.Assemble.apply(s, plan)
    prS.backward(to_dev(dprS))
    ref = oracle.adjoint(r.irank, dprS)
    assert np.array_equal(bits(s.grad.cpu().numpy()), bits(ref))


def test_finite_differences(mesh60):
    t, plan, _ = mesh60
    dprS = to_dev(np.random.Generator(np.random.PCG64(1414)).standard_normal(plan.nnz))
    s = to_dev(t.s)
    grad = fsparse.numeric_adjoint(plan, dprS)
    ks = np.random.Generator(np.random.PCG64(1415)).integers(0, t.L, 1000)
    h = 1.0   # the map is linear: no truncation error, and h is a power of two
    worst = 0.0
    for k in ks:
        v = s[k].item()
        s[k] = v + h
        plus = fsparse.numeric(plan, s)
        s[k] = v - h
        minus = fsparse.numeric(plan, s)
        s[k] = v
        fd = float((dprS * (plus[: plan.nnz] - minus[: plan.nnz])).sum()) / (2 * h)
        g = float(grad[k])
        worst = max(worst, abs(fd - g) / max(abs(g), 1e-300))
    assert worst <= 1e-12, worst


def test_gradcheck_tiny():
    t = inputs.random_small(60, 6, 5, 3, dup=0.5)
    plan = fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), 6, 5)
    s = to_dev(t.s).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: fsparse.Assemble.apply(x, plan), (s,), eps=1e-6,
                                    atol=1e-9)
