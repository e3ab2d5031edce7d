"""Batched numeric re-assembly: one launch == per-plan launches == oracle; CUDA graph replay."""
import numpy as np
import pytest
import torch

import oracle
import pins
from gpu_util import DEV, bits, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch256():
    b = inputs.batch(256, 1416)
    plans = [fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), t.m, t.n) for t in b.instances]
    return b, plans


def test_batch_structure(batch256):
    b, plans = batch256
    for t, p in zip(b.instances, plans):
        assert p.nnz == pins.mesh_nnz(t.meta["N"], t.meta["dim"])
    assert 1.5e8 < b.L < 3.5e8


def test_batched_equals_plain_and_oracle(batch256):
    b, plans = batch256
    bt = fsparse.Batch(plans)
    s_cat = np.concatenate([inputs.mesh_values(t.L, 7000 + i) for i, t in enumerate(b.instances)])
    out = bt.numeric(to_dev(s_cat)).cpu().numpy()
    for i, (t, p) in enumerate(zip(b.instances, plans)):
        lo, hi = bt.len_off[i], bt.len_off[i + 1]
        plain = fsparse.numeric(p, to_dev(s_cat[lo:hi])).cpu().numpy()
        got = out[bt.nnz_off[i]: bt.nnz_off[i + 1]]
        assert np.array_equal(bits(got), bits(plain[: p.nnz])), i
        if i % 16 == 0:
            r = oracle.assemble(t.ii, t.jj, s_cat[lo:hi], t.m, t.n)
            assert np.array_equal(bits(got), bits(r.prS)), i
    bt.close()


def test_graph_replay(batch256):
    b, plans = batch256
    bt = fsparse.Batch(plans)
    total = bt.len_off[-1]
    s_buf = torch.empty(total, dtype=torch.float64, device=DEV)
    out = torch.empty(bt.nnz_off[-1], dtype=torch.float64, device=DEV)
    vals = [torch.from_numpy(np.random.Generator(np.random.PCG64(9 + k)).uniform(-1, 1, total)).to(DEV)
            for k in range(2)]
    s_buf.copy_(vals[0])
    bt.numeric(s_buf, out)   # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bt.numeric(s_buf, out)
    for k in range(2):
        s_buf.copy_(vals[k])
        g.replay()
        torch.cuda.synchronize()
        ref = bt.numeric(vals[k]).cpu().numpy()
        assert np.array_equal(bits(out.cpu().numpy()), bits(ref))
    bt.close()
