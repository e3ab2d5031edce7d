"""Batched assembly of the 256 uneven mesh instances: one symbolic pass for all
of them (fsparse_batch_symbolic) and one numeric launch (fsparse_batch_numeric)
== per-instance calls == the oracle, every instance, every array; CUDA graph
replay of the batched numeric."""
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
    s_cat = np.concatenate([inputs.mesh_values(t.L, 7000 + i) for i, t in enumerate(b.instances)])
    off = np.concatenate([[0], np.cumsum([t.L for t in b.instances])]).astype(np.int64)
    refs = [oracle.assemble(t.ii, t.jj, s_cat[off[i]:off[i + 1]], t.m, t.n)
            for i, t in enumerate(b.instances)]
    yield b, plans, s_cat, off, refs
    for p in plans:
        p.close()


def test_batch_structure(batch256):
    b, plans, _, _, refs = batch256
    for t, p, r in zip(b.instances, plans, refs):
        assert p.nnz == r.nnz == pins.mesh_nnz(t.meta["N"], t.meta["dim"])
    assert 1.5e8 < b.L < 3.5e8


def test_batch_of_plans_equals_plain_and_oracle(batch256):
    b, plans, s_cat, off, refs = batch256
    bt = fsparse.Batch(plans)
    out = bt.numeric(to_dev(s_cat)).cpu().numpy()
    for i, (t, p, r) in enumerate(zip(b.instances, plans, refs)):
        lo, hi = bt.len_off[i], bt.len_off[i + 1]
        plain = fsparse.numeric(p, to_dev(s_cat[lo:hi])).cpu().numpy()
        got = out[bt.nnz_off[i]: bt.nnz_off[i + 1]]
        assert np.array_equal(bits(got), bits(plain[: p.nnz])), i
        assert np.array_equal(bits(got), bits(r.prS)), i
    bt.close()


def _batch_symbolic(insts):
    ii = to_dev(np.concatenate([t.ii for t in insts]))
    jj = to_dev(np.concatenate([t.jj for t in insts]))
    off = np.concatenate([[0], np.cumsum([t.L for t in insts])]).astype(np.int64)
    return fsparse.batch_symbolic(ii, jj, off, [t.m for t in insts], [t.n for t in insts]), off


def test_batch_symbolic_equals_oracle_every_instance(batch256):
    """One symbolic pass over all 256 instances: irank, jcS, irS of every
    instance bit-exact, and the batched numeric's prS at 0 ULP."""
    b, plans, s_cat, off, refs = batch256
    bt, off2 = _batch_symbolic(b.instances)
    assert list(off2) == bt.len_off
    out = bt.numeric(to_dev(s_cat)).cpu().numpy()
    ir, jc, rs, m, n = bt.arrays()
    ir, jc, rs = ir.cpu().numpy(), jc.cpu().numpy(), rs.cpu().numpy()
    c0 = 0
    for i, (t, r) in enumerate(zip(b.instances, refs)):
        assert (m[i], n[i]) == (t.m, t.n)
        assert bt.nnz_off[i + 1] - bt.nnz_off[i] == r.nnz, i
        np.testing.assert_array_equal(ir[bt.len_off[i]:bt.len_off[i + 1]], r.irank, err_msg=str(i))
        np.testing.assert_array_equal(jc[c0:c0 + t.n + 1], r.jcS, err_msg=str(i))
        np.testing.assert_array_equal(rs[bt.nnz_off[i]:bt.nnz_off[i + 1]], r.irS, err_msg=str(i))
        assert np.array_equal(bits(out[bt.nnz_off[i]:bt.nnz_off[i + 1]]), bits(r.prS)), i
        c0 += t.n + 1
    bt.close()


def test_batch_symbolic_uneven_small_and_empty_instances():
    insts = [inputs.random_small(700, 30, 20, 81, dup=0.5), inputs.random_small(0, 5, 6, 82),
             inputs.mesh2d(9, 83), inputs.random_small(1, 1, 1, 84), inputs.random_small(5000, 3, 900, 85),
             inputs.random_small(0, 0, 0, 86), inputs.mesh3d(5, 87)]
    bt, off = _batch_symbolic(insts)
    s_cat = np.concatenate([t.s for t in insts])
    out = bt.numeric(to_dev(s_cat)).cpu().numpy()
    c0 = 0
    for i, t in enumerate(insts):
        r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
        ir, jc, rs = (x.cpu().numpy() for x in bt.instance(i))
        np.testing.assert_array_equal(ir, r.irank)
        np.testing.assert_array_equal(jc, r.jcS)
        np.testing.assert_array_equal(rs, r.irS)
        assert np.array_equal(bits(out[bt.nnz_off[i]:bt.nnz_off[i + 1]]), bits(r.prS)), i
        c0 += t.n + 1
    bt.close()


def test_batch_symbolic_implicit_dims_and_bad_index():
    insts = [inputs.random_small(3000, 40, 50, 91, dup=0.4), inputs.random_small(2000, 70, 9, 92, dup=0.4)]
    ii = to_dev(np.concatenate([t.ii for t in insts]))
    jj = to_dev(np.concatenate([t.jj for t in insts]))
    off = [0, insts[0].L, insts[0].L + insts[1].L]
    bt = fsparse.batch_symbolic(ii, jj, off, [0, 70], [50, 0])
    _, _, _, m, n = bt.arrays(irank=False)
    for i, t in enumerate(insts):
        r = oracle.assemble(t.ii, t.jj, t.s, 0 if i == 0 else 70, 50 if i == 0 else 0)
        assert (m[i], n[i]) == (r.m, r.n)
        ir, jc, rs = (x.cpu().numpy() for x in bt.instance(i))
        np.testing.assert_array_equal(ir, r.irank)
        np.testing.assert_array_equal(jc, r.jcS)
        np.testing.assert_array_equal(rs, r.irS)
    bt.close()
    # an index within the concatenated matrix but outside its own instance
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.batch_symbolic(ii, jj, off, [40, 70], [50, 8])   # instance 1 has a column 9
    assert e.value.status == fsparse.ERR_INDEX
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.batch_symbolic(ii, jj, off, [39, 70], [50, 9])   # instance 0 has a row 40
    assert e.value.status == fsparse.ERR_INDEX


def test_graph_replay(batch256):
    b, plans, _, _, _ = batch256
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
