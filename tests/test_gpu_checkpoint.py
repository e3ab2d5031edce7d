"""Checkpoint / resume of the symbolic state: a plan exported to host memory
and imported again behaves exactly like the original (arrays, numeric fold,
adjoint, batching, appending), and a damaged image is refused."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DEV, bits, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu


def arrays(plan):
    return (plan.irank.cpu().numpy(), plan.jcS.cpu().numpy(), plan.irS.cpu().numpy())


@pytest.mark.parametrize("case", ["mesh", "nzmax", "empty"])
def test_export_import_roundtrip(case):
    if case == "mesh":
        t, nzmax = inputs.mesh3d(18, 81), 0
    elif case == "nzmax":
        t = inputs.random_small(20_000, 300, 200, 82, dup=0.5)
        nzmax = 25_000
    else:
        t, nzmax = inputs.random_small(0, 5, 7, 83), 0
    plan = fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), t.m, t.n, nzmax)
    image = plan.export()
    again = fsparse.import_plan(image)
    assert (again.m, again.n, again.len, again.nnz, again.cap) == (plan.m, plan.n, plan.len, plan.nnz, plan.cap)
    for a, b in zip(arrays(plan), arrays(again)):
        np.testing.assert_array_equal(a, b)
    if t.L:
        s = to_dev(t.s)
        assert np.array_equal(bits(fsparse.numeric(plan, s).cpu()), bits(fsparse.numeric(again, s).cpu()))
        r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n, nzmax)
        assert np.array_equal(bits(fsparse.numeric(again, s).cpu().numpy()[: r.cap]), bits(r.prS))
        d = torch.randn(again.nnz, dtype=torch.float64, device=DEV)
        assert np.array_equal(bits(fsparse.numeric_adjoint(plan, d).cpu()),
                              bits(fsparse.numeric_adjoint(again, d).cpu()))
    assert again.export() == image
    plan.close()
    again.close()


def test_imported_plan_batches_and_appends():
    a = inputs.mesh2d(30, 84)
    b = inputs.mesh3d(9, 85)
    pa = fsparse.import_plan(fsparse.symbolic(to_dev(a.ii), to_dev(a.jj), a.m, a.n).export())
    pb = fsparse.symbolic(to_dev(b.ii), to_dev(b.jj), b.m, b.n)
    batch = fsparse.Batch([pa, pb])
    s_cat = to_dev(np.concatenate([a.s, b.s]))
    out = batch.numeric(s_cat).cpu().numpy()
    ra, rb = oracle.assemble(a.ii, a.jj, a.s, a.m, a.n), oracle.assemble(b.ii, b.jj, b.s, b.m, b.n)
    assert np.array_equal(bits(out[: ra.nnz]), bits(ra.prS))
    assert np.array_equal(bits(out[ra.nnz: ra.nnz + rb.nnz]), bits(rb.prS))
    extra = inputs.random_small(2_000, a.m, a.n, 86)
    p2 = fsparse.append(pa, to_dev(extra.ii), to_dev(extra.jj))
    r2 = oracle.assemble(np.concatenate([a.ii, extra.ii]), np.concatenate([a.jj, extra.jj]),
                         np.concatenate([a.s, extra.s]), a.m, a.n)
    assert np.array_equal(p2.irank.cpu().numpy(), r2.irank)


def test_damaged_image_is_refused():
    t = inputs.random_small(3_000, 40, 30, 87)
    image = bytearray(fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), t.m, t.n).export())
    for bad in (bytes(image[:-4]), bytes(image) + b"\0\0\0\0", b"XXXXXXXX" + bytes(image[8:])):
        with pytest.raises(fsparse.FsparseError) as e:
            fsparse.import_plan(bad)
        assert e.value.status == fsparse.ERR_ARG
    changed = bytearray(image)
    changed[8 + 16] ^= 1          # len field: sizes no longer match the image
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.import_plan(bytes(changed))
    assert e.value.status == fsparse.ERR_ARG
