"""The largest accepted input, len = 2^30 - 1 (the look-back words keep two
flag bits), through the full assembly.  Too large for the oracle as a whole:
checked by properties that hold at any size, the exact unique-pair count,
and the ascending-k fold of sampled slots computed on the CPU.  Inputs are
drawn on the device from a seeded generator (m = n = 2^15, so pairs repeat
about once on average and runs of several triplets occur)."""
import numpy as np
import pytest
import torch

from gpu_util import DEV, bits, check_properties
from paper_1406_1066_gb300 import fsparse

pytestmark = pytest.mark.gpu

L_MAX = 2**30 - 1


def test_maximum_length_full_assembly():
    m = n = 2**15
    g = torch.Generator(device=DEV).manual_seed(1073741823)
    ii = torch.randint(1, m + 1, (L_MAX,), device=DEV, dtype=torch.int32, generator=g)
    jj = torch.randint(1, n + 1, (L_MAX,), device=DEV, dtype=torch.int32, generator=g)
    s = torch.randn(L_MAX, device=DEV, dtype=torch.float64, generator=g)
    jcS, irS, prS, plan = fsparse.assemble(ii, jj, s, m, n)
    torch.cuda.synchronize()
    keys = (jj.long() - 1) * m + (ii.long() - 1)
    nnz = int(torch.unique(keys).numel())
    del keys
    torch.cuda.empty_cache()
    check_properties(ii, jj, plan, expect_nnz=nnz)
    # sampled slots: the fold from +0.0 in ascending k, on the CPU
    irank = plan.irank
    pick = torch.from_numpy(np.random.Generator(np.random.PCG64(30)).integers(0, nnz, 500)).to(DEV)
    pick = torch.unique(pick.to(torch.int32))
    ks = torch.nonzero(torch.isin(irank, pick)).flatten()
    slot_of = irank[ks].cpu().numpy()
    vals = s[ks].cpu().numpy()
    ks_h = ks.cpu().numpy()
    pr = prS[pick.long()].cpu().numpy()
    expect = {}
    for k, sl, v in sorted(zip(ks_h.tolist(), slot_of.tolist(), vals.tolist())):
        expect[sl] = expect.get(sl, 0.0) + v
    for sl, got in zip(pick.cpu().numpy().tolist(), pr.tolist()):
        assert bits([expect[sl]])[0] == bits([got])[0], (sl, expect[sl], got)
    plan.close()


def test_length_above_the_maximum_is_refused():
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.fsparse_symbolic(8, 8, L_MAX + 1, 3, 3, 0, 0)
    assert e.value.status == fsparse.ERR_SIZE
