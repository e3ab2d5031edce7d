"""Column-sharded assembly through the library's kernels, two ranks sharing
cuda:0 and exchanging over gloo through host buffers (no kernel waits on
another process).  Every rank's column block, its slice's irank, and a
numeric re-assembly must equal the oracle's single assembly, bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(kind):
    from paper_1406_1066_gb300 import inputs
    if kind == "mesh":
        return inputs.mesh3d(24, 63)
    return inputs.random_small(150_000, 5000, 3000, 64, dup=0.5)


def _rank_main(rank, world, port, kind, split_kind, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1406_1066_gb300 import inputs, shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t = _problem(kind)
    lo, hi = t.L * rank // world, t.L * (rank + 1) // world
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    split = None if split_kind == "equal" else [0, t.n // 5, t.n][: world + 1]
    sa = shard.assemble(d(t.ii[lo:hi]), d(t.jj[lo:hi]), d(t.s[lo:hi]), t.m, t.n, col_split=split)
    s2 = inputs.mesh_values(t.L, 65)
    pr2 = sa.numeric(d(s2[lo:hi]))
    torch.cuda.synchronize()
    out.put((rank, dict(jcS=sa.jcS.cpu().numpy(), irS=sa.irS.cpu().numpy(), prS=sa.prS.cpu().numpy(),
                        irank=sa.irank.cpu().numpy(), prS2=pr2[: sa.plan.nnz].cpu().numpy(),
                        total=sa.nnz_total, offset=sa.nnz_offset, lo=lo, hi=hi, split=sa.col_split)))
    sa.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind,split_kind", [("mesh", "equal"), ("random", "equal"), ("random", "uneven")])
def test_column_sharded_assembly_two_ranks(kind, split_kind):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, kind, split_kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1406_1066_gb300 import inputs
    t = _problem(kind)
    ref = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
    ref2 = oracle.numeric(ref.irank, inputs.mesh_values(t.L, 65), ref.nnz)
    for r in range(world):
        g = res[r]
        a, b = g["split"][r], g["split"][r + 1]
        s0, s1 = ref.jcS[a], ref.jcS[b]
        assert g["total"] == ref.nnz and g["offset"] == s0
        np.testing.assert_array_equal(g["jcS"], ref.jcS[a:b + 1])
        np.testing.assert_array_equal(g["irS"], ref.irS[s0:s1])
        assert np.array_equal(g["prS"].view(np.int64), ref.prS[s0:s1].view(np.int64))
        assert np.array_equal(g["prS2"].view(np.int64), ref2[s0:s1].view(np.int64))
        np.testing.assert_array_equal(g["irank"], ref.irank[g["lo"]:g["hi"]])
