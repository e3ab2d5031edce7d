"""Host side of the column-sharded assembly on two gloo ranks (CPU only).

The collectives and offsets of ``paper_1406_1066_gb300.shard`` (count and
buffer all-to-alls, the exclusive scan of the ranks' nnz) run for real; the
device steps are replaced by plain numpy: a stable partition of each rank's
slice by the owner of the column, and the oracle for the local assembly.
The stitched blocks must equal the oracle's assembly of the whole input."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_1406_1066_gb300 import inputs
    return inputs.random_small(40_000, 300, 211, 61, dup=0.5)


def _route_numpy(ii, jj, s, split):
    """Stable partition by destination; columns local to the destination."""
    dest = np.searchsorted(np.asarray(split[1:]), jj, side="left")   # split[d] < j <= split[d+1]
    order = np.argsort(dest, kind="stable")
    counts = np.bincount(dest, minlength=len(split) - 1)
    jl = jj[order] - np.asarray(split)[dest[order]]
    return ii[order], jl.astype(np.int32), s[order], order.astype(np.int32), counts.tolist()


def _rank_main(rank, world, port, split_kind, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1406_1066_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = _problem()
    lo, hi = t.L * rank // world, t.L * (rank + 1) // world        # slices in rank order
    ii, jj, s = t.ii[lo:hi], t.jj[lo:hi], t.s[lo:hi]
    split = shard.column_split(t.n, world) if split_kind == "equal" else [0, 0, t.n][: world + 1]
    si, sj, ss, sk, counts = _route_numpy(ii, jj, s, split)
    recv_counts = shard.exchange_counts(counts)
    ri = shard.exchange(torch.from_numpy(si), counts, recv_counts).numpy()
    rj = shard.exchange(torch.from_numpy(sj), counts, recv_counts).numpy()
    rs = shard.exchange(torch.from_numpy(ss), counts, recv_counts).numpy()
    n_local = split[rank + 1] - split[rank]
    loc = oracle.assemble(ri, rj, rs, t.m, n_local)
    offset, total = shard.slot_offset(loc.nnz)
    back = shard.exchange(torch.from_numpy((loc.irank + offset).astype(np.int32)), recv_counts, counts).numpy()
    irank = np.empty(hi - lo, np.int32)
    irank[sk] = back
    out.put((rank, dict(jcS=loc.jcS + offset, irS=loc.irS[: loc.nnz], prS=loc.prS[: loc.nnz], irank=irank,
                        total=total, lo=lo, hi=hi, split=split)))
    dist.destroy_process_group()


@pytest.mark.parametrize("split_kind", ["equal", "all_on_rank_1"])
def test_column_sharded_host_logic_gloo(split_kind):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, split_kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import oracle
    t = _problem()
    ref = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
    for r in range(world):
        g = res[r]
        a, b = g["split"][r], g["split"][r + 1]
        assert g["total"] == ref.nnz
        np.testing.assert_array_equal(g["jcS"], ref.jcS[a:b + 1])
        s0, s1 = ref.jcS[a], ref.jcS[b]
        np.testing.assert_array_equal(g["irS"], ref.irS[s0:s1])
        assert np.array_equal(g["prS"].view(np.int64), ref.prS[s0:s1].view(np.int64))
        np.testing.assert_array_equal(g["irank"], ref.irank[g["lo"]:g["hi"]])


def test_column_split_ranges():
    sys.path.insert(0, ROOT)
    from paper_1406_1066_gb300 import shard
    assert shard.column_split(10, 3) == [0, 3, 6, 10]
    assert shard.column_split(2, 4) == [0, 0, 1, 1, 2]
    assert shard.column_split(7, 1) == [0, 7]
    with pytest.raises(ValueError):
        shard.column_split(5, 0)
