"""Column-sharded assembly on several GPUs, one process per GPU.

The paper's multicore method gives every thread a contiguous range of rows
(§3); across GPUs every rank owns a contiguous range of columns instead, so
that the column-compressed result splits into independent blocks (a
distributed output, which §2 names as an extension of the method).  Rank r
holds a slice of the triplets -- the slices taken in rank order are the
whole input -- and:

1. routes every triplet to the owner of its column (``fsparse_shard_route``:
   a stable partition of the slice by destination, columns made local to the
   destination's block);
2. exchanges the routed triplets with one all-to-all (counts first);
3. assembles what it received with the single-GPU path: the received
   triplets are ordered by (source rank, source position), i.e. in global
   triplet order, so every slot is summed in ascending global k exactly as
   in a single assembly;
4. offsets its slots by the exclusive scan of the ranks' nnz, and sends the
   global slots of the routed triplets back (irank of its own slice).

Numeric re-assembly of the same pattern routes only the new values along the
kept route and folds them with the local plan.

The collectives use ``torch.distributed``.  With NCCL the device buffers are
exchanged directly; with gloo (CPU) they go through host copies, which is how
the tests run two ranks on one GPU.  Every step of the assembly itself runs in
the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

from . import fsparse


def _torch():
    import torch
    return torch


def _dist():
    import torch.distributed as dist
    return dist


def column_split(n: int, nranks: int) -> List[int]:
    """Equal contiguous column ranges: rank r owns columns (split[r], split[r+1]]."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    return [n * r // nranks for r in range(nranks + 1)]


def _on_host(group) -> bool:
    return _dist().get_backend(group) == "gloo"


def exchange_counts(counts: Sequence[int], group=None) -> List[int]:
    """All-to-all of one count per destination: returns the counts this rank receives."""
    torch, dist = _torch(), _dist()
    R = dist.get_world_size(group)
    dev = "cpu" if _on_host(group) else torch.device("cuda", torch.cuda.current_device())
    send = torch.tensor([int(c) for c in counts], dtype=torch.int64, device=dev)
    recv = torch.empty(R, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv, send, group=group)
    return [int(x) for x in recv.tolist()]


def exchange(x, send_counts: Sequence[int], recv_counts: Sequence[int], group=None):
    """All-to-all of a 1-D buffer grouped by destination rank; the result is
    grouped by source rank, in source order (through host memory on gloo)."""
    torch, dist = _torch(), _dist()
    host = _on_host(group)
    src = x.cpu() if (host and x.is_cuda) else x
    out = torch.empty(int(sum(recv_counts)), dtype=x.dtype, device=src.device)
    dist.all_to_all_single(out, src.contiguous(), output_split_sizes=[int(c) for c in recv_counts],
                           input_split_sizes=[int(c) for c in send_counts], group=group)
    return out.to(x.device) if out.device != x.device else out


def slot_offset(nnz: int, group=None) -> Tuple[int, int]:
    """(exclusive prefix of the ranks' nnz below this rank, total nnz)."""
    torch, dist = _torch(), _dist()
    R, r = dist.get_world_size(group), dist.get_rank(group)
    dev = "cpu" if _on_host(group) else torch.device("cuda", torch.cuda.current_device())
    mine = torch.tensor([int(nnz)], dtype=torch.int64, device=dev)
    every = [torch.empty(1, dtype=torch.int64, device=dev) for _ in range(R)]
    dist.all_gather(every, mine, group=group)
    vals = [int(t.item()) for t in every]
    return sum(vals[:r]), sum(vals)


@dataclass
class ShardedAssembly:
    """One rank's part of a column-sharded assembly.

    Columns (col_lo, col_hi] (unit offset) are this rank's; ``jcS`` holds
    their n_local + 1 pointers in GLOBAL slot numbers (jcS[0] = nnz_offset),
    ``irS``/``prS`` their nnz_local rows and values, ``irank`` the global
    slot of every triplet of this rank's own input slice.
    """
    rank: int
    nranks: int
    col_split: List[int]
    col_lo: int
    col_hi: int
    nnz_offset: int
    nnz_total: int
    jcS: object
    irS: object
    prS: object
    irank: object
    plan: fsparse.Plan
    send_k: object
    send_counts: List[int]
    recv_counts: List[int]
    group: object = None

    def numeric(self, s, out=None):
        """Re-assemble this rank's columns with new values for its slice."""
        torch = _torch()
        fsparse._dev(s, torch.float64, "s")
        if s.numel() != self.send_k.numel():
            raise ValueError("s has the wrong length for this rank's slice")
        send_s = torch.empty_like(s)
        fsparse.fsparse_shard_gather(s.data_ptr(), self.send_k.data_ptr(), s.numel(), send_s.data_ptr(),
                                     fsparse._stream())
        recv_s = exchange(send_s, self.send_counts, self.recv_counts, self.group)
        return fsparse.numeric(self.plan, recv_s, out)

    def close(self) -> None:
        self.plan.close()


def assemble(ii, jj, s, m: int, n: int, group=None, col_split: Optional[Sequence[int]] = None
             ) -> ShardedAssembly:
    """Column-sharded ``sparse(i, j, s, m, n)`` over the ranks of ``group``.

    ii, jj (int32) and s (float64) are this rank's slice, on its GPU; m and n
    are the global dimensions (explicit).  Every rank calls it.
    """
    torch, dist = _torch(), _dist()
    fsparse._dev(ii, torch.int32, "ii")
    fsparse._dev(jj, torch.int32, "jj")
    fsparse._dev(s, torch.float64, "s")
    L = ii.numel()
    if jj.numel() != L or s.numel() != L:
        raise ValueError("ii, jj and s differ in length")
    R, r = dist.get_world_size(group), dist.get_rank(group)
    split = list(col_split) if col_split is not None else column_split(n, R)
    if len(split) != R + 1:
        raise ValueError("col_split needs nranks + 1 entries")
    dev = ii.device
    send_i = torch.empty(L, dtype=torch.int32, device=dev)
    send_j = torch.empty(L, dtype=torch.int32, device=dev)
    send_s = torch.empty(L, dtype=torch.float64, device=dev)
    send_k = torch.empty(L, dtype=torch.int32, device=dev)
    with torch.cuda.device(dev):
        counts = fsparse.fsparse_shard_route(ii.data_ptr(), jj.data_ptr(), s.data_ptr(), L, m, n, split,
                                             send_i.data_ptr(), send_j.data_ptr(), send_s.data_ptr(),
                                             send_k.data_ptr(), fsparse._stream())
    recv_counts = exchange_counts(counts, group)
    recv_i = exchange(send_i, counts, recv_counts, group)
    recv_j = exchange(send_j, counts, recv_counts, group)
    recv_s = exchange(send_s, counts, recv_counts, group)
    del send_i, send_j, send_s
    n_local = split[r + 1] - split[r]
    jcS_l, irS_l, prS_l, plan = fsparse.assemble(recv_i, recv_j, recv_s, m, n_local)
    offset, total = slot_offset(plan.nnz, group)
    if total > 2**31 - 1:
        raise ValueError("the sharded result has more than 2^31 - 1 slots")
    # global slots of the received triplets, sent back to their sources
    back = torch.empty(recv_i.numel(), dtype=torch.int32, device=dev)
    jcS = torch.empty(n_local + 1, dtype=torch.int32, device=dev)
    irank = torch.empty(L, dtype=torch.int32, device=dev)
    with torch.cuda.device(dev):
        if recv_i.numel():
            fsparse.fsparse_shard_offset(plan.irank.data_ptr(), recv_i.numel(), offset, back.data_ptr(),
                                         fsparse._stream())
        fsparse.fsparse_shard_offset(jcS_l.data_ptr(), n_local + 1, offset, jcS.data_ptr(), fsparse._stream())
    back_mine = exchange(back, recv_counts, counts, group)   # in this rank's send order
    with torch.cuda.device(dev):
        fsparse.fsparse_shard_unroute(back_mine.data_ptr(), send_k.data_ptr(), L, irank.data_ptr(),
                                      fsparse._stream())
    return ShardedAssembly(rank=r, nranks=R, col_split=split, col_lo=split[r], col_hi=split[r + 1],
                           nnz_offset=offset, nnz_total=total, jcS=jcS, irS=irS_l[: plan.nnz],
                           prS=prS_l[: plan.nnz], irank=irank, plan=plan, send_k=send_k, send_counts=counts,
                           recv_counts=recv_counts, group=group)
