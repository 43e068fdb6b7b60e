"""Several GPUs, one process each (torch.distributed).

* Query: reads are independent, so every rank keeps a replica of the filter
  and queries its own share of the reads (`read_share`); nothing is
  exchanged.
* Insert: every rank inserts its share of the reads into its replica, then
  one bitwise-OR all-reduce of the word array makes all replicas equal to the
  filter of all reads (the filter is the OR of the inserted bits, Alg. 1).
  gloo reduces with ReduceOp.BOR on host words; NCCL has no OR reduction, so
  slices of the words are all-gathered on the device and OR-ed there.
"""
from __future__ import annotations

import numpy as np


def read_share(off: np.ndarray, rank: int, world: int) -> tuple[int, int]:
    """Reads [r0, r1) of rank `rank`: contiguous shares of about equal bytes."""
    off = np.asarray(off, dtype=np.uint64)
    n = off.size - 1
    total = int(off[-1])
    cut = lambda i: int(np.searchsorted(off, (total * i) // world, side="left"))  # noqa: E731
    r0, r1 = min(cut(rank), n), min(cut(rank + 1), n)
    if rank == world - 1:
        r1 = n
    return r0, r1


def allreduce_or_array(words: np.ndarray, group=None) -> np.ndarray:
    """Bitwise OR of every rank's uint64 word array (gloo, host memory)."""
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(words).view(np.int64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.BOR, group=group)
    return t.numpy().view(np.uint64)


def allreduce_or(filt, group=None, slice_words: int = 1 << 25) -> None:
    """Make every rank's filter the OR of all ranks' filters."""
    import torch
    import torch.distributed as dist

    if dist.get_backend(group) != "nccl":
        filt.set_words(allreduce_or_array(filt.words(), group))
        return
    world = dist.get_world_size(group)
    n = filt.n_words
    dev = torch.device("cuda", torch.cuda.current_device())
    mine = torch.empty(min(slice_words, n), dtype=torch.int64, device=dev)
    every = torch.empty(world * mine.numel(), dtype=torch.int64, device=dev)
    for a in range(0, n, slice_words):
        L = min(slice_words, n - a)
        filt.copy_words_device(mine[:L], a)
        dist.all_gather_into_tensor(every[:world * L], mine[:L], group=group)
        parts = every[:world * L].view(world, L)
        acc = parts[0].clone()
        for r in range(1, world):
            acc.bitwise_or_(parts[r])
        filt.copy_words_device(acc, a, to_filter=True)
    torch.cuda.synchronize()


def distributed_insert(filt, seq, off, off_host: np.ndarray, group=None) -> None:
    """Insert reads split over the ranks; every replica ends with all of them.
    seq / off are this rank's device tensors of the whole batch; each rank
    inserts only its share."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    r0, r1 = read_share(off_host, rank, world)
    if r1 > r0:
        a, b = int(off_host[r0]), int(off_host[r1])
        filt.insert(seq[a:b], (off[r0:r1 + 1] - a).contiguous())
    allreduce_or(filt, group)
