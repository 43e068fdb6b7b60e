"""Several GPUs, one process each (torch.distributed).

* Query: reads are independent, so every rank keeps a replica of the filter
  and queries its own share of the reads (`read_share`); nothing is
  exchanged.
* Insert: every rank inserts its share of the reads into its replica, then
  one bitwise-OR all-reduce of the word array makes all replicas equal to the
  filter of all reads (the filter is the OR of the inserted bits, Alg. 1).
  gloo reduces with ReduceOp.BOR on host words.  NCCL has no OR reduction,
  so the words go through an all-to-all (each rank receives every rank's
  piece of its own slice), a device OR of those pieces and an all-gather of
  the OR-ed slices: each rank moves 2 (world - 1) / world of the words.
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


def sharded_or_allreduce(n_words: int, read_chunk, write_chunk, combine, new_buffer,
                         group=None, slice_words: int = 1 << 25) -> None:
    """OR all-reduce of an n_words array held by every rank, shaped like a
    reduce-scatter followed by an all-gather (no library offers an OR
    reduction on the device).  Per chunk of at most slice_words words:

    1. read_chunk(buf, a) fills buf with this rank's words [a, a + len(buf));
       the chunk is padded with zeros to world equal pieces of P words;
    2. all-to-all: rank r receives piece r of every rank;
    3. combine(out, parts) ORs the (world, P) received pieces into out;
    4. all-gather of the combined pieces rebuilds the chunk on every rank;
    5. write_chunk(buf, a) stores it.

    Each rank sends and receives 2 (world - 1) / world of the words, as a
    ring all-reduce would.  new_buffer(n) returns an int64 tensor of n
    elements on the collective's device."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    cap = min(slice_words, n_words)
    pmax = -(-cap // world)
    pmax += pmax & 1                      # even pieces keep 16-byte alignment
    send, recv, full = new_buffer(world * pmax), new_buffer(world * pmax), new_buffer(world * pmax)
    mine = new_buffer(pmax)
    for a in range(0, n_words, slice_words):
        L = min(slice_words, n_words - a)
        P = -(-L // world)
        P += P & 1
        read_chunk(send[:L], a)
        send[L:world * P].zero_()
        dist.all_to_all_single(recv[:world * P], send[:world * P], group=group)
        combine(mine[:P], recv[:world * P].view(world, P))
        dist.all_gather_into_tensor(full[:world * P], mine[:P], group=group)
        write_chunk(full[:L], a)


def allreduce_or(filt, group=None, slice_words: int = 1 << 25) -> None:
    """Make every rank's filter the OR of all ranks' filters."""
    import torch
    import torch.distributed as dist

    if dist.get_backend(group) != "nccl":
        filt.set_words(allreduce_or_array(filt.words(), group))
        return
    from .sbf import or_reduce_device

    dev = torch.device("cuda", torch.cuda.current_device())
    sharded_or_allreduce(
        filt.n_words,
        read_chunk=lambda buf, a: filt.copy_words_device(buf, a),
        write_chunk=lambda buf, a: filt.copy_words_device(buf, a, to_filter=True),
        combine=lambda out, parts: or_reduce_device(out, parts),
        new_buffer=lambda n: torch.empty(n, dtype=torch.int64, device=dev),
        group=group, slice_words=slice_words)
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
