"""The multi-GPU path of the benchmark on CPU ranks (gloo, world size 2):
ranks are independent replicas with their own reads, and the job time is the
maximum over ranks.  No GPU is needed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        vals = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 7.0 * (rank + 1)], dist)
        out[rank] = (vals, bench.rank_read_seed(rank))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == [11.0, 5.0, 14.0]
    assert res[0][1] != res[1][1]     # each rank queries its own reads


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
