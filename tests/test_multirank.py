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


def _or_worker(rank, world, port, out, genome_path, params):
    import numpy as np
    import torch.distributed as dist

    from oracle import OracleSBF
    from paper_2606_24417_gb300.dist import allreduce_or_array, read_share

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data = np.load(genome_path)
        seq, off = data["seq"], data["off"]
        r0, r1 = read_share(off, rank, world)
        o = OracleSBF(*params)
        a, b = int(off[r0]), int(off[r1])
        o.insert(seq[a:b], off[r0:r1 + 1] - off[r0])   # this rank's share only
        out[rank] = (r0, r1, allreduce_or_array(o.words()).tobytes())
    finally:
        dist.destroy_process_group()


def test_distributed_insert_or_allreduce_two_gloo_ranks(tmp_path):
    """Two ranks insert disjoint read shares into their own filters; one OR
    all-reduce gives both the filter of all reads (Alg. 1: insertion is the
    OR of the inserted bits)."""
    import numpy as np
    import torch.multiprocessing as mp

    from oracle import OracleSBF
    from paper_2606_24417_gb300 import synth

    g = synth.bacterial_genome(400_000, seed=5)
    seq, off = synth.sample_reads(g, 3000, 150, 0.01, seed=6)
    p = str(tmp_path / "reads.npz")
    np.savez(p, seq=seq, off=off)
    params = (31, 16, 28, 4, 1 << 22)
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_or_worker, args=(2, port, out, p, params), nprocs=2, join=True)
        res = dict(out)
    full = OracleSBF(*params)
    full.insert(seq, off)
    want = full.words().tobytes()
    assert res[0][2] == want and res[1][2] == want
    assert res[0][0] == 0 and res[0][1] == res[1][0] and res[1][1] == off.size - 1


def _sharded_worker(rank, world, port, out, n_words, slice_words):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2606_24417_gb300.dist import sharded_or_allreduce

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(100 + rank)
        # sparse words so that the OR of the ranks differs from each rank's words
        mine = rng.integers(0, 1 << 63, n_words, dtype=np.int64) & rng.integers(0, 1 << 63, n_words,
                                                                                  dtype=np.int64)
        result = np.zeros(n_words, dtype=np.int64)

        def read_chunk(buf, a):
            buf.copy_(torch.from_numpy(mine[a:a + buf.numel()]))

        def write_chunk(buf, a):
            result[a:a + buf.numel()] = buf.numpy()

        def combine(o, parts):
            acc = parts[0].clone()
            for r in range(1, parts.shape[0]):
                acc.bitwise_or_(parts[r])
            o.copy_(acc)

        sharded_or_allreduce(n_words, read_chunk, write_chunk, combine,
                             lambda n: torch.empty(n, dtype=torch.int64), slice_words=slice_words)
        out[rank] = result.tobytes()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_words,slice_words", [(2, 1001, 300), (3, 64, 1 << 25), (2, 7, 4)])
def test_sharded_or_allreduce_gloo(world, n_words, slice_words):
    """The reduce-scatter-shaped OR all-reduce of the multi-GPU insert
    (all-to-all of pieces, OR of the pieces of one's own slice, all-gather),
    run on CPU ranks with a host OR in place of the device kernel: ragged
    chunks and pieces padded to an even length give every rank the OR of all
    ranks' words."""
    import numpy as np
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_sharded_worker, args=(world, port, out, n_words, slice_words), nprocs=world,
                 join=True)
        res = dict(out)
    want = np.zeros(n_words, dtype=np.int64)
    for r in range(world):
        rng = np.random.default_rng(100 + r)
        want |= rng.integers(0, 1 << 63, n_words, dtype=np.int64) & rng.integers(
            0, 1 << 63, n_words, dtype=np.int64)
    for r in range(world):
        assert res[r] == want.tobytes(), r


class _HostFilter:
    """A CPU stand-in for SuperBloomFilter with the three calls the
    multi-GPU insert makes (insert, words, set_words), backed by the oracle."""

    def __init__(self, params):
        from oracle import OracleSBF

        self.o = OracleSBF(*params)
        self.n_words = self.o.n_words

    def insert(self, seq, off):
        import numpy as np

        self.o.insert(seq.numpy().astype(np.uint8), off.numpy().astype(np.uint64))

    def words(self):
        return self.o.words()

    def set_words(self, w):
        self.o.set_words(w)


def _dist_insert_worker(rank, world, port, out, reads_path, params):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2606_24417_gb300.dist import distributed_insert

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data = np.load(reads_path)
        seq, off = data["seq"], data["off"]
        filt = _HostFilter(params)
        distributed_insert(filt, torch.from_numpy(seq), torch.from_numpy(off.astype(np.int64)),
                           off)
        out[rank] = filt.words().tobytes()
    finally:
        dist.destroy_process_group()


def test_distributed_insert_through_the_product_module(tmp_path):
    """dist.distributed_insert itself (read shares, then allreduce_or) on two
    gloo ranks: both replicas end as the filter of all reads."""
    import numpy as np
    import torch.multiprocessing as mp

    from oracle import OracleSBF
    from paper_2606_24417_gb300 import synth

    g = synth.bacterial_genome(300_000, seed=8)
    seq, off = synth.sample_reads(g, 2500, 150, 0.01, seed=9)
    p = str(tmp_path / "reads.npz")
    np.savez(p, seq=seq, off=off)
    params = (31, 16, 28, 4, 1 << 21)
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_dist_insert_worker, args=(2, port, out, p, params), nprocs=2, join=True)
        res = dict(out)
    full = OracleSBF(*params)
    full.insert(seq, off)
    want = full.words().tobytes()
    assert res[0] == want and res[1] == want
