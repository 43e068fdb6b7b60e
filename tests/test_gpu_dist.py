"""The multi-GPU insert path run as one NCCL rank on one GPU: the device word
copies and the sliced OR all-reduce leave the filter equal to the oracle's
(with one rank the OR is the identity, so the filter must not change), and
read shares cover every read once.  Ranks on several GPUs are not run here
(one GPU per run); the OR of two ranks' filters is checked with gloo on CPU."""
import os
import socket

import numpy as np
import pytest

from oracle import OracleSBF
from paper_2606_24417_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nccl_one_rank():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.distributed as dist

    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    yield dist
    dist.destroy_process_group()


def test_device_word_copies(nccl_one_rank):
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    f = SuperBloomFilter(31, 16, 28, 4, 1 << 20)
    g = synth.uniform_dna(50_000, 3)
    f.insert(torch.from_numpy(g).cuda(), torch.tensor([0, g.size], dtype=torch.int64).cuda())
    w = f.words()
    part = torch.empty(1000, dtype=torch.int64, device="cuda")
    f.copy_words_device(part, word_begin=777)
    assert np.array_equal(part.cpu().numpy().view(np.uint64), w[777:1777])
    part.fill_(0)
    f.copy_words_device(part, word_begin=777, to_filter=True)
    w2 = f.words()
    assert not w2[777:1777].any() and np.array_equal(w2[:777], w[:777])


def test_distributed_insert_one_rank(nccl_one_rank):
    from paper_2606_24417_gb300.dist import allreduce_or, distributed_insert
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    g = synth.bacterial_genome(300_000, seed=7)
    seq, off = synth.sample_reads(g, 4000, 150, 0.01, seed=8)
    f = SuperBloomFilter(31, 16, 28, 4, 1 << 22)
    distributed_insert(f, torch.from_numpy(seq).cuda(), torch.from_numpy(off.astype(np.int64)).cuda(), off)
    o = OracleSBF(31, 16, 28, 4, 1 << 22)
    o.insert(seq, off)
    assert np.array_equal(f.words(), o.words())
    allreduce_or(f, slice_words=10_000)   # several slices; one rank: unchanged
    assert np.array_equal(f.words(), o.words())


def test_read_shares_cover_all_reads():
    from paper_2606_24417_gb300.dist import read_share

    off = np.concatenate([[0], np.cumsum(synth.lognormal_lengths(1000, 150, 1.0, 0, 5000, 3))]).astype(np.uint64)
    for world in (1, 2, 3, 8):
        shares = [read_share(off, r, world) for r in range(world)]
        assert shares[0][0] == 0 and shares[-1][1] == off.size - 1
        assert all(shares[i][1] == shares[i + 1][0] for i in range(world - 1))


@pytest.mark.parametrize("n_parts,n", [(1, 1), (1, 1001), (3, 1000), (8, 1 << 20), (2, 2)])
def test_or_reduce_kernel(n_parts, n):
    """The device OR of the multi-GPU insert: out[i] = OR of parts[j, i],
    against torch's OR of the same rows (odd lengths with one part, even
    lengths with several: every piece stays 16-byte aligned)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    from paper_2606_24417_gb300.sbf import SbfError, or_reduce_device

    g = torch.Generator(device="cpu").manual_seed(n_parts * 1000 + n)
    a = torch.randint(-(1 << 62), 1 << 62, (n_parts, n), generator=g, dtype=torch.int64)
    a &= torch.randint(-(1 << 62), 1 << 62, (n_parts, n), generator=g, dtype=torch.int64)
    parts = a.cuda()
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    or_reduce_device(out, parts)
    want = a[0].clone()
    for r in range(1, n_parts):
        want |= a[r]
    assert torch.equal(out.cpu(), want)
    if n_parts == 3:
        with pytest.raises(SbfError):      # pieces of an odd length would be misaligned
            or_reduce_device(out[:999], parts[:, :999].contiguous())
