"""Parameter sweep parity: every (s, m, H, shard bits) point of the sweep grid
at k = 31, on a 1 Mbp prefix of the bacterial-shaped genome, bit for bit
against the oracle (filter words, query bits, per-read hits)."""
import itertools

import numpy as np
import pytest

from oracle import OracleSBF
from oracle.fpr import conditional_fpr
from paper_2606_24417_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRID = list(itertools.product((24, 26, 28, 31), (12, 14, 16, 20), (1, 2, 4, 8), (256, 512)))


@pytest.fixture(scope="module")
def data():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    g = synth.bacterial_genome(1_000_000, seed=31)
    q, qoff = synth.mixed_query_reads(g, 1000, 1000, 150, 0.01, seed=32)
    return g, q, qoff


@pytest.mark.parametrize("point", GRID, ids=lambda p: "s%d_m%d_H%d_B%d" % p)
def test_sweep_point_bit_exact(point, data):
    from paper_2606_24417_gb300.sbf import SuperBloomFilter
    from paper_2606_24417_gb300.stats import expected_fpr

    s, m, H, B = point
    g, q, qoff = data
    bits = 12 * (g.size - 30)
    f = SuperBloomFilter(31, m, s, H, bits, shard_bits=B)
    assert f.fused
    o = OracleSBF(31, m, s, H, bits, shard_bits=B)
    goff = np.array([0, g.size], dtype=np.uint64)
    f.insert(torch.from_numpy(g).cuda(), torch.from_numpy(goff.astype(np.int64)).cuda())
    o.insert(g, goff)
    words = f.words()
    assert np.array_equal(words, o.words())
    qb, qh = f.query(torch.from_numpy(q).cuda(), torch.from_numpy(qoff.astype(np.int64)).cuda())
    ob, oh = o.query(q, qoff)
    assert np.array_equal(qb.cpu().numpy().view(np.uint32), ob)
    assert np.array_equal(qh.cpu().numpy().view(np.uint32), oh)
    # the sweep's expected-FPR statistic equals the oracle's closed form
    assert abs(expected_fpr(words, 31, s, H, B) - conditional_fpr(words, 31, s, H, B)) <= \
        1e-12 + 1e-9 * conditional_fpr(words, 31, s, H, B)


PAPER_GRID = list(itertools.product((24, 28, 31), (8, 12, 16, 20, 31), (4, 8, 12, 16)))


@pytest.mark.parametrize("point", PAPER_GRID, ids=lambda p: "paper_s%d_m%d_H%d" % p)
def test_paper_layout_sweep_point_bit_exact(point, data):
    """The paper-layout sweep grid (Fig. 5's H in {4, 8, 12, 16}), forward
    strand, 256-bit shards, 2^P of them: the kernel that serves each point
    agrees with the oracle bit for bit."""
    from paper_2606_24417_gb300.sbf import LAYOUT_PAPER, SuperBloomFilter
    from paper_2606_24417_gb300.stats import expected_fpr

    s, m, H = point
    g, q, qoff = data
    bits = 21 * (g.size - 30)
    f = SuperBloomFilter(31, m, s, H, bits, shard_bits=256, canonical=False, layout=LAYOUT_PAPER)
    o = OracleSBF(31, m, s, H, bits, shard_bits=256, canonical=False, layout=1)
    assert f.n_shards == o.n_shards
    goff = np.array([0, g.size], dtype=np.uint64)
    f.insert(torch.from_numpy(g).cuda(), torch.from_numpy(goff.astype(np.int64)).cuda())
    o.insert(g, goff)
    words = f.words()
    assert np.array_equal(words, o.words())
    qb, qh = f.query(torch.from_numpy(q).cuda(), torch.from_numpy(qoff.astype(np.int64)).cuda())
    ob, oh = o.query(q, qoff)
    assert np.array_equal(qb.cpu().numpy().view(np.uint32), ob)
    assert np.array_equal(qh.cpu().numpy().view(np.uint32), oh)
    assert abs(expected_fpr(words, 31, s, H, 256, layout=1) -
               conditional_fpr(words, 31, s, H, 256, layout=1)) <= \
        1e-12 + 1e-9 * conditional_fpr(words, 31, s, H, 256, layout=1)
