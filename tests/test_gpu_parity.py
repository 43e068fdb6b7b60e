"""GPU parity: libsbf (through the C ABI) against the oracle, bit for bit.

Integer work, so the bar is exact equality of the filter words, of every
query bit and of every per-read hit count.  Inputs are seeded synthetic
workloads; sizes span many kernel tiles with ragged tails, and the
bacterial-genome workload runs at full size with sampled answers checked.
"""
import os

import numpy as np
import pytest

from oracle import OracleSBF
from paper_2606_24417_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def dev_off(off):
    return dev(np.asarray(off, dtype=np.uint64).astype(np.int64))


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def make_filter(k, m, s, H, bits, B=512, canonical=True, layout=0):
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    return SuperBloomFilter(k, m, s, H, bits, shard_bits=B, canonical=canonical, layout=layout)


def check_insert_query(params, ins_seq, ins_off, q_seq, q_off, check_stats=True):
    k, m, s, H, bits, B, canon, *rest = params
    layout = rest[0] if rest else 0
    f = make_filter(k, m, s, H, bits, B, canon, layout)
    o = OracleSBF(k, m, s, H, bits, shard_bits=B, canonical=canon, layout=layout)
    assert f.n_shards == o.n_shards
    f.insert(dev(ins_seq), dev_off(ins_off))
    o.insert(ins_seq, ins_off)
    assert np.array_equal(f.words(), o.words()), f"words differ for {params}"
    stats = torch.zeros(3, dtype=torch.int64, device="cuda") if check_stats else None
    qb, qh = f.query(dev(q_seq), dev_off(q_off), stats=stats)
    ob, oh = o.query(q_seq, q_off)
    gb = u32(qb)
    if not np.array_equal(gb, ob):
        bad = np.nonzero(gb != ob)[0][:5]
        raise AssertionError(f"query bits differ for {params} at words {bad}: "
                             f"{gb[bad]} vs {ob[bad]}")
    assert np.array_equal(u32(qh), oh), f"hits differ for {params}"
    if check_stats:
        valid, runs = o.count_runs(q_seq, q_off)
        st = stats.cpu().numpy()
        assert st[0] == valid and st[1] == runs and st[2] == int(oh.sum()), (st, valid, runs)
    return f, o


def ragged_reads(n_reads, seed, genome=None, median=150, sigma=1.2, hi=5000, n_frac=0.0005):
    """Reads of lognormal lengths (some shorter than k, some empty), part sampled
    from `genome`, with scattered invalid bytes and lower-case stretches."""
    lens = synth.lognormal_lengths(n_reads, median, sigma, 0, hi, seed)
    total = int(lens.sum())
    seq = synth.uniform_dna(total, seed + 1)
    if genome is not None:
        src = synth.randint(seed, 3, n_reads, 0, max(1, genome.size - hi))
        pos = 0
        for i, L in enumerate(lens):
            if i % 2 == 0 and L:
                seq[pos:pos + L] = genome[src[i]:src[i] + L]
            pos += L
    u = synth.uniform01(seed, 5, 0, total)
    seq[u < n_frac] = ord("N")
    seq[(u > 0.3) & (u < 0.3 + 0.02)] += 32  # lower case
    off = np.zeros(n_reads + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    return seq, off


# ---------------------------------------------------------------------------
# the tiny workload: 1 Mbp uniform random, 2^24 bits in 512-bit shards
# ---------------------------------------------------------------------------
def test_tiny_uniform_1mbp_bit_exact():
    g = synth.uniform_dna(1_000_000, 0)
    goff = np.array([0, g.size], dtype=np.uint64)
    other = synth.uniform_dna(1_000_000, 1)
    q = np.concatenate([g, other])
    qoff = np.array([0, g.size, q.size], dtype=np.uint64)
    f, o = check_insert_query((31, 16, 28, 4, 1 << 24, 512, True), g, goff, q, qoff)
    _, oh = o.query(q, qoff)
    assert int(oh[0]) == 1_000_000 - 31 + 1   # every inserted k-mer is found


PARAMS = [
    # k, m, s, H, bits, B, canonical
    (31, 16, 28, 4, 1 << 22, 512, True),
    (31, 16, 28, 4, 1 << 21, 256, True),
    (31, 16, 28, 4, 3_000_000, 512, False),
    (31, 12, 24, 8, 1 << 22, 512, True),
    (31, 14, 26, 2, 1 << 22, 256, True),
    (31, 20, 31, 1, 1 << 22, 512, True),
    (31, 16, 28, 8, 1 << 22, 256, True),
    (31, 20, 24, 4, 1 << 23, 512, True),
    (31, 12, 31, 2, 1 << 22, 512, True),
    (31, 16, 28, 16, 1 << 22, 512, True),   # salted multiply
    (9, 5, 6, 2, 1 << 16, 256, True),       # Fig. 2 parameters
    (32, 16, 30, 4, 1 << 22, 512, True),
    (21, 11, 17, 12, 5000 * 512, 512, True),
    # the paper's literal layout (Sec. IV-B, Alg. 1/2): k, m, s, H, bits, B, canonical, layout
    (31, 16, 28, 4, 1 << 21, 256, False, 1),     # fused
    (31, 16, 28, 8, 3_000_000, 256, True, 1),    # fused; 11,719 shards rounded up to 16,384
    (31, 20, 24, 4, 1 << 22, 256, True, 1),      # fused, 64-bit order keys
    (31, 12, 24, 8, 1 << 22, 256, False, 1),     # fused, w = 20
    (31, 16, 28, 2, 1 << 21, 256, False, 1),     # generic: words 2, 3 unused
    (31, 16, 28, 12, 1 << 21, 256, False, 1),    # generic: salted multiply (Fig. 5 H = 12)
    (31, 16, 28, 16, 1 << 21, 256, True, 1),     # generic: H = 16
]


@pytest.mark.parametrize("params", PARAMS, ids=lambda p: "_".join(map(str, p)))
def test_ragged_reads_bit_exact(params):
    genome = synth.uniform_dna(300_000, 7)
    ins_seq, ins_off = ragged_reads(1500, 11, genome)
    q_seq, q_off = ragged_reads(2500, 12, genome)
    check_insert_query(params, ins_seq, ins_off, q_seq, q_off)


def test_edge_cases():
    params = (31, 16, 28, 4, 1 << 20, 512, True)
    f = make_filter(*params[:5], params[5], params[6])
    o = OracleSBF(*params[:5], shard_bits=params[5])
    # empty batch
    f.insert(dev(np.zeros(0, np.uint8)), dev_off([0]))
    qb, qh = f.query(dev(np.zeros(0, np.uint8)), dev_off([0]))
    assert qb.numel() == 0 and qh.numel() == 0
    # reads shorter than k, exactly k, all-N, separators at every offset
    g = synth.uniform_dna(5000, 3)
    reads = [g[:30], g[30:61], np.full(100, ord("N"), np.uint8), g[:0], g[100:131]]
    for p in range(0, 31, 5):
        r = g[200:262].copy()
        r[p] = ord("N")
        reads.append(r)
    seq, off = synth.concat(reads)
    f.insert(dev(seq), dev_off(off))
    o.insert(seq, off)
    assert np.array_equal(f.words(), o.words())
    qb, qh = f.query(dev(seq), dev_off(off))
    ob, oh = o.query(seq, off)
    assert np.array_equal(u32(qb), ob) and np.array_equal(u32(qh), oh)
    assert oh[0] == 0 and oh[1] == 1 and oh[2] == 0 and oh[3] == 0 and oh[4] == 1


@pytest.mark.parametrize("params", [(31, 16, 28, 4, 1 << 22, 512, True),
                                    (31, 20, 24, 4, 1 << 22, 256, True)],
                         ids=lambda p: "_".join(map(str, p)))
def test_many_short_reads(params):
    """Reads of 0-40 bases: more than 32 read ends fall in one kernel window,
    so the boundary loops take several batches; most reads hold no k-mer."""
    lens = synth.randint(61, 1, 60000, 0, 41)
    seq = synth.uniform_dna(int(lens.sum()), 62)
    off = np.zeros(lens.size + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    check_insert_query(params, seq, off, seq, off)


@pytest.mark.parametrize("params", [(31, 16, 28, 4, 1 << 22, 512, True),   # fused kernels
                                    (31, 20, 24, 8, 1 << 22, 256, True)],  # fused, 64-bit keys
                         ids=lambda p: "_".join(map(str, p)))
@pytest.mark.parametrize("hits_pass", [True, False], ids=["pass", "in_kernel"])
def test_read_hits_at_the_short_read_limit(params, hits_pass, monkeypatch):
    """With both outputs on a large enough launch, the query kernel counts
    hits of reads longer than 2048 positions and a second pass counts the
    rest from the answer words; otherwise the kernel counts every read.
    Reads of lengths around the limit, mixed with short, empty and long reads
    in a shuffled order, give the oracle's hits both ways on the device path
    (the pass is forced onto this small input by its knob), and on the host
    path, which counts every read in the kernel."""
    if hits_pass:
        monkeypatch.setenv("SBF_HITS_PASS_MIN_POSITIONS", "0")
    else:
        monkeypatch.delenv("SBF_HITS_PASS_MIN_POSITIONS", raising=False)
    genome = synth.uniform_dna(400_000, 71)
    lens = [0, 1, 30, 31, 32, 150, 2046, 2047, 2048, 2049, 2050, 2079, 2080, 4096, 20_000,
            150, 151, 2048, 0, 2049, 60_000] * 6
    lens = np.asarray(lens, dtype=np.int64)[synth.randint(72, 1, len(lens), 0, 1 << 30).argsort()]
    src = synth.randint(73, 1, lens.size, 0, genome.size - 60_001)
    reads = []
    for i, L in enumerate(lens):
        r = genome[src[i]:src[i] + L].copy() if i % 3 else synth.uniform_dna(int(L), 74 + i)
        reads.append(r)
    seq, off = synth.concat(reads)
    f, o = check_insert_query(params, genome, np.array([0, genome.size], np.uint64), seq, off)
    ob, oh = o.query(seq, off)
    assert int(oh[lens > 2048].sum()) > 0 and int(oh[(lens > 0) & (lens <= 2048)].sum()) > 0
    qb, _ = f.query(dev(seq), dev_off(off), want_hits=False)
    _, qh = f.query(dev(seq), dev_off(off), want_bits=False)
    assert np.array_equal(u32(qb), ob) and np.array_equal(u32(qh), oh)
    monkeypatch.setenv("SBF_HOST_CHUNK_BYTES", "50000")   # chunk seams between long reads
    hb, hh = f.query_host(seq, off)
    assert np.array_equal(hb, ob) and np.array_equal(hh, oh)
    _, hh2 = f.query_host(seq, off, want_bits=False)
    assert np.array_equal(hh2, oh)
    f.close()


def test_insert_order_and_repeats_on_gpu():
    params = (31, 16, 28, 4, 1 << 21, 512, True)
    seq, off = ragged_reads(3000, 21)
    f1 = make_filter(*params[:5], params[5], params[6])
    f1.insert(dev(seq), dev_off(off))
    # reversed read order, inserted twice
    lens = np.diff(off.astype(np.int64))
    reads = [seq[int(off[i]):int(off[i + 1])] for i in range(len(lens))][::-1]
    s2, o2 = synth.concat(reads)
    f2 = make_filter(*params[:5], params[5], params[6])
    f2.insert(dev(s2), dev_off(o2))
    f2.insert(dev(s2), dev_off(o2))
    assert np.array_equal(f1.words(), f2.words())
    # highly repetitive input (contention on few shards)
    rep = np.tile(synth.uniform_dna(500, 4), 400)
    check_insert_query(params, rep, np.array([0, rep.size], np.uint64), rep,
                       np.array([0, rep.size], np.uint64))


@pytest.mark.parametrize("params", [(31, 16, 28, 4, 1 << 22, 512, True),   # fused kernels
                                    (9, 5, 6, 2, 1 << 18, 256, True)],     # generic kernels
                         ids=["fused", "generic"])
def test_host_path_matches_device(monkeypatch, params):
    ins_seq, ins_off = ragged_reads(4000, 31)
    q_seq, q_off = ragged_reads(6000, 32)
    monkeypatch.setenv("SBF_HOST_CHUNK_BYTES", "40000")   # many chunk seams
    f = make_filter(*params[:5], params[5], params[6])
    assert f.fused == (params[0] == 31)
    f.insert_host(ins_seq, ins_off)
    o = OracleSBF(*params[:5], shard_bits=params[5])
    o.insert(ins_seq, ins_off)
    assert np.array_equal(f.words(), o.words())
    hb, hh = f.query_host(q_seq, q_off)
    ob, oh = o.query(q_seq, q_off)
    assert np.array_equal(hb, ob) and np.array_equal(hh, oh)
    # pinned output buffers (answers copied straight in) give the same as the
    # pageable ones above (answers staged through pinned memory)
    pb = torch.empty(hb.size, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    ph = torch.empty(hh.size, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    f.query_host(q_seq, q_off, bits=pb, hits=ph)
    assert np.array_equal(pb, ob) and np.array_equal(ph, oh)
    # pinned inputs (copied in by chunks like pageable ones, without the
    # staging step): same answers, same filter
    pq = torch.from_numpy(q_seq).pin_memory().numpy()
    po = torch.from_numpy(q_off.view(np.int64)).pin_memory().numpy().view(np.uint64)
    f.query_host(pq, po, bits=pb, hits=ph)
    assert np.array_equal(pb, ob) and np.array_equal(ph, oh)
    f2 = make_filter(*params[:5], params[5], params[6])
    f2.insert_host(torch.from_numpy(ins_seq).pin_memory().numpy(),
                   torch.from_numpy(ins_off.view(np.int64)).pin_memory().numpy().view(np.uint64))
    assert np.array_equal(f2.words(), o.words())
    monkeypatch.delenv("SBF_HOST_CHUNK_BYTES")
    hb2, hh2 = f.query_host(q_seq, q_off)
    assert np.array_equal(hb2, ob) and np.array_equal(hh2, oh)


@pytest.mark.parametrize("layout", [0, 1])
def test_checkpoint_roundtrip(tmp_path, layout):
    params = (31, 16, 28, 4, 1000 * 256, 256, False)
    seq, off = ragged_reads(500, 41)
    f = make_filter(*params[:5], params[5], params[6], layout)
    f.insert(dev(seq), dev_off(off))
    p = tmp_path / "f.sbf"
    f.save(str(p))
    g = type(f).load(str(p))
    assert (g.k, g.m, g.s, g.H, g.shard_bits, g.canonical, g.layout, g.n_shards) == \
        (31, 16, 28, 4, 256, False, layout, f.n_shards)
    assert np.array_equal(f.words(), g.words())
    qb1, qh1 = f.query(dev(seq), dev_off(off))
    qb2, qh2 = g.query(dev(seq), dev_off(off))
    assert torch.equal(qb1, qb2) and torch.equal(qh1, qh2)


def test_paper_layout_kernel_choice():
    assert make_filter(31, 16, 28, 4, 1 << 20, 256, False, 1).fused
    assert make_filter(31, 16, 28, 8, 1 << 20, 256, False, 1).fused
    assert not make_filter(31, 16, 28, 2, 1 << 20, 256, False, 1).fused
    f = make_filter(31, 16, 28, 4, 3 * 256 * 1000, 256, False, 1)
    assert f.n_shards == 4096 and f.layout == 1


def test_fused_grid_is_used():
    for params in [(31, 16, 28, 4, 512), (31, 12, 24, 8, 256), (31, 14, 26, 2, 512),
                   (31, 20, 24, 1, 256)]:
        k, m, s, H, B = params
        assert make_filter(k, m, s, H, 1 << 20, B).fused, params
    assert not make_filter(9, 5, 6, 2, 1 << 16, 256).fused


@pytest.mark.parametrize("params", [(31, 16, 28, 4, 1 << 26, 512, True),
                                    (31, 12, 24, 8, 1 << 25, 256, True),
                                    (31, 20, 26, 2, 1 << 26, 512, False)],
                         ids=lambda p: "_".join(map(str, p)))
def test_fused_matches_generic_large(params, monkeypatch):
    """Fused against generic kernels (a second, independent GPU path) on a
    20 Mbp genome and 1M reads: identical words, bits and hits."""
    k, m, s, H, bits, B, canon = params
    g = synth.bacterial_genome(20_000_000, seed=8)
    goff = np.array([0, g.size], dtype=np.uint64)
    q, qoff = synth.mixed_query_reads(g, 500_000, 500_000, 150, 0.01, seed=9)
    monkeypatch.setenv("SBF_FORCE_GENERIC", "1")
    fg = make_filter(k, m, s, H, bits, B, canon)
    monkeypatch.delenv("SBF_FORCE_GENERIC")
    ff = make_filter(k, m, s, H, bits, B, canon)
    assert ff.fused and not fg.fused
    dg, dgo, dq, dqo = dev(g), dev_off(goff), dev(q), dev_off(qoff)
    fg.insert(dg, dgo)
    ff.insert(dg, dgo)
    assert np.array_equal(fg.words(), ff.words())
    sg = torch.zeros(3, dtype=torch.int64, device="cuda")
    sf = torch.zeros(3, dtype=torch.int64, device="cuda")
    bg, hg = fg.query(dq, dqo, stats=sg)
    bf, hf = ff.query(dq, dqo, stats=sf)
    assert torch.equal(bg, bf) and torch.equal(hg, hf) and torch.equal(sg, sf)


@pytest.mark.parametrize("params", [(31, 16, 28, 4, 1 << 33, 512, True),
                                    (31, 16, 26, 8, 1 << 33, 256, True),
                                    (31, 20, 26, 4, 1 << 33, 512, True)],
                         ids=lambda p: "_".join(map(str, p)))
def test_large_filter_bulk_copies(params):
    """Filters of 1 GiB load part of their shards with TMA bulk copies on an
    mbarrier (slots from 32 on of an iteration; up to 95 for the w = 12
    kernel): words, bits and hits equal the oracle's, and no wait ran out."""
    g = synth.bacterial_genome(3_000_000, seed=31)
    goff = np.array([0, g.size], dtype=np.uint64)
    q, qoff = ragged_reads(60_000, 32, genome=g)
    f, o = check_insert_query(params, g, goff, q, qoff)
    assert f.fused and f.nbytes >= 1 << 30
    # the host entry point takes the same kernels and checks the status word itself
    hb, hh = f.query_host(q, qoff)
    ob, oh = o.query(q, qoff)
    assert np.array_equal(hb, ob) and np.array_equal(hh, oh)
    assert f.device_status() == 0
    f.close()


def test_batch_mixes_bulk_and_plain_copies():
    """One persistent launch over a 1 GiB filter (bulk copies) and a 4 MiB
    one (cp.async only): every warp switches between the two per segment;
    answers equal the single-filter calls."""
    from paper_2606_24417_gb300.sbf import BATCH_FUSED, BATCH_GRAPH, FilterBatch

    g = synth.bacterial_genome(2_000_000, seed=33)
    goff = np.array([0, g.size], dtype=np.uint64)
    big = make_filter(31, 16, 28, 4, 1 << 33)
    small = make_filter(31, 16, 28, 4, 1 << 25)
    for f in (big, small):
        f.insert(dev(g), dev_off(goff))
    qa, qa_off = ragged_reads(30_000, 34, genome=g)
    qb, qb_off = ragged_reads(30_000, 35, genome=g)
    seq = np.concatenate([qa, qb])
    off = np.concatenate([qa_off, qa_off[-1] + qb_off[1:]]).astype(np.uint64)
    group = np.array([0, qa_off.size - 1, off.size - 1], dtype=np.uint64)
    ref_bits, ref_hits = [], []
    for f, (qs, qo) in ((big, (qa, qa_off)), (small, (qb, qb_off))):
        bb, hh = f.query(dev(qs), dev_off(qo))
        ref_bits.append(u32(bb))
        ref_hits.append(u32(hh))
    batch = FilterBatch([big, small])
    for mode in (BATCH_FUSED, BATCH_GRAPH):
        for dynamic in (False, True):
            batch.set_schedule(dynamic, 4)
            bits, hits = batch.query(dev(seq), dev_off(off), off, group, mode=mode)
            hb = u32(hits)
            assert np.array_equal(hb[:qa_off.size - 1], ref_hits[0])
            assert np.array_equal(hb[qa_off.size - 1:], ref_hits[1])
            # answer bits of the first group's positions (its reads end where the second begin)
            na = int(qa_off[-1])
            gb = u32(bits)
            assert np.array_equal(gb[:na // 32], ref_bits[0][:na // 32])
    assert big.device_status() == 0 and small.device_status() == 0
    batch.close()
    big.close()
    small.close()


def test_unaligned_sequence_pointer():
    params = (31, 16, 28, 4, 1 << 22, 512, True)
    seq, off = ragged_reads(2000, 51)
    buf = torch.empty(seq.size + 3, dtype=torch.uint8, device="cuda")
    buf[3:] = dev(seq)
    dseq = buf[3:]
    assert dseq.data_ptr() % 16 != 0
    f = make_filter(*params[:5], params[5], params[6])
    o = OracleSBF(*params[:5], shard_bits=params[5])
    f.insert(dseq, dev_off(off))
    o.insert(seq, off)
    assert np.array_equal(f.words(), o.words())
    qb, qh = f.query(dseq, dev_off(off))
    ob, oh = o.query(seq, off)
    assert np.array_equal(u32(qb), ob) and np.array_equal(u32(qh), oh)


# ---------------------------------------------------------------------------
# bacterial-genome workload at full size: 100 Mbp Markov genome with repeats,
# 2^30-bit filter, 10M sampled reads (1% errors) + 10M random 150 bp reads
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def bacterial():
    g = synth.bacterial_genome(100_000_000, seed=2)
    q, qoff = synth.mixed_query_reads(g, 10_000_000, 10_000_000, 150, 0.01, seed=3)
    return g, q, qoff


def test_bacterial_full_size(bacterial, tmp_path):
    g, q, qoff = bacterial
    params = (31, 16, 28, 4, 1 << 30, 512, True)
    f = make_filter(*params[:5], params[5], params[6])
    goff = np.array([0, g.size], dtype=np.uint64)
    dg = dev(g)
    f.insert(dg, dev_off(goff))
    o = OracleSBF(*params[:5], shard_bits=params[5])
    o.insert(g, goff)
    assert np.array_equal(f.words(), o.words())   # the whole 128 MiB filter
    # every genome k-mer is positive
    _, gh = f.query(dg, dev_off(goff), want_bits=False)
    assert int(u32(gh)[0]) == g.size - 30
    del dg
    # the 20M-read query in the launch configuration the benchmark times
    dq = dev(q)
    qb, qh = f.query(dq, dev_off(qoff))
    bits = u32(qb)
    hits = u32(qh)
    rng = np.random.default_rng(5)
    pos = np.sort(rng.choice(q.size, 200_000, replace=False)).astype(np.uint64)
    want = o.query_positions(q, qoff, pos)
    got = ((bits[(pos >> np.uint64(5)).astype(np.int64)] >> (pos & np.uint64(31)).astype(np.uint32)) & 1)
    assert np.array_equal(got.astype(np.uint8), want)
    reads = np.sort(rng.choice(qoff.size - 1, 3000, replace=False))
    sub = [q[int(qoff[r]):int(qoff[r + 1])] for r in reads]
    sseq, soff = synth.concat(sub)
    _, oh = o.query(sseq, soff)
    assert np.array_equal(hits[reads], oh)
    # sampled reads from the genome are mostly positive, random reads almost never
    n = (qoff.size - 1) // 2
    assert hits[:n].mean() > 20 and hits[n:].mean() < 0.05
    # every read: the oracle, holding the (identical) filter words, answers all
    # 20M reads in parallel processes; chunks of 262,144 reads start at
    # multiples of 32 bytes (150 * 262144 = 32 * 1228800), so answer words
    # compare word for word (the last word of a chunk up to its end)
    from oracle_pool import query_all

    words = o.words()
    checked = 0
    for r0, r1, a, b, obits, ohits in query_all(params, words, q, qoff, str(tmp_path)):
        assert a % 32 == 0
        assert np.array_equal(hits[r0:r1], ohits), (r0, r1)
        w0, nw = a // 32, (b - a + 31) // 32
        gw = bits[w0:w0 + nw].copy()
        if (b - a) % 32:
            gw[-1] &= np.uint32((1 << ((b - a) % 32)) - 1)
        assert np.array_equal(gw, obits), (r0, r1)
        checked += r1 - r0
    assert checked == qoff.size - 1
