"""Protein and DNA-triplet filters (Sec. IV-A alphabets) on the GPU through
the C ABI, bit for bit against the oracle: filter words, answer bits, hits
and run statistics on ragged reads; the host path; checkpoints; FASTA input
of proteins."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_off(off):
    return dev(np.asarray(off, dtype=np.uint64).astype(np.int64))


def ragged(source, n, seed, hi=2000, junk=b"*-X.1"):
    """Reads of lognormal lengths cut from `source`, with scattered junk bytes."""
    lens = synth.lognormal_lengths(n, 120, 1.0, 0, hi, seed)
    starts = synth.randint(seed, 2, n, 0, source.size - hi)
    seq = np.concatenate([source[s:s + L] for s, L in zip(starts, lens)] + [np.zeros(0, np.uint8)])
    u = synth.uniform01(seed, 3, 0, seq.size)
    jk = np.frombuffer(junk, dtype=np.uint8)
    bad = u < 0.001
    seq[bad] = jk[synth.randint(seed, 4, int(bad.sum()), 0, jk.size)]
    seq[(u > 0.5) & (u < 0.52)] |= 0x20  # lower case
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    return seq, off


CASES = [
    # k, m, s, H, bits, B, layout, alphabet
    (12, 6, 10, 4, 1 << 22, 512, 0, 1),
    (12, 7, 12, 1, 1 << 21, 512, 0, 1),
    (10, 4, 8, 8, 1 << 22, 256, 0, 1),
    (12, 6, 9, 16, 1 << 22, 512, 0, 1),
    (12, 6, 10, 4, 1 << 22, 256, 1, 1),
    (10, 5, 8, 4, 1 << 22, 512, 0, 2),
    (10, 6, 10, 2, 1 << 21, 512, 0, 2),
    (8, 4, 6, 4, 1 << 21, 256, 1, 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "_".join(map(str, c)))
def test_alphabet_bit_exact(case):
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    k, m, s, H, bits, B, layout, alphabet = case
    if alphabet == 1:
        src = synth.protein_sequence(2_000_000, 31)
        ins, ins_off = ragged(src, 3000, 32)
        q1, q1_off = ragged(src, 2000, 33)
        q2, q2_off = ragged(synth.protein_sequence(500_000, 34, dup_frac=0), 2000, 35)
    else:
        src = synth.bacterial_genome(2_000_000, seed=31)
        ins, ins_off = ragged(src, 3000, 32, junk=b"N")
        q1, q1_off = ragged(src, 2000, 33, junk=b"N")
        q2, q2_off = ragged(synth.uniform_dna(500_000, 34), 2000, 35, junk=b"N")
    q = np.concatenate([q1, q2])
    q_off = np.concatenate([q1_off, q2_off[1:] + q1_off[-1]])
    f = SuperBloomFilter(k, m, s, H, bits, shard_bits=B, canonical=False, layout=layout,
                         alphabet=alphabet)
    assert not f.fused and f.alphabet == alphabet
    o = OracleSBF(k, m, s, H, bits, shard_bits=B, canonical=False, layout=layout, alphabet=alphabet)
    f.insert(dev(ins), dev_off(ins_off))
    o.insert(ins, ins_off)
    assert np.array_equal(f.words(), o.words())
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    qb, qh = f.query(dev(q), dev_off(q_off), stats=stats)
    ob, oh = o.query(q, q_off)
    assert np.array_equal(qb.cpu().numpy().view(np.uint32), ob)
    assert np.array_equal(qh.cpu().numpy().view(np.uint32), oh)
    valid, runs = o.count_runs(q, q_off)
    assert stats.cpu().tolist() == [valid, runs, int(oh.sum())]
    assert int(oh[:2000].sum()) > 0
    # the host path gives the same answers
    hb, hh = f.query_host(q, q_off)
    assert np.array_equal(hb, ob) and np.array_equal(hh, oh)
    f2 = SuperBloomFilter(k, m, s, H, bits, shard_bits=B, canonical=False, layout=layout,
                          alphabet=alphabet)
    f2.insert_host(ins, ins_off)
    assert np.array_equal(f2.words(), o.words())


def test_alphabet_checkpoint_and_refusals(tmp_path):
    from paper_2606_24417_gb300.sbf import SbfError, SuperBloomFilter

    f = SuperBloomFilter(12, 6, 10, 4, 1 << 20, canonical=False, alphabet="protein")
    p = synth.protein_sequence(100_000, 5)
    f.insert(dev(p), dev_off(np.array([0, p.size], dtype=np.uint64)))
    f.save(str(tmp_path / "p.sbf"))
    g = type(f).load(str(tmp_path / "p.sbf"))
    assert g.alphabet == 1 and np.array_equal(g.words(), f.words())
    with pytest.raises(SbfError):
        SuperBloomFilter(12, 6, 10, 4, 1 << 20, canonical=True, alphabet="protein")
    with pytest.raises(SbfError):
        SuperBloomFilter(13, 6, 10, 4, 1 << 20, canonical=False, alphabet="protein")  # 65 bits
    with pytest.raises(SbfError):
        SuperBloomFilter(11, 6, 10, 4, 1 << 20, canonical=False, alphabet="dna_triplet")


def test_protein_fasta_input(tmp_path):
    from paper_2606_24417_gb300.fastx import insert_fastx, query_fastx
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    recs = [synth.protein_sequence(n, 40 + i) for i, n in enumerate((30_000, 5, 12_345))]
    text = b"".join(b">p%d\n" % i + b"\n".join(bytes(r[j:j + 60]) for j in range(0, r.size, 60)) + b"\n"
                    for i, r in enumerate(recs))
    (tmp_path / "p.fa").write_bytes(text)
    f = SuperBloomFilter(12, 6, 10, 4, 1 << 21, canonical=False, alphabet="protein")
    insert_fastx(f, str(tmp_path / "p.fa"), batch_bytes=4096, max_pieces=5)
    o = OracleSBF(12, 6, 10, 4, 1 << 21, canonical=False, alphabet="protein")
    seq = np.concatenate(recs)
    off = np.zeros(4, dtype=np.uint64)
    np.cumsum([r.size for r in recs], out=off[1:])
    o.insert(seq, off)
    assert np.array_equal(f.words(), o.words())
    hits, kmers, _ = query_fastx(f, str(tmp_path / "p.fa"), batch_bytes=4096, max_pieces=5)
    _, oh = o.query(seq, off)
    assert np.array_equal(hits, oh.astype(np.uint64))
    t = SuperBloomFilter(10, 5, 8, 4, 1 << 20, canonical=False, alphabet="dna_triplet")
    with pytest.raises(ValueError):
        insert_fastx(t, str(tmp_path / "p.fa"))


ROLLING_CASES = [
    # k, m, s, H, bits, B, canonical, layout, alphabet
    (12, 6, 10, 4, 1 << 24, 512, False, 0, 1),
    (10, 5, 8, 4, 1 << 23, 512, False, 0, 2),
    (31, 16, 28, 16, 1 << 24, 512, True, 0, 0),    # DNA outside the fused grid (H = 16)
    (25, 11, 21, 3, 1 << 24, 256, True, 0, 0),     # w = 15, H = 3
    (31, 16, 28, 12, 1 << 24, 256, False, 1, 0),   # the paper's layout, salted multiply
]


@pytest.mark.parametrize("case", ROLLING_CASES, ids=lambda c: "_".join(map(str, c)))
def test_rolling_kernels_equal_generic_and_oracle(case, monkeypatch):
    """Every filter outside the fused grid runs the rolling kernels; on a
    larger workload (whole genome inserted, 200,000 ragged reads, junk bytes)
    their words, answer bits, hits and run statistics equal the generic
    one-k-mer-per-thread kernels' and, on a sample, the oracle's."""
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    k, m, s, H, bits, B, canon, layout, alphabet = case
    if alphabet == 1:
        src = synth.protein_sequence(5_000_000, 41)
        q, q_off = ragged(src, 200_000, 43)
        junk = b"*-X.1"
    else:
        src = synth.bacterial_genome(5_000_000, seed=41)
        q, q_off = ragged(src, 200_000, 43, junk=b"N")
        junk = b"N"
    ins, ins_off = ragged(src, 20_000, 42, junk=junk)
    kw = dict(shard_bits=B, canonical=canon, layout=layout, alphabet=alphabet)
    fr = SuperBloomFilter(k, m, s, H, bits, **kw)
    monkeypatch.setenv("SBF_FORCE_GENERIC", "1")
    fg = SuperBloomFilter(k, m, s, H, bits, **kw)
    monkeypatch.delenv("SBF_FORCE_GENERIC")
    assert fr.kernel_variant == "rolling" and fg.kernel_variant == "generic"
    for f in (fr, fg):
        f.insert(dev(ins), dev_off(ins_off))
    assert np.array_equal(fr.words(), fg.words())
    out = []
    for f in (fr, fg):
        st = torch.zeros(3, dtype=torch.int64, device="cuda")
        b_, h_ = f.query(dev(q), dev_off(q_off), stats=st)
        out.append((b_.cpu().numpy(), h_.cpu().numpy(), st.cpu().tolist()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][2][2] > 0
    o = OracleSBF(k, m, s, H, bits, **kw)
    o.set_words(fr.words())
    n = 3000
    ob, oh = o.query(q[:int(q_off[n])], q_off[:n + 1])
    assert np.array_equal(out[0][1].view(np.uint32)[:n], oh)
    got = np.unpackbits(out[0][0].view(np.uint8), bitorder="little")[:int(q_off[n])]
    assert np.array_equal(got, np.unpackbits(ob.view(np.uint8), bitorder="little")[:int(q_off[n])])
