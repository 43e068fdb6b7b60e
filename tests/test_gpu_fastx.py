"""FASTA / FASTQ input end to end on the GPU: inserting a FASTA file and
querying a gzip FASTQ file through the streaming reader gives the oracle's
filter words and per-record hit counts, also when batches are small enough
to split records."""
import gzip

import numpy as np
import pytest

from oracle import OracleSBF
from paper_2606_24417_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def fasta_text(records, width=60):
    out = []
    for i, s in enumerate(records):
        out.append(b">chr%d synthetic\n" % i)
        out += [bytes(s[j:j + width]) + b"\n" for j in range(0, len(s), width)]
    return b"".join(out)


def fastq_text(seq, off):
    out = []
    for r in range(off.size - 1):
        s = bytes(seq[int(off[r]):int(off[r + 1])])
        out.append(b"@r%d\n%s\n+\n%s\n" % (r, s, b"I" * len(s)))
    return b"".join(out)


@pytest.fixture(scope="module")
def files(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    d = tmp_path_factory.mktemp("fastx")
    g1 = synth.bacterial_genome(300_000, seed=41)
    g2 = synth.uniform_dna(50_000, seed=42)
    g2[1000:1100] = ord("N")
    recs = [g1, g2, synth.uniform_dna(20, seed=43)]  # the last is shorter than k
    (d / "g.fa").write_bytes(fasta_text(recs))
    q, qoff = synth.mixed_query_reads(g1, 3000, 3000, 150, 0.01, seed=44)
    (d / "r.fq.gz").write_bytes(gzip.compress(fastq_text(q, qoff), compresslevel=1))
    return d, recs, q, qoff


@pytest.mark.parametrize("batch_bytes,max_pieces", [(64 << 20, 1 << 20), (4096, 7)])
def test_fasta_insert_fastq_query(files, batch_bytes, max_pieces):
    from paper_2606_24417_gb300.fastx import insert_fastx, query_fastx
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    d, recs, q, qoff = files
    f = SuperBloomFilter(31, 16, 28, 4, 1 << 22)
    info = insert_fastx(f, str(d / "g.fa"), batch_bytes=batch_bytes, max_pieces=max_pieces,
                        chunk_bytes=10_000)
    assert info["records"] == 3
    o = OracleSBF(31, 16, 28, 4, 1 << 22)
    seq = np.concatenate(recs)
    off = np.zeros(len(recs) + 1, dtype=np.uint64)
    np.cumsum([r.size for r in recs], out=off[1:])
    o.insert(seq, off)
    assert np.array_equal(f.words(), o.words())

    hits, kmers, qinfo = query_fastx(f, str(d / "r.fq.gz"), batch_bytes=batch_bytes,
                                     max_pieces=max_pieces, chunk_bytes=10_000)
    _, oh = o.query(q, qoff)
    assert qinfo["records"] == qoff.size - 1
    assert np.array_equal(hits, oh.astype(np.uint64))
    assert np.array_equal(kmers, np.full(qoff.size - 1, 150 - 30, dtype=np.uint64))
    # the FASTA records queried back: every k-mer of every record is positive
    hits_g, kmers_g, _ = query_fastx(f, str(d / "g.fa"), batch_bytes=batch_bytes,
                                     max_pieces=max_pieces)
    _, og = o.query(seq, off)
    assert np.array_equal(hits_g, og.astype(np.uint64))
    assert list(kmers_g) == [max(0, r.size - 30) for r in recs]
