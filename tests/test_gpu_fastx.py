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


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()


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


# ---------------------------------------------------------------------------
# tokenising on the device
# ---------------------------------------------------------------------------
def _device_parse(text: bytes, fastq: bool):
    import ctypes

    from paper_2606_24417_gb300.sbf import _check, load_library

    lib = load_library()
    n = len(text)
    d_text = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
    d_text[:n].copy_(torch.frombuffer(bytearray(text), dtype=torch.uint8))
    d_seq = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
    max_rec = n // 2 + 2
    d_off = torch.empty(max_rec + 1, dtype=torch.int64, device="cuda")
    need = ctypes.c_uint64()
    _check(lib.sbf_fastx_device_scratch(n, ctypes.byref(need)))
    scratch = torch.empty(int(need.value) + 16, dtype=torch.uint8, device="cuda")
    res = (ctypes.c_uint64 * 3)()
    _check(lib.sbf_fastx_parse_device(d_text.data_ptr(), n, 1 if fastq else 0, d_seq.data_ptr(),
                                      d_off.data_ptr(), max_rec, scratch.data_ptr(), int(need.value),
                                      res, torch.cuda.current_stream().cuda_stream))
    n_rec, kept, bad = int(res[0]), int(res[1]), int(res[2])
    if bad:
        return None
    off = d_off[:n_rec + 1].cpu().numpy()
    seq = bytes(d_seq[:kept].cpu().numpy())
    return [seq[int(off[i]):int(off[i + 1])] for i in range(n_rec)]


def _gen(rng, fastq, n_rec, crlf=False, spaces=False):
    import random as _r  # noqa: F401

    nl = b"\r\n" if crlf else b"\n"
    out, want = [], []
    for r in range(n_rec):
        L = rng.choice([0, 1, 31, 150, 3000, 70_000])
        seq = bytes(rng.choice(b"ACGTNacgt") for _ in range(L))
        want.append(seq)
        if fastq:
            out.append(b"@r%d x" % r + nl + seq + nl + b"+" + nl + b"I" * L + nl)
        else:
            w = rng.choice([60, 61, 1000, 10 ** 6])
            lines = [seq[j:j + w] for j in range(0, L, w)]
            if spaces and lines:
                lines[0] = b" " + lines[0] + b"\t"
            out.append(b">chr%d desc" % r + nl + nl.join(lines) + (nl if lines else b"") +
                       (nl if rng.random() < 0.2 else b""))
    return b"".join(out), want


@pytest.mark.parametrize("fastq,crlf,spaces", [(False, False, False), (False, True, True),
                                                (True, False, False), (True, True, False)])
def test_device_tokeniser_matches_definition(fastq, crlf, spaces):
    import random

    rng = random.Random(hash((fastq, crlf, spaces)) & 0xFFFF)
    text, want = _gen(rng, fastq, 60, crlf, spaces)
    got = _device_parse(text, fastq)
    assert got is not None
    assert got == [w for w in want]


def test_device_tokeniser_rejects_other_shapes():
    # FASTA line starting with '@', multi-line FASTQ, quality of another length
    assert _device_parse(b">a\nACGT\n@b\nAC\n+\nII\n", False) is None
    assert _device_parse(b"@a\nAC\nGT\n+\nIIII\n", True) is None
    assert _device_parse(b"@a\nACGT\n+\nIII\n", True) is None


@pytest.mark.parametrize("chunk", [1 << 16, 1 << 20])
def test_device_pipeline_matches_host_pipeline(files, chunk):
    from paper_2606_24417_gb300.fastx import DeviceFastx, insert_fastx, query_fastx
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    d, recs, q, qoff = files
    f1 = SuperBloomFilter(31, 16, 28, 4, 1 << 22)
    f2 = SuperBloomFilter(31, 16, 28, 4, 1 << 22)
    insert_fastx(f1, str(d / "g.fa"))
    ins = DeviceFastx(f2, chunk_bytes=chunk).insert(str(d / "g.fa"))
    assert np.array_equal(f1.words(), f2.words())
    if chunk < 300_000:  # the 300 kbp record does not fit: the buffers grew
        assert ins["grown_to"] >= 300_000
    h1, k1, _ = query_fastx(f1, str(d / "r.fq.gz"))
    h2, k2, st = DeviceFastx(f2, chunk_bytes=chunk).query(str(d / "r.fq.gz"))
    assert np.array_equal(h1, h2) and np.array_equal(k1, k2)
    assert st["host_fallback_chunks"] == 0 and st["chunks"] >= 1
    # a mixed file goes through the host parser for the chunks that need it
    mixed = d / "mixed.fa"
    mixed.write_bytes(b">x\nACGTACGTACGTACGTACGTACGTACGTACGTACG\n@y\nACGTAC\n+\nIIIIII\n")
    h3, _, st3 = DeviceFastx(f2, chunk_bytes=chunk).query(str(mixed))
    h4, _, _ = query_fastx(f2, str(mixed))
    assert np.array_equal(h3, h4) and st3["host_fallback_chunks"] == 1
