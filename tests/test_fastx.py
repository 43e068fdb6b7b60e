"""FASTA / FASTQ input (host logic, no GPU): libsbf's incremental parser
against a whole-text reference parser written here, on generated files with
multi-line records, CRLF, blank lines, empty records, qualities starting with
'@', mixed formats and gzip (one or many members), fed in chunks of every
size and with output buffers small enough to split records."""
import gzip
import random

import numpy as np
import pytest

from paper_2606_24417_gb300 import fastx


def reference_records(text: bytes):
    """Sequences of the records of a FASTA/FASTQ text (whole-text reading)."""
    lines = text.replace(b"\r", b"").split(b"\n")
    out, i = [], 0
    while i < len(lines):
        ln = lines[i]
        if ln.startswith(b">"):
            i += 1
            seq = []
            while i < len(lines) and not lines[i].startswith((b">", b"@")):
                seq.append(lines[i])
                i += 1
            out.append(b"".join(seq).replace(b" ", b"").replace(b"\t", b""))
        elif ln.startswith(b"@"):
            i += 1
            seq = []
            while i < len(lines) and not lines[i].startswith(b"+"):
                seq.append(lines[i])
                i += 1
            s = b"".join(seq).replace(b" ", b"").replace(b"\t", b"")
            i += 1  # the '+' line
            need = len(s)
            while need > 0 and i < len(lines):
                need -= len(lines[i])
                i += 1
            out.append(s)
        else:
            i += 1
    return out


def make_text(rng: random.Random, n_records: int) -> bytes:
    parts = [b"garbage before the first record\n\n"] if rng.random() < 0.5 else []
    for r in range(n_records):
        L = rng.choice([0, 1, 5, 30, 31, 32, 100, 1000, 5000])
        seq = bytes(rng.choice(b"ACGTacgtN") for _ in range(L))
        nl = b"\r\n" if rng.random() < 0.3 else b"\n"
        if rng.random() < 0.5:
            w = rng.choice([7, 60, 80, 10 ** 6])
            body = nl.join(seq[j:j + w] for j in range(0, len(seq), w)) if seq else b""
            parts.append(b">rec%d some description" % r + nl + body + nl)
            if rng.random() < 0.2:
                parts.append(nl)  # blank line
        else:
            qual = bytes(rng.choice(b"@+!#I5") for _ in range(L))
            if rng.random() < 0.3 and L > 10:  # multi-line FASTQ
                body = seq[:L // 2] + nl + seq[L // 2:]
                qbody = qual[:L // 3] + nl + qual[L // 3:]
            else:
                body, qbody = seq, qual
            parts.append(b"@read%d" % r + nl + body + nl + b"+" + nl + qbody + nl)
    text = b"".join(parts)
    if rng.random() < 0.3 and text.endswith(b"\n"):
        text = text[:-1]  # no final newline
    return text


def parse_native(text: bytes, k: int, chunk: int, seq_cap: int, pieces_cap: int):
    """Drive the parser directly: returns (pieces, rec ids) in order."""
    import ctypes

    from paper_2606_24417_gb300.sbf import _check, load_library

    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.sbf_fastx_create(k, ctypes.byref(h)))
    seq = np.empty(seq_cap, dtype=np.uint8)
    off = np.empty(pieces_cap + 1, dtype=np.uint64)
    rec = np.empty(pieces_cap, dtype=np.uint64)
    n, L, used = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    pieces, recs = [], []
    data = np.frombuffer(text, dtype=np.uint8)
    pos = 0
    fed = 0
    try:
        while True:
            fed = min(len(text), max(fed, pos) + chunk) if fed < len(text) else fed
            final = 1 if fed == len(text) else 0
            view = data[pos:fed]
            _check(lib.sbf_fastx_parse(h, view.ctypes.data if view.size else None, view.size,
                                       final, seq.ctypes.data, seq_cap, off.ctypes.data,
                                       rec.ctypes.data, pieces_cap, ctypes.byref(n),
                                       ctypes.byref(L), ctypes.byref(used)))
            for i in range(int(n.value)):
                pieces.append(bytes(seq[int(off[i]):int(off[i + 1])]))
                recs.append(int(rec[i]))
            assert int(off[int(n.value)]) == int(L.value)
            pos += int(used.value)
            if final and pos == len(text):
                return pieces, recs
    finally:
        lib.sbf_fastx_destroy(h)


def reassemble(pieces, recs, k):
    """Records from pieces: each continuing piece starts with the record's
    last min(k-1, length so far) bases, which are dropped."""
    out = {}
    for p, r in zip(pieces, recs):
        if r not in out:
            out[r] = p
        else:
            carried = min(k - 1, len(out[r]))
            assert p[:carried] == out[r][len(out[r]) - carried:]
            out[r] += p[carried:]
    return [out[r] for r in sorted(out)]


def kmer_windows(pieces, recs, k):
    win = {}
    for p, r in zip(pieces, recs):
        win.setdefault(r, []).extend(p[i:i + k] for i in range(len(p) - k + 1))
    return win


@pytest.fixture(scope="module")
def lib():
    from paper_2606_24417_gb300 import build_lib
    from paper_2606_24417_gb300.sbf import load_library

    build_lib.build()
    return load_library()


@pytest.mark.parametrize("seed", range(12))
def test_parser_matches_reference(lib, seed):
    rng = random.Random(seed)
    k = rng.choice([5, 21, 31, 32])
    text = make_text(rng, rng.randint(1, 40))
    want = reference_records(text)
    for chunk, seq_cap, pieces_cap in [(len(text) + 1, 1 << 20, 1 << 16),
                                       (rng.randint(1, 50), 2 * (k - 1) + 64, 3),
                                       (rng.randint(100, 5000), 2 * (k - 1) + 64 + rng.randint(0, 500),
                                        rng.randint(1, 8))]:
        pieces, recs = parse_native(text, k, chunk, seq_cap, pieces_cap)
        assert recs == sorted(recs)
        assert len(set(recs)) == len(want)
        assert reassemble(pieces, recs, k) == want
        # every k-mer of every record is in exactly one piece
        win = kmer_windows(pieces, recs, k)
        for r, s in enumerate(want):
            assert win.get(r, []) == [s[i:i + k] for i in range(len(s) - k + 1)]


def test_parser_argument_checks(lib):
    import ctypes

    h = ctypes.c_void_p()
    assert lib.sbf_fastx_create(0, ctypes.byref(h)) == -1
    assert lib.sbf_fastx_create(33, ctypes.byref(h)) == -1
    assert lib.sbf_fastx_create(31, ctypes.byref(h)) == 0
    buf = np.empty(64, dtype=np.uint8)
    off = np.empty(2, dtype=np.uint64)
    n = ctypes.c_uint64()
    # seq_cap below 2(k-1) + 64 is refused
    assert lib.sbf_fastx_parse(h, None, 0, 1, buf.ctypes.data, 64, off.ctypes.data,
                               off.ctypes.data, 1, ctypes.byref(n), ctypes.byref(n),
                               ctypes.byref(n)) == -1
    lib.sbf_fastx_destroy(h)


@pytest.mark.parametrize("members", [1, 3])
def test_gzip_text_chunks(members):
    rng = random.Random(7)
    text = make_text(rng, 30)
    cut = [0] + sorted(rng.sample(range(1, len(text)), members - 1)) + [len(text)]
    gz = b"".join(gzip.compress(text[a:b]) for a, b in zip(cut, cut[1:]))
    assert b"".join(fastx.text_chunks(gz, chunk_bytes=100)) == text
    assert b"".join(fastx.text_chunks(text, chunk_bytes=100)) == text


def test_reader_pipeline_on_cpu(lib, tmp_path):
    rng = random.Random(11)
    text = make_text(rng, 60)
    p = tmp_path / "x.fq.gz"
    p.write_bytes(gzip.compress(text))
    k = 31
    rd = fastx.FastxReader(str(p), k, batch_bytes=2 * (k - 1) + 64 + 300, max_pieces=4,
                           chunk_bytes=333, pinned=False)
    pieces, recs = [], []
    for seq, off, rec in rd:
        for i in range(rec.size):
            pieces.append(bytes(seq[int(off[i]):int(off[i + 1])]))
            recs.append(int(rec[i]))
    want = reference_records(text)
    assert rd.records == len(want)
    assert reassemble(pieces, recs, k) == want


def test_bgzf_parallel_inflate(lib, tmp_path):
    """BGZF members are found from their size fields and inflated in
    parallel; the writer's output is valid gzip (Python's reader agrees)."""
    rng = random.Random(21)
    text = make_text(rng, 300)
    z = fastx.write_bgzf(text, block=4000)
    assert gzip.decompress(z) == text                  # independent reader
    blocks = fastx.bgzf_blocks(z)
    assert blocks is not None and len(blocks) == (len(text) + 3999) // 4000 + 1
    assert b"".join(fastx.text_chunks(z)) == text
    p = tmp_path / "x.fq.gz"
    p.write_bytes(z)
    assert b"".join(fastx.text_chunks(str(p))) == text
    assert fastx.bgzf_blocks(gzip.compress(text)) is None  # plain gzip: serial path
    # records through the reader equal the whole-text reading
    rd = fastx.FastxReader(str(p), 31, batch_bytes=1 << 16, max_pieces=64, pinned=False)
    pieces, recs = [], []
    for seq, off, rec in rd:
        for i in range(rec.size):
            pieces.append(bytes(seq[int(off[i]):int(off[i + 1])]))
            recs.append(int(rec[i]))
    assert reassemble(pieces, recs, 31) == reference_records(text)
