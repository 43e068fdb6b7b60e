"""The command line (python -m paper_2606_24417_gb300): size parsing and
argument checks on CPU; a build / query / info round trip on the GPU against
the oracle."""
import gzip

import numpy as np
import pytest

from paper_2606_24417_gb300.__main__ import _parser, parse_bits


def test_parse_bits():
    assert parse_bits("2^30") == 1 << 30
    assert parse_bits("1<<24") == 1 << 24
    assert parse_bits("128MiB") == 1 << 30       # bytes of filter
    assert parse_bits("1 GiB") == 1 << 33
    assert parse_bits("4096") == 4096


def test_arguments():
    a = _parser().parse_args(["build", "g.fa", "-o", "f.sbf", "--bits", "2^20", "--layout", "paper",
                              "--shard-bits", "256"])
    assert a.cmd == "build" and a.bits == 1 << 20 and a.layout == "paper" and a.shard_bits == 256
    with pytest.raises(SystemExit):
        _parser().parse_args(["build", "g.fa"])          # no output file
    with pytest.raises(SystemExit):
        _parser().parse_args(["query", "f.sbf"])         # no input


@pytest.mark.gpu
def test_build_query_info_round_trip(tmp_path, capsys):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import OracleSBF
    from paper_2606_24417_gb300 import build_lib, synth
    from paper_2606_24417_gb300.__main__ import main

    build_lib.build()
    g = synth.bacterial_genome(200_000, seed=51)
    (tmp_path / "g.fa").write_bytes(b">g\n" + b"\n".join(bytes(g[i:i + 60]) for i in range(0, g.size, 60)) + b"\n")
    q, qoff = synth.mixed_query_reads(g, 300, 300, 150, 0.01, seed=52)
    fq = b"".join(b"@r\n%s\n+\n%s\n" % (bytes(q[int(qoff[r]):int(qoff[r + 1])]), b"I" * 150)
                  for r in range(qoff.size - 1))
    (tmp_path / "r.fq.gz").write_bytes(gzip.compress(fq))
    assert main(["build", str(tmp_path / "g.fa"), "-o", str(tmp_path / "f.sbf"), "--bits", "2^22"]) == 0
    assert main(["query", str(tmp_path / "f.sbf"), str(tmp_path / "r.fq.gz"),
                 "--out", str(tmp_path / "hits.tsv")]) == 0
    rows = [ln.split("\t") for ln in (tmp_path / "hits.tsv").read_text().splitlines()[1:]]
    o = OracleSBF(31, 16, 28, 4, 1 << 22)
    o.insert(g, np.array([0, g.size], dtype=np.uint64))
    _, oh = o.query(q, qoff)
    assert [int(r[2]) for r in rows] == oh.tolist()
    assert all(int(r[3]) == 120 for r in rows)
    assert main(["query", str(tmp_path / "f.sbf"), str(tmp_path / "r.fq.gz"), "--host-parse",
                 "--min-frac", "0.5", "--out", str(tmp_path / "h2.tsv")]) == 0
    rows2 = [ln.split("\t") for ln in (tmp_path / "h2.tsv").read_text().splitlines()[1:]]
    assert [int(r[1]) for r in rows2] == [i for i, h in enumerate(oh.tolist()) if h / 120 >= 0.5]
    assert main(["info", str(tmp_path / "f.sbf")]) == 0
    assert "k=31 m=16 s=28 H=4" in capsys.readouterr().out
