"""Command line: build a filter from FASTA/FASTQ files, query files against it.

  python -m paper_2606_24417_gb300 build genome.fa [more.fa ...] -o filter.sbf --bits 2^30
  python -m paper_2606_24417_gb300 query filter.sbf reads.fq.gz [--out hits.tsv] [--min-frac 0.5]
  python -m paper_2606_24417_gb300 info filter.sbf

Files are read as text (plain, gzip or BGZF) and tokenised on the GPU
(`fastx.DeviceFastx`); `--host-parse` uses the host parser instead.  `query`
writes one line per record: index, positive k-mers, k-mer positions and their
ratio; with --min-frac only records at or above that ratio are written.
"""
from __future__ import annotations

import argparse
import sys
import time

import numpy as np


def parse_bits(text: str) -> int:
    """'2^30', '1<<30', '128MiB' (bytes of filter) or a plain number of bits."""
    t = text.strip().lower().replace(" ", "")
    if "^" in t:
        base, exp = t.split("^", 1)
        return int(base) ** int(exp)
    if "<<" in t:
        a, b = t.split("<<", 1)
        return int(a) << int(b)
    for suffix, mult in (("gib", 8 << 30), ("mib", 8 << 20), ("kib", 8 << 10)):
        if t.endswith(suffix):
            return int(float(t[: -len(suffix)]) * mult)
    return int(t)


def _parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser(prog="python -m paper_2606_24417_gb300",
                                 description="GB300 Super Bloom filter for k-mers")
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("build", help="insert FASTA/FASTQ files into a new filter and save it")
    b.add_argument("inputs", nargs="+")
    b.add_argument("-o", "--out", required=True)
    b.add_argument("--k", type=int, default=31)
    b.add_argument("--m", type=int, default=16)
    b.add_argument("--s", type=int, default=28)
    b.add_argument("--H", type=int, default=4)
    b.add_argument("--bits", type=parse_bits, default=1 << 30,
                   help="filter size: bits, 2^P, 1<<P or bytes with KiB/MiB/GiB")
    b.add_argument("--shard-bits", type=int, default=512, choices=(256, 512))
    b.add_argument("--forward-only", action="store_true", help="no canonical k-mers")
    b.add_argument("--layout", default="default", choices=("default", "paper"))
    b.add_argument("--alphabet", default="dna", choices=("dna", "protein", "dna_triplet"))
    b.add_argument("--host-parse", action="store_true")
    q = sub.add_parser("query", help="per-record positive k-mers of FASTA/FASTQ files")
    q.add_argument("filter")
    q.add_argument("inputs", nargs="+")
    q.add_argument("--out", default="-", help="TSV output ('-': standard output)")
    q.add_argument("--min-frac", type=float, default=None)
    q.add_argument("--host-parse", action="store_true")
    i = sub.add_parser("info", help="parameters and fill of a saved filter")
    i.add_argument("filter")
    return ap


class _Files:
    """Inserts or queries files through one device pipeline (its pinned and
    device buffers are allocated once), or through the host parser."""

    def __init__(self, f, host_parse: bool):
        from .fastx import DeviceFastx

        self.f = f
        self.dev = None if host_parse or f.alphabet == 2 else DeviceFastx(f)

    def insert(self, path):
        from .fastx import insert_fastx

        return insert_fastx(self.f, path) if self.dev is None else self.dev.insert(path)

    def query(self, path):
        from .fastx import query_fastx

        return query_fastx(self.f, path) if self.dev is None else self.dev.query(path)


def main(argv=None) -> int:
    args = _parser().parse_args(argv)
    from .sbf import LAYOUT_DEFAULT, LAYOUT_PAPER, SuperBloomFilter

    if args.cmd == "build":
        f = SuperBloomFilter(args.k, args.m, args.s, args.H, args.bits, shard_bits=args.shard_bits,
                             canonical=not args.forward_only and args.alphabet == "dna",
                             layout=LAYOUT_PAPER if args.layout == "paper" else LAYOUT_DEFAULT,
                             alphabet=args.alphabet)
        t = time.perf_counter()
        files = _Files(f, args.host_parse)
        for path in args.inputs:
            files.insert(path)
        f.save(args.out)
        print(f"{args.out}: {len(args.inputs)} file(s) inserted in {time.perf_counter() - t:.2f} s, "
              f"{f.n_shards} shards of {f.shard_bits} bits", file=sys.stderr)
        return 0
    f = SuperBloomFilter.load(args.filter)
    if args.cmd == "info":
        w = f.words()
        fill = float(np.bitwise_count(w).sum()) / (w.size * 64) if hasattr(np, "bitwise_count") else None
        print(f"k={f.k} m={f.m} s={f.s} H={f.H} shard_bits={f.shard_bits} shards={f.n_shards} "
              f"canonical={int(f.canonical)} layout={f.layout} alphabet={f.alphabet} "
              f"fill={fill if fill is None else round(fill, 6)}")
        return 0
    out = sys.stdout if args.out == "-" else open(args.out, "w")
    try:
        out.write("file\trecord\tpositive_kmers\tkmers\tfraction\n")
        files = _Files(f, args.host_parse)
        for path in args.inputs:
            hits, kmers, _ = files.query(path)
            frac = np.divide(hits, kmers, out=np.zeros(hits.size, dtype=np.float64), where=kmers > 0)
            keep = np.arange(hits.size) if args.min_frac is None else np.flatnonzero(frac >= args.min_frac)
            for r in keep.tolist():
                out.write(f"{path}\t{r}\t{int(hits[r])}\t{int(kmers[r])}\t{frac[r]:.4f}\n")
    finally:
        if out is not sys.stdout:
            out.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
