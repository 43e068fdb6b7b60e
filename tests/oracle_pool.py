"""The oracle's query run over many read chunks in parallel processes (tests
only).  Workers are started with `spawn` (the parent may hold a CUDA
context) and read the inputs from memory-mapped .npy files, so a full-size
check needs no copies through pipes.  Every worker loads the filter words
given to it into its own oracle, which answers exactly as one that inserted
the same k-mers (the words are the whole state)."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_STATE = {}


def _init(params, words_path, seq_path, off_path):
    from oracle import OracleSBF

    k, m, s, H, bits, B, canonical = params
    o = OracleSBF(k, m, s, H, bits, shard_bits=B, canonical=canonical)
    o.set_words(np.load(words_path, mmap_mode="r"))
    _STATE["o"] = o
    _STATE["seq"] = np.load(seq_path, mmap_mode="r")
    _STATE["off"] = np.load(off_path, mmap_mode="r")


def _run(task):
    r0, r1 = task
    off = np.asarray(_STATE["off"][r0:r1 + 1], dtype=np.uint64)
    a, b = int(off[0]), int(off[-1])
    seq = np.ascontiguousarray(_STATE["seq"][a:b])
    bits, hits = _STATE["o"].query(seq, off - np.uint64(a))
    return r0, r1, a, b, bits, hits


def query_all(params, words, seq, off, tmpdir, chunk_reads=262_144, workers=None):
    """Yields (r0, r1, a, b, bits, hits) for read chunks [r0, r1) covering all
    reads; chunk starts are multiples of `chunk_reads` (pick it so that the
    chunks' first bytes are multiples of 32 when the answer words are to be
    compared word for word)."""
    wp, sp, op = (os.path.join(tmpdir, n) for n in ("words.npy", "seq.npy", "off.npy"))
    np.save(wp, np.asarray(words, dtype=np.uint64))
    np.save(sp, np.asarray(seq, dtype=np.uint8))
    np.save(op, np.asarray(off, dtype=np.uint64))
    n_reads = off.size - 1
    tasks = [(r, min(r + chunk_reads, n_reads)) for r in range(0, n_reads, chunk_reads)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers or os.cpu_count(), initializer=_init, initargs=(params, wp, sp, op)) as pool:
        yield from pool.imap_unordered(_run, tasks)
