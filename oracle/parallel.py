"""The oracle on all host cores: many single-threaded oracles, one per process.

TEST INFRASTRUCTURE ONLY (the CPU baseline and tests).  The oracle itself is
unchanged; this only splits the work the way the definition allows:

* insert: the filter after inserting a set of k-mers is the OR of their bits
  (Alg. 1), so each process inserts a slice of the sequence into its own
  filter and the parent ORs the words.  Slice i covers k-mer starts
  [a_i, b_i) and holds bytes [a_i, b_i + k - 1), so every k-mer is inserted
  by exactly one process;
* query: reads are independent (Alg. 2), so each process loads the filter
  words and answers a chunk of reads.

Processes are started with `spawn` (the parent may hold a CUDA context) and
read their inputs from memory-mapped .npy files.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_W = {}


def _init(params):
    from oracle import OracleSBF

    _W["params"] = params
    _W["make"] = lambda: OracleSBF(params["k"], params["m"], params["s"], params["H"], params["bits"],
                                   shard_bits=params["shard_bits"], canonical=params["canonical"])


def _insert_slice(task):
    path, a, b, out = task
    k = _W["params"]["k"]
    seq = np.load(path, mmap_mode="r")
    end = min(seq.size, b + k - 1)
    piece = np.ascontiguousarray(seq[a:end])
    f = _W["make"]()
    f.insert(piece, np.array([0, piece.size], dtype=np.uint64))
    np.save(out, f.words())
    return out


def _query_chunk(task):
    words_path, seq_path, off_path, r0, r1 = task
    if _W.get("words_path") != words_path:
        f = _W["make"]()
        f.set_words(np.load(words_path, mmap_mode="r"))
        _W["q"], _W["words_path"] = f, words_path
    off = np.asarray(np.load(off_path, mmap_mode="r")[r0:r1 + 1], dtype=np.uint64)
    a, b = int(off[0]), int(off[-1])
    seq = np.ascontiguousarray(np.load(seq_path, mmap_mode="r")[a:b])
    _, hits = _W["q"].query(seq, off - np.uint64(a))
    return int(hits.sum())


class OraclePool:
    """A pool of oracle processes for one parameter set."""

    def __init__(self, k, m, s, H, bits, shard_bits=512, canonical=True, workers=None):
        self.params = dict(k=k, m=m, s=s, H=H, bits=bits, shard_bits=shard_bits,
                           canonical=canonical)
        self.workers = workers or os.cpu_count() or 1
        self._pool = mp.get_context("spawn").Pool(self.workers, initializer=_init,
                                                  initargs=(self.params,))
        self._pool.map(len, [()] * self.workers)  # processes up before any timing

    def close(self):
        self._pool.close()
        self._pool.join()

    def insert(self, seq_path: str, n: int, tmpdir: str, tag: str = "w") -> np.ndarray:
        """Filter words after inserting the k-mers of seq[0:n) (one read)."""
        k = self.params["k"]
        starts = max(0, n - k + 1)
        cuts = np.linspace(0, starts, self.workers + 1).astype(np.int64)
        tasks = [(seq_path, int(cuts[i]), int(cuts[i + 1]), os.path.join(tmpdir, f"{tag}{i}.npy"))
                 for i in range(self.workers) if cuts[i + 1] > cuts[i]]
        words = None
        for out in self._pool.imap_unordered(_insert_slice, tasks):
            w = np.load(out)
            words = w if words is None else np.bitwise_or(words, w, out=words)
            os.remove(out)
        return words

    def query_hits(self, words_path: str, seq_path: str, off_path: str, n_reads: int,
                   chunk_reads: int = 65_536) -> int:
        """Positive k-mers of reads [0, n_reads)."""
        tasks = [(words_path, seq_path, off_path, r, min(r + chunk_reads, n_reads))
                 for r in range(0, n_reads, chunk_reads)]
        return sum(self._pool.imap_unordered(_query_chunk, tasks))
