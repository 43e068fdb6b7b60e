"""The oracle at the sizes of the batched and served workloads (tests only).

The oracle itself is unchanged; these helpers only split its work the way
Alg. 1 and Alg. 2 allow, in processes started with `spawn` (the parent holds
a CUDA context):

* insert: a filter after inserting a set of k-mers is the OR of their bits,
  so a sequence is cut into slices that overlap by k - 1 bytes (every k-mer
  in exactly one slice), each slice goes into its own oracle filter, and the
  words are OR-ed;
* query: reads are independent, so any subset of reads can be answered by an
  oracle holding the filter's words.

Multi-GiB filters are OR-ed into one file-backed accumulator, block by block
under per-block locks, so memory holds one filter per worker plus the
accumulator; the worker count follows the host's available memory.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os

import numpy as np

_S = {}


def mem_available() -> int:
    """MemAvailable of /proc/meminfo in bytes (0 if unknown)."""
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def workers_for(bytes_per_worker: int, reserve: int) -> int:
    """Processes that fit next to `reserve` bytes of other use (0 = none)."""
    cpus = os.cpu_count() or 1
    free = mem_available() - reserve
    return max(0, min(cpus, free // max(1, bytes_per_worker)))


def slices(n: int, k: int, parts: int):
    """k-mer start ranges [a, b) covering the n - k + 1 starts of n bytes."""
    starts = max(0, n - k + 1)
    cuts = np.linspace(0, starts, parts + 1).astype(np.int64)
    return [(int(cuts[i]), int(cuts[i + 1])) for i in range(parts) if cuts[i + 1] > cuts[i]]


# ---------------------------------------------------------------------------
# many small filters (the batched workload)
# ---------------------------------------------------------------------------
def _init_many(params, gseq_path, words_dir):
    _S["params"] = params
    _S["gseq"] = np.load(gseq_path, mmap_mode="r")
    _S["words_dir"] = words_dir


def _oracle(bits):
    from oracle import OracleSBF

    k, m, s, H, B, canonical = _S["params"]
    return OracleSBF(k, m, s, H, bits, shard_bits=B, canonical=canonical)


def _insert_piece(task):
    f, bits, g0, a, b = task
    k = _S["params"][0]
    piece = np.ascontiguousarray(_S["gseq"][g0 + a:g0 + b + k - 1])
    o = _oracle(bits)
    o.insert(piece, np.array([0, piece.size], dtype=np.uint64))
    return f, o.words()


def _query_reads(task):
    f, bits, seq, off = task
    o = _oracle(bits)
    o.set_words(np.load(os.path.join(_S["words_dir"], f"f{f}.npy"), mmap_mode="r"))
    ob, oh = o.query(seq, off)
    return f, ob, oh


class ManyFilters:
    """Oracle inserts and queries for many independent filters (one genome
    each, concatenated in `gseq` with offsets `goff`)."""

    def __init__(self, params, gseq, tmpdir, workers=None):
        self.params = params
        self.tmpdir = str(tmpdir)
        self.words_dir = os.path.join(self.tmpdir, "words")
        os.makedirs(self.words_dir, exist_ok=True)
        gp = os.path.join(self.tmpdir, "gseq.npy")
        np.save(gp, np.asarray(gseq, dtype=np.uint8))
        self.workers = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_init_many,
                                                 initargs=(params, gp, self.words_dir))

    def close(self):
        self.pool.close()
        self.pool.join()

    def insert_all(self, bits, goff, piece_bases=8_000_000):
        """Words of every filter f after inserting genome f (one read)."""
        k = self.params[0]
        tasks = []
        for f, nb in enumerate(bits):
            n = int(goff[f + 1] - goff[f])
            parts = max(1, -(-n // piece_bases))
            for a, b in slices(n, k, parts):
                tasks.append((f, int(nb), int(goff[f]), a, b))
        # longest pieces first keeps the tail short
        tasks.sort(key=lambda t: t[4] - t[3], reverse=True)
        words = {}
        for f, w in self.pool.imap_unordered(_insert_piece, tasks):
            if f in words:
                np.bitwise_or(words[f], w, out=words[f])
            else:
                words[f] = w
        return words

    def save_words(self, f, w):
        np.save(os.path.join(self.words_dir, f"f{f}.npy"), w)

    def query(self, tasks):
        """tasks: (f, bits, seq, off) -> yields (f, answer words, hits)."""
        yield from self.pool.imap_unordered(_query_reads, tasks)


# ---------------------------------------------------------------------------
# one multi-GiB filter (the served workload)
# ---------------------------------------------------------------------------
_BLOCK_WORDS = 1 << 23   # 64 MiB blocks of the accumulator


def _init_big(params, bits, seq_path, acc_path, n_words, locks):
    _S["params"] = params
    _S["bits"] = bits
    _S["seq"] = np.load(seq_path, mmap_mode="r")
    _S["acc_path"], _S["n_words"], _S["locks"] = acc_path, n_words, locks


def _insert_into_acc(task):
    from oracle import OracleSBF

    a, b = task
    k, m, s, H, B, canonical = _S["params"]
    piece = np.ascontiguousarray(_S["seq"][a:b + k - 1])
    o = OracleSBF(k, m, s, H, _S["bits"], shard_bits=B, canonical=canonical)
    o.insert(piece, np.array([0, piece.size], dtype=np.uint64))
    del piece
    w = o.words_view()
    acc = np.memmap(_S["acc_path"], dtype=np.uint64, mode="r+", shape=(_S["n_words"],))
    locks = _S["locks"]
    nblk = len(locks)
    # start at a block of our own so that the workers rarely wait on a lock
    first = (a * 7919) % nblk
    for j in range(nblk):
        blk = (first + j) % nblk
        lo = blk * _BLOCK_WORDS
        hi = min(lo + _BLOCK_WORDS, _S["n_words"])
        with locks[blk]:
            np.bitwise_or(acc[lo:hi], w[lo:hi], out=acc[lo:hi])
    acc.flush()
    del acc, w, o
    return b - a


def _query_big(task):
    from oracle import OracleSBF

    tag, seq, off = task
    if "q" not in _S:
        k, m, s, H, B, canonical = _S["params"]
        o = OracleSBF(k, m, s, H, _S["bits"], shard_bits=B, canonical=canonical)
        o.set_words(np.memmap(_S["acc_path"], dtype=np.uint64, mode="r", shape=(_S["n_words"],)))
        _S["q"] = o
    ob, oh = _S["q"].query(seq, off)
    return tag, ob, oh


class BigFilter:
    """The oracle filter of one long sequence in a multi-GiB filter."""

    def __init__(self, params, bits, seq, tmpdir, workers):
        self.params, self.bits = params, bits
        self.tmpdir = str(tmpdir)
        self.seq_path = os.path.join(self.tmpdir, "seq.npy")
        np.save(self.seq_path, np.asarray(seq, dtype=np.uint8))
        self.n = int(seq.size)
        B = params[4]
        shards = -(-bits // B)
        self.n_words = shards * B // 64
        self.acc_path = os.path.join(self.tmpdir, "acc.u64")
        with open(self.acc_path, "wb") as fh:
            fh.truncate(self.n_words * 8)
        ctx = mp.get_context("spawn")
        nblk = -(-self.n_words // _BLOCK_WORDS)
        self.locks = [ctx.Lock() for _ in range(nblk)]
        self.workers = workers
        self.pool = ctx.Pool(workers, initializer=_init_big,
                             initargs=(params, bits, self.seq_path, self.acc_path, self.n_words,
                                       self.locks), maxtasksperchild=1)

    def close(self):
        self.pool.close()
        self.pool.join()

    def insert(self):
        """OR of all slices' filters into the accumulator."""
        k = self.params[0]
        done = sum(self.pool.imap_unordered(_insert_into_acc, slices(self.n, k, self.workers)))
        assert done == max(0, self.n - k + 1)

    def words(self) -> np.ndarray:
        return np.memmap(self.acc_path, dtype=np.uint64, mode="r", shape=(self.n_words,))

    def query(self, tasks, workers):
        """tasks: (tag, seq, off) answered by `workers` processes, each holding
        a copy of the accumulated words."""
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_init_big,
                      initargs=(self.params, self.bits, self.seq_path, self.acc_path,
                                self.n_words, self.locks)) as pool:
            yield from pool.imap_unordered(_query_big, tasks)


def compare_in_chunks(got: np.ndarray, want: np.ndarray, chunk_words: int = 1 << 25):
    """Compares two word arrays chunk by chunk with BLAKE2b digests; on a
    mismatching chunk, counts its differing words.  Returns a list of
    (chunk start, differing words, first differing index)."""
    assert got.size == want.size, (got.size, want.size)
    bad = []
    for lo in range(0, got.size, chunk_words):
        hi = min(lo + chunk_words, got.size)
        g, w = np.ascontiguousarray(got[lo:hi]), np.ascontiguousarray(want[lo:hi])
        if hashlib.blake2b(g.view(np.uint8)).digest() != hashlib.blake2b(w.view(np.uint8)).digest():
            diff = np.nonzero(g != w)[0]
            bad.append((lo, int(diff.size), int(lo + diff[0]) if diff.size else -1))
    return bad
