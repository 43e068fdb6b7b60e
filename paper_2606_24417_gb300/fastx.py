"""FASTA / FASTQ input for the host entry points (Sec. IV-A streamed FASTX
input with transparent gzip; Sec. V-F host-resident sequences).

``FastxReader`` turns a file (plain or gzip, including multi-member gzip such
as bgzip) into read batches for ``SuperBloomFilter.insert_host`` /
``query_host``: the text is decompressed and parsed by libsbf's incremental
parser (``sbf_fastx_parse``) on a producer thread while the caller's previous
batch is on the GPU; batches live in two (pinned, when CUDA is available)
buffer sets used in turn.  A record longer than a batch is split and its next
piece repeats its last k-1 bases, so every k-mer is in exactly one piece;
``rec`` gives each piece's record index.
"""
from __future__ import annotations

import ctypes
import queue
import threading
import time
import zlib

import numpy as np

from .sbf import _check, _host_ptr, load_library

_GZIP_MAGIC = b"\x1f\x8b"


def _host_buffer(n: int, dtype, pinned: bool) -> np.ndarray:
    if pinned:
        import torch

        t = torch.empty(n * np.dtype(dtype).itemsize, dtype=torch.uint8).pin_memory()
        return t.numpy().view(dtype)
    return np.empty(n, dtype=dtype)


def text_chunks(src, chunk_bytes: int = 16 << 20):
    """Decompressed text of a path, bytes or file object, in chunks."""
    if isinstance(src, (bytes, bytearray, memoryview)):
        data = bytes(src)
        fh = None
    else:
        fh = open(src, "rb") if isinstance(src, str) else src
        data = None
    try:
        read = (lambda n: fh.read(n)) if fh is not None else None
        if data is not None:
            pos = [0]

            def read(n):  # noqa: F811
                b = data[pos[0]:pos[0] + n]
                pos[0] += len(b)
                return b
        first = read(chunk_bytes)
        if first[:2] != _GZIP_MAGIC:
            while first:
                yield first
                first = read(chunk_bytes)
            return
        d = zlib.decompressobj(16 + zlib.MAX_WBITS)
        buf = first
        while True:
            if not buf:
                buf = read(chunk_bytes)
                if not buf:
                    tail = d.flush()
                    if tail:
                        yield tail
                    return
            out = d.decompress(buf)
            if out:
                yield out
            buf = b""
            if d.eof:  # next gzip member (bgzip writes many)
                rest = d.unused_data
                tail = d.flush()
                if tail:
                    yield tail
                d = zlib.decompressobj(16 + zlib.MAX_WBITS)
                buf = rest
    finally:
        if fh is not None and isinstance(src, str):
            fh.close()


class FastxReader:
    """Iterates (seq, off, rec) batches of a FASTA/FASTQ source.

    seq: uint8 sequence bytes; off: uint64 offsets (pieces + 1); rec: uint64
    record index per piece.  The arrays are views into reused buffers: a batch
    stays valid until the iterator is asked for the next one."""

    def __init__(self, src, k: int, batch_bytes: int = 64 << 20, max_pieces: int = 1 << 20,
                 chunk_bytes: int = 16 << 20, pinned: bool | None = None, symbol_bytes: int = 1):
        self._lib = load_library()
        if symbol_bytes != 1:
            raise ValueError("FASTX batches split records at any byte; multi-byte symbols "
                             "(DNA triplets) need whole records: use the host entry points")
        if pinned is None:
            try:
                import torch

                pinned = torch.cuda.is_available()
            except ImportError:
                pinned = False
        self.src, self.k, self.pinned = src, k, pinned
        self.batch_bytes, self.max_pieces, self.chunk_bytes = batch_bytes, max_pieces, chunk_bytes
        self._bufs = [(_host_buffer(batch_bytes, np.uint8, pinned),
                       _host_buffer(max_pieces + 1, np.uint64, pinned),
                       _host_buffer(max_pieces, np.uint64, pinned)) for _ in range(2)]
        self.records = 0
        self.text_bytes = 0
        self.parse_seconds = 0.0

    def _produce(self, filled: queue.Queue, free: queue.Queue, stop: threading.Event):
        lib = self._lib
        h = ctypes.c_void_p()
        _check(lib.sbf_fastx_create(self.k, ctypes.byref(h)))
        n_out, len_out, used = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        min_room = 2 * (self.k - 1) + 64
        try:
            chunks = text_chunks(self.src, self.chunk_bytes)
            text = np.empty(0, dtype=np.uint8)
            tpos, eof, done = 0, False, False
            b = free.get()
            seq, off, rec = self._bufs[b]
            cur_len = cur_n = 0
            while not done:
                if stop.is_set():
                    return
                if tpos == text.size and not eof:
                    nxt = next(chunks, None)
                    if nxt is None:
                        eof = True
                        text = np.empty(0, dtype=np.uint8)
                    else:
                        text = np.frombuffer(nxt, dtype=np.uint8)
                        self.text_bytes += text.size
                    tpos = 0
                    continue
                if self.batch_bytes - cur_len < min_room or self.max_pieces - cur_n < 1:
                    filled.put((b, cur_len, cur_n))
                    b = free.get()
                    if b is None:
                        return
                    seq, off, rec = self._bufs[b]
                    cur_len = cur_n = 0
                    continue
                t0 = time.perf_counter()
                _check(lib.sbf_fastx_parse(
                    h, _host_ptr(text[tpos:]) if tpos < text.size else None, text.size - tpos,
                    1 if eof else 0, seq.ctypes.data + cur_len, self.batch_bytes - cur_len,
                    off.ctypes.data + 8 * cur_n, rec.ctypes.data + 8 * cur_n,
                    self.max_pieces - cur_n, ctypes.byref(n_out), ctypes.byref(len_out),
                    ctypes.byref(used)))
                self.parse_seconds += time.perf_counter() - t0
                n, L = int(n_out.value), int(len_out.value)
                if cur_len:
                    off[cur_n:cur_n + n + 1] += np.uint64(cur_len)
                if n:
                    self.records = max(self.records, int(rec[cur_n + n - 1]) + 1)
                cur_n += n
                cur_len += L
                tpos += int(used.value)
                if eof and tpos == text.size:
                    done = True
            filled.put((b, cur_len, cur_n))
        except BaseException as exc:  # surfaced to the consumer
            filled.put(exc)
            return
        finally:
            lib.sbf_fastx_destroy(h)
        filled.put(None)

    def __iter__(self):
        filled: queue.Queue = queue.Queue()
        free: queue.Queue = queue.Queue()
        for i in range(len(self._bufs)):
            free.put(i)
        stop = threading.Event()
        th = threading.Thread(target=self._produce, args=(filled, free, stop), daemon=True)
        th.start()
        held = None
        try:
            while True:
                item = filled.get()
                if held is not None:
                    free.put(held)  # the batch before this one is released
                    held = None
                if item is None:
                    break
                if isinstance(item, BaseException):
                    raise item
                b, L, n = item
                if n == 0:
                    free.put(b)
                    continue
                held = b
                seq, off, rec = self._bufs[b]
                yield seq[:L], off[:n + 1], rec[:n]
        finally:
            stop.set()
            free.put(None)
            th.join(timeout=10)


def insert_fastx(filt, src, **reader_kw) -> dict:
    """Insert every record of a FASTA/FASTQ source (Alg. 1 over each record)."""
    rd = FastxReader(src, filt.k, symbol_bytes=3 if filt.alphabet == 2 else 1, **reader_kw)
    t0 = time.perf_counter()
    bases = batches = 0
    for seq, off, _ in rd:
        filt.insert_host(seq, off)
        bases += seq.size
        batches += 1
    return {"records": rd.records, "bases": bases, "batches": batches,
            "text_bytes": rd.text_bytes, "seconds": time.perf_counter() - t0,
            "parse_seconds": rd.parse_seconds}


def query_fastx(filt, src, **reader_kw):
    """Per-record positive k-mer counts and k-mer positions of a FASTA/FASTQ
    source (Alg. 2 over each record): (hits uint64[records], kmers
    uint64[records], info dict)."""
    rd = FastxReader(src, filt.k, symbol_bytes=3 if filt.alphabet == 2 else 1, **reader_kw)
    hits_rec = np.zeros(1024, dtype=np.uint64)
    kmers_rec = np.zeros(1024, dtype=np.uint64)
    hits_buf = _host_buffer(rd.max_pieces, np.uint32, rd.pinned)
    t0 = time.perf_counter()
    batches = 0
    for seq, off, rec in rd:
        n = rec.size
        _, h = filt.query_host(seq, off, hits=hits_buf[:n], want_bits=False)
        top = int(rec[-1]) + 1
        if top > hits_rec.size:
            grow = max(top, 2 * hits_rec.size)
            hits_rec = np.concatenate([hits_rec, np.zeros(grow - hits_rec.size, np.uint64)])
            kmers_rec = np.concatenate([kmers_rec, np.zeros(grow - kmers_rec.size, np.uint64)])
        lens = np.diff(off.astype(np.int64))
        np.add.at(hits_rec, rec.astype(np.int64), h.astype(np.uint64))
        np.add.at(kmers_rec, rec.astype(np.int64),
                  np.maximum(lens - (filt.k - 1), 0).astype(np.uint64))
        batches += 1
    n_rec = rd.records
    return hits_rec[:n_rec], kmers_rec[:n_rec], {
        "records": n_rec, "batches": batches, "text_bytes": rd.text_bytes,
        "seconds": time.perf_counter() - t0, "parse_seconds": rd.parse_seconds}
