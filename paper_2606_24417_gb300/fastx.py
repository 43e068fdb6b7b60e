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
import os
import queue
import threading
import time
import zlib
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .sbf import _check, _host_ptr, load_library

_GZIP_MAGIC = b"\x1f\x8b"


def _host_buffer(n: int, dtype, pinned: bool) -> np.ndarray:
    if pinned:
        import torch

        t = torch.empty(n * np.dtype(dtype).itemsize, dtype=torch.uint8).pin_memory()
        return t.numpy().view(dtype)
    return np.empty(n, dtype=dtype)


def bgzf_blocks(data) -> list | None:
    """Member boundaries [(start, end), ...] of a BGZF file (gzip members whose
    header carries the 'BC' extra field with the member size), or None if
    `data` (a bytes-like object) is not BGZF throughout."""
    mv = memoryview(data)
    n, at, out = len(mv), 0, []
    while at < n:
        if n - at < 18 or mv[at] != 0x1F or mv[at + 1] != 0x8B or mv[at + 2] != 8 or not (mv[at + 3] & 4):
            return None
        xlen = mv[at + 10] | (mv[at + 11] << 8)
        x, xe, bsize = at + 12, at + 12 + xlen, None
        while x + 4 <= xe:
            slen = mv[x + 2] | (mv[x + 3] << 8)
            if mv[x] == ord("B") and mv[x + 1] == ord("C") and slen == 2:
                bsize = (mv[x + 4] | (mv[x + 5] << 8)) + 1
            x += 4 + slen
        if bsize is None or at + bsize > n:
            return None
        out.append((at, at + bsize))
        at += bsize
    return out


def write_bgzf(data: bytes, level: int = 1, block: int = 65280) -> bytes:
    """BGZF encoding of `data`: gzip members of at most `block` input bytes,
    each header carrying the 'BC' extra field with the member size, and the
    empty end-of-file member (the SAM/BAM specification's layout)."""
    import struct

    def member(chunk: bytes, comp: bytes) -> bytes:
        bsize = 18 + len(comp) + 8
        hdr = (b"\x1f\x8b\x08\x04" + b"\0\0\0\0" + b"\0\xff" + struct.pack("<H", 6) + b"BC" +
               struct.pack("<HH", 2, bsize - 1))
        return hdr + comp + struct.pack("<II", zlib.crc32(chunk) & 0xFFFFFFFF, len(chunk) & 0xFFFFFFFF)

    out = []
    for i in range(0, len(data), block):
        chunk = bytes(data[i:i + block])
        c = zlib.compressobj(level, zlib.DEFLATED, -15)
        out.append(member(chunk, c.compress(chunk) + c.flush()))
    c = zlib.compressobj(level, zlib.DEFLATED, -15)
    out.append(member(b"", c.compress(b"") + c.flush()))
    return b"".join(out)


def _inflate_group(data, blocks):
    return b"".join(zlib.decompress(bytes(data[a:b]), 31) for a, b in blocks)


def text_chunks(src, chunk_bytes: int = 16 << 20):
    """Decompressed text of a path, bytes or file object, in chunks.  BGZF
    input is inflated by several threads at once (zlib releases the GIL),
    other gzip input member by member on one thread."""
    if isinstance(src, str):
        with open(src, "rb") as fh:
            head = fh.read(4)
        if head[:2] == _GZIP_MAGIC and len(head) == 4 and head[3] & 4:
            import mmap

            with open(src, "rb") as fh, mmap.mmap(fh.fileno(), 0, access=mmap.ACCESS_READ) as mm:
                blocks = bgzf_blocks(mm)
                if blocks:
                    yield from _bgzf_text(mm, blocks)
                    return
    elif isinstance(src, (bytes, bytearray, memoryview)) and bytes(src[:2]) == _GZIP_MAGIC:
        blocks = bgzf_blocks(src)
        if blocks:
            yield from _bgzf_text(src, blocks)
            return
    yield from _serial_text_chunks(src, chunk_bytes)


def _bgzf_text(data, blocks, group: int = 256, workers: int = 16):
    groups = [blocks[i:i + group] for i in range(0, len(blocks), group)]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        for piece in ex.map(lambda g: _inflate_group(data, g), groups):
            if piece:
                yield piece


def _serial_text_chunks(src, chunk_bytes: int = 16 << 20):
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


# ---------------------------------------------------------------------------
# parsing on the device: the host moves raw text, the GPU tokenises it
# ---------------------------------------------------------------------------
def _fastq_start_ok(win: bytes, q: int) -> bool:
    """True if a FASTQ record starts at win[q] and its four lines lie in win."""
    parts = win[q:].split(b"\n", 4)
    if len(parts) < 5:
        return False
    h, sq, plus, qual = parts[:4]
    return (h[:1] == b"@" and plus[:1] == b"+"
            and len(sq.rstrip(b"\r")) == len(qual.rstrip(b"\r")))


def _last_record_start(buf: np.ndarray, lo: int, hi: int, fastq: bool) -> int:
    """Position in (lo, hi) of the last record start of buf[lo:hi], or -1."""
    win_len = 1 << 20
    while True:
        a = max(lo, hi - win_len)
        win = buf[a:hi].tobytes()
        if fastq:
            j = len(win)
            while True:
                j = win.rfind(b"\n@", 0, j)
                if j < 0:
                    break
                if _fastq_start_ok(win, j + 1):
                    if a + j + 1 > lo:
                        return a + j + 1
                    break
        else:
            j = win.rfind(b"\n>")
            if j >= 0 and a + j + 1 > lo:
                return a + j + 1
        if a == lo:
            return -1
        win_len *= 4


def record_chunks(src, owner):
    """Yields (buffer, start, end, fastq) with buffer[start:end] whole records
    ending in '\\n'.  owner.bufs holds two buffers of owner.cap + 16 bytes used
    in turn (a chunk stays valid until the next-but-one is produced); when a
    record does not fit, owner.grow() is called and must double owner.cap
    (with new buffers)."""
    if isinstance(src, str):
        with open(src, "rb") as fh:
            gz = fh.read(2) == _GZIP_MAGIC
    else:
        gz = bytes(src[:2]) == _GZIP_MAGIC
    fh = open(src, "rb") if isinstance(src, str) and not gz else None
    pieces = None if fh is not None else text_chunks(src, 16 << 20)
    pend = b""  # decompressed bytes not yet placed
    carry = np.zeros(0, dtype=np.uint8)
    first, fastq, i, eof = True, None, 0, False
    pos = 0  # file offset of the next byte to read (plain files)
    readers = ThreadPoolExecutor(max_workers=8) if fh is not None else None

    def pread_into(buf, lo, hi):
        """buf[lo:hi] from the file at `pos`, read by several threads at
        once (os.preadv releases the GIL); returns the bytes read."""
        parts = np.linspace(lo, hi, 9).astype(np.int64)
        jobs = [(int(a), int(b)) for a, b in zip(parts[:-1], parts[1:]) if b > a]

        def one(job):
            a, b = job
            got, mv = 0, memoryview(buf)[a:b]
            while got < b - a:
                r = os.preadv(fh.fileno(), [mv[got:]], pos + (a - lo) + got)
                if r == 0:
                    break
                got += r
            return got

        counts = list(readers.map(one, jobs))
        total = 0
        for (a, b), c in zip(jobs, counts):  # stop at the first short part (end of file)
            total += c
            if c < b - a:
                break
        return total

    try:
        while not eof or carry.size:
            buf = owner.bufs[i % 2]
            i += 1
            n = carry.size
            buf[:n] = carry
            s0 = 0
            while True:
                cap = owner.cap
                while n < cap and not eof:  # fill the rest of the buffer
                    if fh is not None:
                        got = pread_into(buf, n, cap)
                        if got < cap - n:
                            eof = True
                        n += got
                        pos += got
                    else:
                        if not pend:
                            pend = next(pieces, b"")
                            if not pend:
                                eof = True
                                break
                        take = min(len(pend), cap - n)
                        buf[n:n + take] = np.frombuffer(pend, dtype=np.uint8, count=take)
                        pend = pend[take:]
                        n += take
                if first:  # skip anything before the first record
                    head = buf[:min(n, 1 << 20)].tobytes()
                    if head[:1] not in (b">", b"@"):
                        cand = [j for j in (head.find(b"\n>"), head.find(b"\n@")) if j >= 0]
                        if not cand:
                            return
                        s0 = min(cand) + 1
                    fastq = bool(buf[s0] == ord("@"))
                    first = False
                if eof:
                    break
                cut = _last_record_start(buf, s0, n, fastq)
                if cut > s0:
                    break
                old = buf[:n].copy()  # one record fills the buffer: grow and go on
                owner.grow()
                buf = owner.bufs[(i - 1) % 2]
                buf[:n] = old
            if eof:
                end = n
                if end > s0 and buf[end - 1] != ord("\n"):
                    buf[end] = ord("\n")
                    end += 1
                carry = np.zeros(0, dtype=np.uint8)
                if end > s0:
                    yield buf, s0, end, fastq
                return
            carry = buf[cut:n].copy()
            yield buf, s0, cut, fastq
    finally:
        if fh is not None:
            fh.close()
            readers.shutdown()


class DeviceFastx:
    """Insert or query FASTA/FASTQ with the tokenising on the GPU: raw text is
    copied to the device in chunks of whole records and parsed there
    (sbf_fastx_parse_device) into a read batch that the filter's kernels take
    directly.  Chunks the device parser does not accept (multi-line FASTQ,
    mixed formats) go through the host parser.  Gzip input is decompressed on
    the host first.  A chunk holds whole records; when one record does not
    fit (512 MB by default, more than any human chromosome), the buffers are
    doubled until it does."""

    def __init__(self, filt, chunk_bytes: int = 512 << 20):
        import torch

        if filt.alphabet == 2:
            raise ValueError("multi-byte symbols (DNA triplets) need the host entry points")
        self.f, self.k, self.cap = filt, filt.k, chunk_bytes
        self._lib = load_library()
        self._torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self._alloc(chunk_bytes)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.h_off = torch.empty(0, dtype=torch.int64)   # pinned, grown on demand
        self.h_hits = torch.empty(0, dtype=torch.int32)
        self.result = (ctypes.c_uint64 * 3)()
        self._reset()

    def _reset(self) -> None:
        """Statistics of one insert or query call."""
        self.stats = {"chunks": 0, "host_fallback_chunks": 0, "records": 0, "bases": 0,
                      "text_bytes": 0, "seconds": 0.0}

    def _alloc(self, cap: int) -> None:
        torch = self._torch
        self.cap = cap
        self.bufs = [torch.empty(cap + 16, dtype=torch.uint8).pin_memory().numpy() for _ in range(2)]
        self.max_records = cap // 2 + 2  # a record takes at least 2 bytes
        self.d_text = torch.empty(cap + 16, dtype=torch.uint8, device=self.dev)
        self.d_seq = torch.empty(cap + 16, dtype=torch.uint8, device=self.dev)
        self.d_off = torch.empty(self.max_records + 1, dtype=torch.int64, device=self.dev)
        need = ctypes.c_uint64()
        _check(self._lib.sbf_fastx_device_scratch(cap + 16, ctypes.byref(need)))
        self.scratch = torch.empty(int(need.value) + 16, dtype=torch.uint8, device=self.dev)
        self.scratch_bytes = int(need.value)

    def grow(self) -> None:
        """Double the chunk size (a record did not fit)."""
        self.stream.synchronize()
        self.stats["grown_to"] = 2 * self.cap
        self._alloc(2 * self.cap)

    def _parse(self, buf, s0, end, fastq):
        """Device batch (seq, off, n_records) of one chunk, or None if the
        device parser rejected it."""
        torch = self._torch
        n = end - s0
        with torch.cuda.stream(self.stream):
            self.d_text[:n].copy_(torch.from_numpy(buf[s0:end]), non_blocking=True)
        _check(self._lib.sbf_fastx_parse_device(
            self.d_text.data_ptr(), n, 1 if fastq else 0, self.d_seq.data_ptr(), self.d_off.data_ptr(),
            self.max_records, self.scratch.data_ptr(), self.scratch_bytes, self.result,
            self.stream.cuda_stream))
        n_rec, kept, bad = int(self.result[0]), int(self.result[1]), int(self.result[2])
        self.stats["chunks"] += 1
        self.stats["text_bytes"] += n
        if bad:
            return None
        return self.d_seq[:kept], self.d_off[:n_rec + 1], n_rec

    def _host_batches(self, buf, s0, end):
        self.stats["host_fallback_chunks"] += 1
        rd = FastxReader(bytes(buf[s0:end]), self.k, batch_bytes=max(1 << 20, end - s0 + 64),
                         max_pieces=self.max_records, pinned=False)
        for seq, off, rec in rd:
            yield seq, off, rec, rd

    def insert(self, src) -> dict:
        self._reset()
        t0 = time.perf_counter()
        for buf, s0, end, fastq in record_chunks(src, self):
            b = self._parse(buf, s0, end, fastq)
            if b is None:
                for seq, off, _, _ in self._host_batches(buf, s0, end):
                    self.f.insert_host(seq, off)
                    self.stats["bases"] += seq.size
                continue
            seq, off, n_rec = b
            self.f.insert(seq, off, stream=self.stream)
            self.stats["records"] += n_rec
            self.stats["bases"] += seq.numel()
        self.stream.synchronize()
        self.stats["seconds"] = time.perf_counter() - t0
        return dict(self.stats)

    def query(self, src):
        """Per-record positive k-mers and k-mer positions (as query_fastx)."""
        torch = self._torch
        self._reset()
        hits_all, kmers_all = [], []
        t0 = time.perf_counter()
        for buf, s0, end, fastq in record_chunks(src, self):
            b = self._parse(buf, s0, end, fastq)
            if b is None:
                per_rec_h, per_rec_k = {}, {}
                for seq, off, rec, _ in self._host_batches(buf, s0, end):
                    _, h = self.f.query_host(seq, off, want_bits=False)
                    lens = np.diff(off.astype(np.int64))
                    for r, hh, L in zip(rec.tolist(), h.tolist(), lens.tolist()):
                        per_rec_h[r] = per_rec_h.get(r, 0) + hh
                        per_rec_k[r] = per_rec_k.get(r, 0) + max(0, L - (self.k - 1))
                n = max(per_rec_h) + 1 if per_rec_h else 0
                hits_all.append(np.array([per_rec_h.get(r, 0) for r in range(n)], dtype=np.uint64))
                kmers_all.append(np.array([per_rec_k.get(r, 0) for r in range(n)], dtype=np.uint64))
                continue
            seq, off, n_rec = b
            if self.h_hits.numel() < n_rec + 1:
                cap = max(n_rec + 1, 2 * self.h_hits.numel())
                self.h_hits = torch.empty(cap, dtype=torch.int32).pin_memory()
                self.h_off = torch.empty(cap + 1, dtype=torch.int64).pin_memory()
            hits = torch.empty(max(n_rec, 1), dtype=torch.int32, device=seq.device)
            self.f.query(seq, off, hits=hits[:n_rec], want_bits=False, stream=self.stream)
            with torch.cuda.stream(self.stream):
                self.h_hits[:n_rec].copy_(hits[:n_rec], non_blocking=True)
                self.h_off[:n_rec + 1].copy_(off, non_blocking=True)
            self.stream.synchronize()
            o = self.h_off[:n_rec + 1].numpy()
            hits_all.append(self.h_hits[:n_rec].numpy().view(np.uint32).astype(np.uint64))
            kmers_all.append(np.maximum(np.diff(o) - (self.k - 1), 0).astype(np.uint64))
            self.stats["records"] += n_rec
            self.stats["bases"] += seq.numel()
        self.stats["seconds"] = time.perf_counter() - t0
        hits = np.concatenate(hits_all) if hits_all else np.zeros(0, np.uint64)
        kmers = np.concatenate(kmers_all) if kmers_all else np.zeros(0, np.uint64)
        return hits, kmers, dict(self.stats)
