"""ctypes binding of libsbf (include/sbf.h).  Argument marshalling only.

Device inputs are torch CUDA tensors (uint8 sequences, int64 offsets, which
the library reads as uint64); host inputs are numpy arrays.  Every operation
runs in libsbf's kernels; if the library is not built the first call raises
``SbfError`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import struct
import threading

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libsbf.so")
_lib = None
_lock = threading.Lock()

SBF_OK = 0
_STATUS = {
    -1: "SBF_EINVAL", -2: "SBF_ENOMEM", -3: "SBF_ECUDA", -4: "SBF_EUNSUPPORTED",
    -5: "SBF_ETIMEOUT", -6: "SBF_EBUSY",
}


class SbfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _LIB_PATH


def load_library() -> ctypes.CDLL:
    """Load libsbf.so (in-tree build).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise SbfError(-4, f"{_LIB_PATH} is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        P, U64, I, U32P = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        sig = {
            "sbf_create": (I, [I, I, I, I, U64, ctypes.POINTER(P)]),
            "sbf_create_ex": (I, [I, I, I, I, U64, I, I, ctypes.POINTER(P)]),
            "sbf_create_layout": (I, [I, I, I, I, U64, I, I, I, ctypes.POINTER(P)]),
            "sbf_create_full": (I, [I, I, I, I, U64, I, I, I, I, ctypes.POINTER(P)]),
            "sbf_layout": (I, [P]),
            "sbf_alphabet": (I, [P]),
            "sbf_destroy": (None, [P]),
            "sbf_info": (I, [P] + [ctypes.POINTER(I)] * 6 + [ctypes.POINTER(U64)]),
            "sbf_num_words": (U64, [P]),
            "sbf_device_words": (P, [P]),
            "sbf_kernel_variant": (I, [P]),
            "sbf_device_status": (I, [P, ctypes.POINTER(ctypes.c_uint32), I]),
            "sbf_clear": (I, [P, P]),
            "sbf_get_bits": (I, [P, P]),
            "sbf_copy_bits_device": (I, [P, P, U64, U64, I, P]),
            "sbf_or_reduce_device": (I, [P, P, U64, I, P]),
            "sbf_set_bits": (I, [P, P]),
            "sbf_insert_seqs": (I, [P, P, U64, P, U64, P]),
            "sbf_query_seqs": (I, [P, P, U64, P, U64, U32P, U32P, P]),
            "sbf_query_seqs_ex": (I, [P, P, U64, P, U64, U32P, U32P, P, P]),
            "sbf_insert_seqs_host": (I, [P, P, U64, P, U64]),
            "sbf_query_seqs_host": (I, [P, P, U64, P, U64, U32P, U32P]),
            "sbf_num_kmers": (I, [P, U64, I, ctypes.POINTER(U64)]),
            "sbf_last_error": (ctypes.c_char_p, []),
            "sbf_server_create": (I, [P, U64, I, ctypes.c_uint32, ctypes.POINTER(P)]),
            "sbf_server_create_ex": (I, [P, U64, I, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.POINTER(P)]),
            "sbf_server_submit_batch": (I, [P, U64, P, P, P, P, P, P, P]),
            "sbf_server_breakdown": (I, [P, P, P, ctypes.POINTER(U64), ctypes.POINTER(U64)]),
            "sbf_server_destroy": (None, [P]),
            "sbf_server_submit": (I, [P, P, U64, P, U64, U32P, U32P, ctypes.POINTER(U64)]),
            "sbf_server_wait": (I, [P, U64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
            "sbf_server_stats": (I, [P, ctypes.POINTER(U64), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(U64)]),
            "sbf_server_reset_stats": (I, [P]),
            "sbf_batch_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P)]),
            "sbf_batch_query_noalloc": (I, [ctypes.POINTER(P), I, P, U64, P, P, U64, P, U32P, U32P,
                                            P]),
            "sbf_batch_destroy": (None, [P]),
            "sbf_batch_insert": (I, [P, P, U64, P, P, U64, P, I, P]),
            "sbf_batch_query": (I, [P, P, U64, P, P, U64, P, U32P, U32P, I, P]),
            "sbf_batch_set_schedule": (I, [P, I, I, ctypes.c_uint32, ctypes.c_uint32]),
            "sbf_batch_get_schedule": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_uint32),
                                           ctypes.POINTER(ctypes.c_uint32)]),
            "sbf_batch_tune": (I, [P, I, P, U64, P, P, U64, P, U32P, U32P, P,
                                   ctypes.POINTER(ctypes.c_float)]),
            "sbf_probe_sectors": (I, [P, U64, I, U64, U64, I, P, P]),
            "sbf_fastx_create": (I, [I, ctypes.POINTER(P)]),
            "sbf_fastx_device_scratch": (I, [U64, ctypes.POINTER(U64)]),
            "sbf_fastx_parse_device": (I, [P, U64, I, P, P, U64, P, U64, P, P]),
            "sbf_fastx_destroy": (None, [P]),
            "sbf_fastx_parse": (I, [P, P, U64, I, P, U64, P, P, U64, ctypes.POINTER(U64),
                                    ctypes.POINTER(U64), ctypes.POINTER(U64)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int) -> None:
    if rc != SBF_OK:
        msg = load_library().sbf_last_error()
        raise SbfError(rc, msg.decode() if msg else "")


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_ptr(t, dtype_size: int | None = None) -> int:
    if t is None:
        return 0
    if not t.is_cuda:
        raise SbfError(-1, "expected a CUDA tensor")
    if not t.is_contiguous():
        raise SbfError(-1, "expected a contiguous tensor")
    if dtype_size is not None and t.element_size() != dtype_size:
        raise SbfError(-1, f"expected {dtype_size}-byte elements, got {t.dtype}")
    return int(t.data_ptr())


def _host_ptr(a) -> int:
    return int(a.ctypes.data) if a is not None and a.size else 0


class SuperBloomFilter:
    """A Super Bloom filter resident in device memory (owned by libsbf).

    k, m, s, H: k-mer, minimizer and Findere s-mer lengths and hash count;
    bits: filter size (rounded up to whole shards); shard_bits: 256 or 512;
    canonical: treat a k-mer and its reverse complement as one key;
    layout: LAYOUT_DEFAULT, or LAYOUT_PAPER for the paper's literal layout
    (256-bit shards, 2^P of them, shard = minimizer key & (2^P - 1), hash i
    in 64-bit word i mod 4);
    alphabet: "dna" (or 0), "protein" (1) or "dna_triplet" (2); the latter two
    are forward only (pass canonical=False).
    """

    def __init__(self, k: int = 31, m: int = 16, s: int = 28, H: int = 4, bits: int = 1 << 30,
                 shard_bits: int = 512, canonical: bool = True, layout: int = 0, alphabet=0):
        lib = load_library()
        alphabet = ALPHABETS.get(alphabet, alphabet)
        h = ctypes.c_void_p()
        _check(lib.sbf_create_full(k, m, s, H, bits, shard_bits, 1 if canonical else 0, layout,
                                   alphabet, ctypes.byref(h)))
        self._h = h
        self._lib = lib
        ki, mi, si, Hi, Bi, ci = (ctypes.c_int() for _ in range(6))
        n = ctypes.c_uint64()
        _check(lib.sbf_info(h, ctypes.byref(ki), ctypes.byref(mi), ctypes.byref(si),
                            ctypes.byref(Hi), ctypes.byref(Bi), ctypes.byref(ci), ctypes.byref(n)))
        self.k, self.m, self.s, self.H = ki.value, mi.value, si.value, Hi.value
        self.shard_bits, self.canonical = Bi.value, bool(ci.value)
        self.n_shards = int(n.value)
        self.n_words = int(lib.sbf_num_words(h))
        self.layout = int(lib.sbf_layout(h))
        self.alphabet = int(lib.sbf_alphabet(h))

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.sbf_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def nbytes(self) -> int:
        return self.n_words * 8

    @property
    def fused(self) -> bool:
        """True if the fused kernels serve this filter."""
        return self._lib.sbf_kernel_variant(self._h) == 1

    @property
    def kernel_variant(self) -> str:
        """The kernels that serve this filter: 'fused', 'rolling' (every
        parameter set outside the fused grid) or 'generic' (one k-mer per
        thread, only when the environment sets SBF_FORCE_GENERIC)."""
        return {0: "generic", 1: "fused", 2: "rolling"}[self._lib.sbf_kernel_variant(self._h)]

    def device_status(self, clear: bool = False) -> int:
        """0 while every launch on this filter ran to completion; bit 0 set
        after a fused query gave up a bounded wait for shard copies (its
        answers are then incomplete).  Synchronous."""
        st = ctypes.c_uint32()
        _check(self._lib.sbf_device_status(self._h, ctypes.byref(st), 1 if clear else 0))
        return int(st.value)

    def device_words_ptr(self) -> int:
        return int(self._lib.sbf_device_words(self._h))

    # -- device-resident batches ------------------------------------------
    def insert(self, seq, off, stream=None) -> None:
        """seq: uint8 CUDA tensor; off: int64 CUDA tensor of n_reads + 1 offsets."""
        _check(self._lib.sbf_insert_seqs(self._h, _dev_ptr(seq, 1), seq.numel(), _dev_ptr(off, 8),
                                         off.numel() - 1, _stream_handle(stream)))

    def query(self, seq, off, bits=None, hits=None, stats=None, stream=None, want_bits=True,
              want_hits=True):
        """Returns (bits int32[ceil(len/32)], hits int32[n_reads]) CUDA tensors.

        The int32 tensors hold the library's uint32 words (reinterpret with
        ``.view(torch.uint32)`` or mask with 0xFFFFFFFF)."""
        import torch

        n = off.numel() - 1
        if bits is None and want_bits:
            bits = torch.empty((seq.numel() + 31) // 32, dtype=torch.int32, device=seq.device)
        if hits is None and want_hits:
            hits = torch.empty(max(n, 0), dtype=torch.int32, device=seq.device)
        _check(self._lib.sbf_query_seqs_ex(self._h, _dev_ptr(seq, 1), seq.numel(), _dev_ptr(off, 8),
                                           n, _dev_ptr(bits, 4), _dev_ptr(hits, 4),
                                           _dev_ptr(stats, 8), _stream_handle(stream)))
        return bits, hits

    def clear(self, stream=None) -> None:
        _check(self._lib.sbf_clear(self._h, _stream_handle(stream)))

    # -- host-resident batches --------------------------------------------
    def insert_host(self, seq: np.ndarray, off: np.ndarray) -> None:
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        _check(self._lib.sbf_insert_seqs_host(self._h, _host_ptr(seq), seq.size, _host_ptr(off),
                                              off.size - 1))

    def query_host(self, seq: np.ndarray, off: np.ndarray, bits: np.ndarray | None = None,
                   hits: np.ndarray | None = None, want_bits: bool = True):
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        if bits is None and want_bits:
            bits = np.empty((seq.size + 31) // 32, dtype=np.uint32)
        if hits is None:
            hits = np.empty(off.size - 1, dtype=np.uint32)
        _check(self._lib.sbf_query_seqs_host(self._h, _host_ptr(seq), seq.size, _host_ptr(off),
                                             off.size - 1, _host_ptr(bits), _host_ptr(hits)))
        return bits, hits

    # -- bit array and checkpoints -----------------------------------------
    def words(self) -> np.ndarray:
        out = np.empty(self.n_words, dtype=np.uint64)
        _check(self._lib.sbf_get_bits(self._h, _host_ptr(out)))
        return out

    def copy_words_device(self, dst, word_begin: int = 0, to_filter: bool = False,
                          stream=None) -> None:
        """Copy words [word_begin, word_begin + dst.numel()) of the filter to
        the int64 CUDA tensor dst (or from it into the filter)."""
        _check(self._lib.sbf_copy_bits_device(self._h, _dev_ptr(dst, 8), word_begin, dst.numel(),
                                              1 if to_filter else 0, _stream_handle(stream)))

    def set_words(self, w: np.ndarray) -> None:
        w = np.ascontiguousarray(w, dtype=np.uint64)
        if w.size != self.n_words:
            raise SbfError(-1, f"expected {self.n_words} words, got {w.size}")
        _check(self._lib.sbf_set_bits(self._h, _host_ptr(w)))

    _MAGIC = b"SBFGB300"
    _VERSION = 3  # version 1: no layout (0); version 2: no alphabet (DNA)

    def save(self, path: str) -> None:
        """Checkpoint: header (magic, version, k, m, s, H, shard_bits,
        canonical, n_shards, layout, alphabet) followed by the raw
        little-endian words."""
        hdr = struct.pack("<8sIiiiiiiQii", self._MAGIC, self._VERSION, self.k, self.m, self.s,
                          self.H, self.shard_bits, int(self.canonical), self.n_shards, self.layout,
                          self.alphabet)
        with open(path, "wb") as fh:
            fh.write(hdr)
            fh.write(self.words().astype("<u8").tobytes())

    @classmethod
    def load(cls, path: str) -> "SuperBloomFilter":
        size1 = struct.calcsize("<8sIiiiiiiQ")
        with open(path, "rb") as fh:
            hdr = fh.read(size1)
            magic, ver, k, m, s, H, B, canon, n = struct.unpack("<8sIiiiiiiQ", hdr)
            if magic != cls._MAGIC or ver not in (1, 2, 3):
                raise SbfError(-1, f"{path}: not a filter checkpoint")
            layout = struct.unpack("<i", fh.read(4))[0] if ver >= 2 else 0
            alphabet = struct.unpack("<i", fh.read(4))[0] if ver >= 3 else 0
            f = cls(k, m, s, H, n * B, shard_bits=B, canonical=bool(canon), layout=layout,
                    alphabet=alphabet)
            w = np.frombuffer(fh.read(), dtype="<u8")
            f.set_words(w)
        return f


BATCH_PER_FILTER, BATCH_FUSED, BATCH_GRAPH = 0, 1, 2
LAYOUT_DEFAULT, LAYOUT_PAPER = 0, 1
ALPHABET_DNA, ALPHABET_PROTEIN, ALPHABET_DNA_TRIPLET = 0, 1, 2
ALPHABETS = {"dna": 0, "protein": 1, "dna_triplet": 2}


class FilterBatch:
    """Filters with one parameter set served by one persistent launch.

    Reads are grouped by filter: ``group[f]:group[f+1]`` are filter f's reads.
    ``off`` must be given both on the device (int64 CUDA tensor) and on the
    host (numpy uint64)."""

    def __init__(self, filters):
        lib = load_library()
        self._filters = list(filters)  # keep them alive
        arr = (ctypes.c_void_p * len(self._filters))(*[f.handle.value for f in self._filters])
        h = ctypes.c_void_p()
        _check(lib.sbf_batch_create(arr, len(self._filters), ctypes.byref(h)))
        self._h = h
        self._lib = lib

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.sbf_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _host(off_host, group):
        off_host = np.ascontiguousarray(off_host, dtype=np.uint64)
        group = np.ascontiguousarray(group, dtype=np.uint64)
        return off_host, group

    def insert(self, seq, off, off_host, group, mode: int = BATCH_GRAPH, stream=None) -> None:
        oh, gr = self._host(off_host, group)
        _check(self._lib.sbf_batch_insert(self._h, _dev_ptr(seq, 1), seq.numel(), _dev_ptr(off, 8),
                                          _host_ptr(oh), oh.size - 1, _host_ptr(gr), mode,
                                          _stream_handle(stream)))

    def query(self, seq, off, off_host, group, bits=None, hits=None, mode: int = BATCH_GRAPH,
              stream=None):
        import torch

        oh, gr = self._host(off_host, group)
        n = oh.size - 1
        if bits is None:
            bits = torch.empty((seq.numel() + 31) // 32, dtype=torch.int32, device=seq.device)
        if hits is None:
            hits = torch.empty(n, dtype=torch.int32, device=seq.device)
        _check(self._lib.sbf_batch_query(self._h, _dev_ptr(seq, 1), seq.numel(), _dev_ptr(off, 8),
                                         _host_ptr(oh), n, _host_ptr(gr), _dev_ptr(bits, 4),
                                         _dev_ptr(hits, 4), mode, _stream_handle(stream)))
        return bits, hits

    def set_schedule(self, dynamic: bool, chunk: int, grid_blocks: int = 0,
                     insert: bool = False) -> None:
        _check(self._lib.sbf_batch_set_schedule(self._h, 1 if insert else 0, 1 if dynamic else 0,
                                                chunk, grid_blocks))

    def schedule(self, insert: bool = False):
        d, c, g = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(self._lib.sbf_batch_get_schedule(self._h, 1 if insert else 0, ctypes.byref(d),
                                                ctypes.byref(c), ctypes.byref(g)))
        return bool(d.value), int(c.value), int(g.value)

    def tune(self, seq, off, off_host, group, insert: bool = False, bits=None, hits=None,
             stream=None) -> float:
        """Autotune the schedule on this call; returns the best time in ms."""
        import torch

        oh, gr = self._host(off_host, group)
        n = oh.size - 1
        if not insert:
            if bits is None:
                bits = torch.empty((seq.numel() + 31) // 32, dtype=torch.int32, device=seq.device)
            if hits is None:
                hits = torch.empty(n, dtype=torch.int32, device=seq.device)
        best = ctypes.c_float()
        _check(self._lib.sbf_batch_tune(self._h, 1 if insert else 0, _dev_ptr(seq, 1), seq.numel(),
                                        _dev_ptr(off, 8), _host_ptr(oh), n, _host_ptr(gr),
                                        _dev_ptr(bits, 4), _dev_ptr(hits, 4),
                                        _stream_handle(stream), ctypes.byref(best)))
        return float(best.value)


class FilterServer:
    """Continuous-batching request loop around one resident filter.

    ``submit`` queues host reads and returns a ticket; ``wait`` blocks (with a
    timeout) until the answers are in the caller's buffers.  Buffers passed
    to ``submit`` are kept alive here until waited for."""

    def __init__(self, filt: "SuperBloomFilter", read_budget_bytes: int = 256 << 20,
                 max_inflight: int = 3, max_per_launch: int = 4096, stage_inputs: bool = False):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.sbf_server_create_ex(filt.handle, read_budget_bytes, max_inflight,
                                        max_per_launch, 1 if stage_inputs else 0,
                                        ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self._filter = filt
        self._keep = {}
        self._lock = threading.Lock()

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.sbf_server_destroy(h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, seq: np.ndarray, off: np.ndarray, want_bits: bool = False):
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        n = off.size - 1
        hits = np.empty(n, dtype=np.uint32)
        bits = np.empty((seq.size + 31) // 32, dtype=np.uint32) if want_bits else None
        t = ctypes.c_uint64()
        _check(self._lib.sbf_server_submit(self._h, _host_ptr(seq), seq.size, _host_ptr(off), n,
                                           _host_ptr(hits), _host_ptr(bits), ctypes.byref(t)))
        with self._lock:
            self._keep[t.value] = (seq, off, hits, bits)
        return t.value

    def submit_many(self, requests, want_bits: bool = False):
        """Queue many (seq, off) requests with one call; returns their tickets."""
        n = len(requests)
        if n == 0:
            return []
        seqs = [np.ascontiguousarray(q[0], dtype=np.uint8) for q in requests]
        offs = [np.ascontiguousarray(q[1], dtype=np.uint64) for q in requests]
        hits = [np.empty(o.size - 1, dtype=np.uint32) for o in offs]
        bits = [np.empty((q.size + 31) // 32, dtype=np.uint32) for q in seqs] if want_bits else None
        ptr = lambda arrs: np.array([a.ctypes.data for a in arrs], dtype=np.uint64)  # noqa: E731
        p_seq, p_off, p_hits = ptr(seqs), ptr(offs), ptr(hits)
        p_bits = ptr(bits) if want_bits else None
        lens = np.array([q.size for q in seqs], dtype=np.uint64)
        nr = np.array([o.size - 1 for o in offs], dtype=np.uint64)
        t = np.empty(n, dtype=np.uint64)
        _check(self._lib.sbf_server_submit_batch(self._h, n, _host_ptr(p_seq), _host_ptr(lens),
                                                 _host_ptr(p_off), _host_ptr(nr), _host_ptr(p_hits),
                                                 _host_ptr(p_bits) if want_bits else None,
                                                 _host_ptr(t)))
        tickets = [int(x) for x in t]
        with self._lock:
            for i, tk in enumerate(tickets):
                self._keep[tk] = (seqs[i], offs[i], hits[i], bits[i] if want_bits else None)
        return tickets

    def breakdown(self) -> dict:
        """p50 / p99 seconds per stage (queued, launching, device, delivery)
        and how many requests were read in place or staged."""
        p50 = (ctypes.c_double * 4)()
        p99 = (ctypes.c_double * 4)()
        d, st = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.sbf_server_breakdown(self._h, p50, p99, ctypes.byref(d), ctypes.byref(st)))
        names = ("queued", "launching", "device", "delivery")
        return {"p50_s": dict(zip(names, list(p50))), "p99_s": dict(zip(names, list(p99))),
                "direct_requests": int(d.value), "staged_requests": int(st.value)}

    def wait(self, ticket: int, timeout_s: float = 60.0):
        """Returns (hits, bits or None, latency seconds)."""
        lat = ctypes.c_double()
        rc = self._lib.sbf_server_wait(self._h, ticket, timeout_s, ctypes.byref(lat))
        with self._lock:
            keep = self._keep.pop(ticket, None) if rc != -5 else self._keep.get(ticket)
        _check(rc)
        return keep[2], keep[3], float(lat.value)

    def stats(self) -> dict:
        c, l = ctypes.c_uint64(), ctypes.c_uint64()
        p50, p99, mean, kps = (ctypes.c_double() for _ in range(4))
        _check(self._lib.sbf_server_stats(self._h, ctypes.byref(c), ctypes.byref(p50),
                                          ctypes.byref(p99), ctypes.byref(mean), ctypes.byref(kps),
                                          ctypes.byref(l)))
        return {"completed": int(c.value), "p50_s": p50.value, "p99_s": p99.value,
                "mean_s": mean.value, "kmers_per_s": kps.value, "launches": int(l.value)}

    def reset_stats(self) -> None:
        _check(self._lib.sbf_server_reset_stats(self._h))


def or_reduce_device(out, parts, stream=None) -> None:
    """out[i] = OR over rows j of parts[j, i]: int64 CUDA tensors, parts of
    shape (n_parts, n) contiguous, out of n elements (the OR of filters that
    inserted disjoint read shares).  Asynchronous on `stream`."""
    if parts.dim() != 2 or not parts.is_contiguous() or out.numel() != parts.shape[1]:
        raise SbfError(-1, "parts must be a contiguous (n_parts, n) tensor and out hold n words")
    _check(load_library().sbf_or_reduce_device(_dev_ptr(out, 8), _dev_ptr(parts, 8), out.numel(),
                                               parts.shape[0], _stream_handle(stream)))


def batch_query_noalloc(filters, seq, off, off_host, group, bits, hits, stream=None):
    """Batched query whose scratch is a fixed array inside libsbf: for callers
    that cannot allocate device memory.  ``bits`` and ``hits`` must be given
    (preallocated int32 CUDA tensors); nothing is allocated here."""
    lib = load_library()
    arr = (ctypes.c_void_p * len(filters))(*[f.handle.value for f in filters])
    oh = np.ascontiguousarray(off_host, dtype=np.uint64)
    gr = np.ascontiguousarray(group, dtype=np.uint64)
    # the C side reads group[n_filters] and off_host[n_reads] and writes up to
    # these sizes on the device: refuse short arrays before the call
    if gr.size != len(filters) + 1:
        raise SbfError(-1, f"group has {gr.size} entries, want {len(filters) + 1}")
    if oh.size < 1 or off.numel() != oh.size:
        raise SbfError(-1, "device and host offsets differ in length")
    if bits is None or hits is None:
        raise SbfError(-1, "bits and hits must be preallocated")
    if bits.numel() < (seq.numel() + 31) // 32 or hits.numel() < oh.size - 1:
        raise SbfError(-1, "bits or hits too small for the batch")
    _check(lib.sbf_batch_query_noalloc(arr, len(filters), _dev_ptr(seq, 1), seq.numel(),
                                       _dev_ptr(off, 8), _host_ptr(oh), oh.size - 1, _host_ptr(gr),
                                       _dev_ptr(bits, 4), _dev_ptr(hits, 4), _stream_handle(stream)))
    return bits, hits


def probe_sectors(buf, sector_bytes: int, n: int, seed: int = 0, rmw: bool = False, sink=None,
                  stream=None) -> None:
    """Random-sector bandwidth probe over the device tensor `buf` (measurement
    only): n random sector loads, or n atomicOr read-modify-writes of a whole
    sector when `rmw`.  Asynchronous; time it with CUDA events."""
    import torch

    lib = load_library()
    if sink is None:
        sink = torch.zeros(1, dtype=torch.int64, device=buf.device)
    _check(lib.sbf_probe_sectors(_dev_ptr(buf), buf.numel() * buf.element_size(), sector_bytes, n,
                                 seed, 1 if rmw else 0, _dev_ptr(sink, 8), _stream_handle(stream)))


def num_kmers(off: np.ndarray, k: int) -> int:
    off = np.ascontiguousarray(off, dtype=np.uint64)
    out = ctypes.c_uint64()
    _check(load_library().sbf_num_kmers(_host_ptr(off), off.size - 1, k, ctypes.byref(out)))
    return int(out.value)
