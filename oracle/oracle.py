"""ctypes wrapper of the C oracle (``sbf_oracle.c``).  Test infrastructure only.

The library is compiled with plain ``gcc`` into ``oracle/liboracle.so``
(``build_oracle``); nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def oracle_library_path() -> str:
    return _LIB_PATH


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (host code only; same result on x86 and Arm)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(os.path.join(_HERE, "sbf_oracle.h")))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra",
                   "-o", tmp, _SRC]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        U64 = ctypes.c_uint64
        I = ctypes.c_int
        lib.oracle_create.restype = P
        lib.oracle_create.argtypes = [I, I, I, I, I, I, U64]
        lib.oracle_create_layout.restype = P
        lib.oracle_create_layout.argtypes = [I, I, I, I, I, I, U64, I]
        lib.oracle_create_full.restype = P
        lib.oracle_create_full.argtypes = [I, I, I, I, I, I, U64, I, I]
        lib.oracle_destroy.argtypes = [P]
        lib.oracle_destroy.restype = None
        lib.oracle_num_shards.argtypes = [P]
        lib.oracle_num_shards.restype = U64
        lib.oracle_num_words.argtypes = [P]
        lib.oracle_num_words.restype = U64
        lib.oracle_words.argtypes = [P]
        lib.oracle_words.restype = P
        lib.oracle_insert.argtypes = [P, P, U64, P, U64]
        lib.oracle_insert.restype = None
        lib.oracle_query.argtypes = [P, P, U64, P, U64, P, P]
        lib.oracle_query.restype = None
        lib.oracle_query_positions.argtypes = [P, P, U64, P, U64, P, U64, P]
        lib.oracle_query_positions.restype = None
        lib.oracle_count_runs.argtypes = [P, P, U64, P, U64, P, P]
        lib.oracle_count_runs.restype = None
        lib.oracle_kmer_info.argtypes = [P, P, P, P]
        lib.oracle_kmer_info.restype = None
        lib.oracle_runs_of_keys.argtypes = [P, P, U64]
        lib.oracle_runs_of_keys.restype = U64
        lib.oracle_mix64.argtypes = [U64]
        lib.oracle_mix64.restype = U64
        _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a)
    assert a.dtype == np.uint8
    return a


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


class OracleSBF:
    """Plain CPU Super Bloom filter with the library's parameter domain."""

    ALPHABETS = {"dna": 0, "protein": 1, "dna_triplet": 2}
    SYMBOL_BYTES = {0: 1, 1: 1, 2: 3}

    def __init__(self, k: int, m: int, s: int, H: int, bits: int, shard_bits: int = 512,
                 canonical: bool = True, layout: int = 0, alphabet: int = 0):
        lib = _load()
        alphabet = self.ALPHABETS.get(alphabet, alphabet)
        h = lib.oracle_create_full(k, m, s, H, shard_bits, 1 if canonical else 0, bits, layout,
                                   alphabet)
        if not h:
            raise ValueError(f"invalid oracle parameters k={k} m={m} s={s} H={H} "
                             f"shard_bits={shard_bits} bits={bits} layout={layout} "
                             f"alphabet={alphabet} canonical={canonical}")
        self.alphabet = alphabet
        self.symbol_bytes = self.SYMBOL_BYTES[alphabet]
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        self.k, self.m, self.s, self.H = k, m, s, H
        self.shard_bits = shard_bits
        self.canonical = bool(canonical)
        self.layout = layout
        self.n_shards = int(lib.oracle_num_shards(self._h))
        self.n_words = int(lib.oracle_num_words(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.oracle_destroy(h)
            self._h = None

    # -- bit array ---------------------------------------------------------
    def words(self) -> np.ndarray:
        """Copy of the filter as uint64 words."""
        addr = self._lib.oracle_words(self._h)
        buf = (ctypes.c_uint64 * self.n_words).from_address(addr)
        return np.frombuffer(buf, dtype=np.uint64).copy()

    def words_view(self) -> np.ndarray:
        """The filter's uint64 words without a copy; valid while this object
        lives (for tests that reduce multi-GiB filters across processes)."""
        addr = self._lib.oracle_words(self._h)
        buf = (ctypes.c_uint64 * self.n_words).from_address(addr)
        return np.frombuffer(buf, dtype=np.uint64)

    def set_words(self, w: np.ndarray) -> None:
        w = _u64(w)
        assert w.size == self.n_words
        addr = self._lib.oracle_words(self._h)
        ctypes.memmove(addr, w.ctypes.data, w.nbytes)

    # -- sequence operations -----------------------------------------------
    def insert(self, seq, off) -> None:
        seq = _u8(seq)
        off = _u64(off)
        self._lib.oracle_insert(self._h, _ptr(seq), seq.size, _ptr(off), off.size - 1)

    def query(self, seq, off):
        """Returns (bits uint32[ceil(len/32)], hits uint32[n_reads])."""
        seq = _u8(seq)
        off = _u64(off)
        n = off.size - 1
        bits = np.zeros((seq.size + 31) // 32, dtype=np.uint32)
        hits = np.zeros(n, dtype=np.uint32)
        self._lib.oracle_query(self._h, _ptr(seq), seq.size, _ptr(off), n, _ptr(bits), _ptr(hits))
        return bits, hits

    def query_positions(self, seq, off, positions) -> np.ndarray:
        seq = _u8(seq)
        off = _u64(off)
        pos = _u64(positions)
        out = np.zeros(pos.size, dtype=np.uint8)
        self._lib.oracle_query_positions(self._h, _ptr(seq), seq.size, _ptr(off), off.size - 1,
                                         _ptr(pos), pos.size, _ptr(out))
        return out

    def count_runs(self, seq, off):
        """(valid k-mers, super-k-mer runs) of a read batch."""
        seq = _u8(seq)
        off = _u64(off)
        v = ctypes.c_uint64(0)
        r = ctypes.c_uint64(0)
        self._lib.oracle_count_runs(self._h, _ptr(seq), seq.size, _ptr(off), off.size - 1,
                                    ctypes.byref(v), ctypes.byref(r))
        return int(v.value), int(r.value)

    def kmer_info(self, kmer) -> tuple[int, int]:
        """(minimizer value, shard) of one k-mer given as k bytes."""
        x = _u8(kmer)
        assert x.size == self.k * self.symbol_bytes
        mu = ctypes.c_uint64(0)
        sh = ctypes.c_uint64(0)
        self._lib.oracle_kmer_info(self._h, _ptr(x), ctypes.byref(mu), ctypes.byref(sh))
        return int(mu.value), int(sh.value)


def runs_of_keys(keys, active) -> int:
    """Run count of a lane sequence (Fig. 4's segmented reduction)."""
    lib = _load()
    k = _u64(keys)
    a = np.ascontiguousarray(np.asarray(active, dtype=np.uint8))
    assert k.size == a.size
    return int(lib.oracle_runs_of_keys(_ptr(k), _ptr(a), k.size))


def mix64(x: int) -> int:
    """The oracle's 64-bit finaliser (SplitMix64's output function)."""
    return int(_load().oracle_mix64(int(x) & 0xFFFFFFFFFFFFFFFF))
