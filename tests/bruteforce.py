"""A second, string-level Super Bloom filter for tiny inputs (tests only).

It works on Python strings and integers and shares nothing with the C oracle:
k-mers, m-mers and s-mers are substrings, reverse complements come from
str.translate + reversal, values from base-4 digit strings.  The filter is
rebuilt from the SET of (shard, canonical s-mer) pairs that the inserted
k-mers produce, so it also checks that the oracle's bit array is exactly the
union of the pairs' bits (order- and multiplicity-free, Sec. II-B / Alg. 1).
"""
from __future__ import annotations

_DIGIT = str.maketrans("ACGTacgt", "01230123")
_RC = str.maketrans("ACGTacgt", "TGCAtgca")
_M64 = (1 << 64) - 1
_DNA = "ACGTacgt"
# alphabet -> (bits per symbol, bytes per symbol)
ALPHABETS = {0: (2, 1), 1: (5, 1), 2: (6, 3)}


def value(x: str) -> int:
    return int(x.translate(_DIGIT), 4) if x else 0


def symbol_codes(x: str, alphabet: int):
    """Codes of the symbols of x (DNA: one base each; protein: A..Z -> 0..25;
    triplet: three bases -> base-4 number), or None if one is invalid."""
    if alphabet == 0:
        return [int(ch.translate(_DIGIT)) for ch in x] if all(ch in _DNA for ch in x) else None
    if alphabet == 1:
        if not all(ch.isascii() and ch.isalpha() for ch in x):
            return None
        return [ord(ch.upper()) - ord("A") for ch in x]
    if len(x) % 3 or not all(ch in _DNA for ch in x):
        return None
    return [int(x[i:i + 3].translate(_DIGIT), 4) for i in range(0, len(x), 3)]


def revcomp(x: str) -> str:
    return x.translate(_RC)[::-1]


def mix64(x: int) -> int:
    x ^= x >> 30
    x = (x * 0xBF58476D1CE4E5B9) & _M64
    x ^= x >> 27
    x = (x * 0x94D049BB133111EB) & _M64
    x ^= x >> 31
    return x


class BruteSBF:
    def __init__(self, k, m, s, H, bits, shard_bits=512, canonical=True, layout=0, alphabet=0):
        self.k, self.m, self.s, self.H, self.B = k, m, s, H, shard_bits
        self.canonical = canonical
        self.layout = layout
        self.alphabet = alphabet
        self.sym_bits, self.sym_bytes = ALPHABETS[alphabet]
        self.N = -(-bits // shard_bits)
        if layout == 1:  # the paper's literal layout: 2^P shards of 256 bits
            assert shard_bits == 256
            self.N = 1 << (self.N - 1).bit_length()
        self.pairs = set()

    def canon(self, x: str) -> int:
        if self.alphabet != 0:  # symbol codes as digits in base 2^bits, forward only
            v = 0
            for c in symbol_codes(x, self.alphabet):
                v = (v << self.sym_bits) | c
            return v
        v = value(x)
        return min(v, value(revcomp(x))) if self.canonical else v

    def key(self, v: int) -> int:
        if self.sym_bits * self.m <= 32:
            return (v * 0x9E3779B9) % (1 << 32)
        return (v * 0x9E3779B97F4A7C15) % (1 << 64)

    def sub(self, kmer: str, i: int, length: int) -> str:
        """The length-symbol window starting at symbol i."""
        b = self.sym_bytes
        return kmer[b * i:b * (i + length)]

    def minimizer(self, kmer: str) -> int:
        mmers = [self.canon(self.sub(kmer, i, self.m)) for i in range(self.k - self.m + 1)]
        return min(mmers, key=self.key)

    def shard(self, kmer: str) -> int:
        if self.layout == 1:  # shardIdx = minHash & (NumShards - 1), Alg. 1
            return self.key(self.minimizer(kmer)) & (self.N - 1)
        return (mix64(self.minimizer(kmer) ^ 0x14057B7EF767814F) * self.N) >> 64

    def smers(self, kmer: str):
        return [self.canon(self.sub(kmer, t, self.s)) for t in range(self.k - self.s + 1)]

    def bit_positions(self, x: int, v: int):
        """Absolute bit indices of canonical s-mer v in shard x."""
        h = mix64(v ^ 0x5851F42D4C957F2D)
        W = self.B // 64
        S = W if self.layout == 1 else 1 << (min(self.H, W).bit_length() - 1)
        sector_bits = self.B // S
        b = sector_bits.bit_length() - 1
        q = 64 // self.H
        out = []
        for i in range(self.H):
            if q >= b:
                p = (h >> (i * q)) % sector_bits
            else:
                p = ((h * ((0x9E3779B97F4A7C15 * (2 * i + 1)) & _M64)) & _M64) >> (64 - b)
            out.append(x * self.B + (i % S) * sector_bits + p)
        return out

    def kmers_of(self, read: str):
        """(start byte, k-mer) of the valid k-mers of a read: one per symbol."""
        b, span = self.sym_bytes, self.k * self.sym_bytes
        for p in range(0, len(read) - span + 1, b):
            km = read[p:p + span]
            if symbol_codes(km, self.alphabet) is not None:
                yield p, km

    def insert_read(self, read: str):
        for _, km in self.kmers_of(read):
            x = self.shard(km)
            for v in self.smers(km):
                self.pairs.add((x, v))

    def bitset(self) -> set:
        out = set()
        for x, v in self.pairs:
            out.update(self.bit_positions(x, v))
        return out

    def words(self):
        import numpy as np

        w = np.zeros(self.N * self.B // 64, dtype=np.uint64)
        for bit in self.bitset():
            w[bit // 64] |= np.uint64(1 << (bit % 64))
        return w

    def query_kmer(self, km: str, bitset: set) -> bool:
        x = self.shard(km)
        return all(b in bitset for v in self.smers(km) for b in self.bit_positions(x, v))

    def query_kmer_exact(self, km: str) -> bool:
        """Membership of all of the k-mer's (shard, s-mer) pairs in the inserted set."""
        x = self.shard(km)
        return all((x, v) in self.pairs for v in self.smers(km))
