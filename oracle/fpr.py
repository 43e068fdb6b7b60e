"""Closed-form false-positive rates.  Test infrastructure only.

* ``bloom_fpr``: Eq. 1 of the cuSBF paper, eps = (1 - exp(-H n / M))^H.
* ``findere_fpr``: Eq. 2, eps_kmer = eps^(k-s+1).
* ``conditional_fpr``: the shard-aware form of Eq. 2 for a built filter.  A
  random alien k-mer lands in a uniform shard x; hash i of each of its k-s+1
  s-mers tests a uniform bit of sector (i mod S), which is set with
  probability f[x, i mod S] = popcount(sector) / sector_bits.  With c_j hash
  functions on sector j the k-mer is a false positive with probability
  prod_j f[x, j]^((k-s+1) c_j); averaging over x gives the expected rate.
* ``blocked_bloom_fpr``: the a-priori rate of the s = k reduction (one s-mer
  per k-mer: a blocked Bloom filter, Sec. II-A) with Poisson shard loads.
"""
from __future__ import annotations

import math

import numpy as np


def bloom_fpr(H: int, n: float, M: float) -> float:
    """Eq. 1: standard Bloom filter with M bits, H hashes, n inserted items."""
    return (1.0 - math.exp(-H * n / M)) ** H


def findere_fpr(eps: float, k: int, s: int) -> float:
    """Eq. 2: eps^(k-s+1)."""
    return eps ** (k - s + 1)


def sector_layout(H: int, shard_bits: int, layout: int = 0):
    """(S sectors, sector_bits, c_j counts) of the sectorised shard.  Layout 1
    (the paper's, Sec. IV-B) makes every 64-bit word a sector, used or not."""
    W = shard_bits // 64
    S = 1
    while 2 * S <= min(H, W):   # largest power of two not above min(H, W)
        S *= 2
    if layout == 1:
        S = W
    sector_bits = shard_bits // S
    c = np.array([sum(1 for i in range(H) if i % S == j) for j in range(S)], dtype=np.int64)
    return S, sector_bits, c


def _popcount_u64(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.uint64, copy=False)
    b = a.view(np.uint8).reshape(a.shape + (8,))
    return np.unpackbits(b, axis=-1).sum(axis=-1).astype(np.int64)


def sector_fill(words: np.ndarray, H: int, shard_bits: int, layout: int = 0) -> np.ndarray:
    """f[x, j]: fraction of set bits in sector j of shard x."""
    S, sector_bits, _ = sector_layout(H, shard_bits, layout)
    W = shard_bits // 64
    pc = _popcount_u64(np.asarray(words, dtype=np.uint64)).reshape(-1, W)
    per_sector = pc.reshape(pc.shape[0], S, W // S).sum(axis=2)
    return per_sector / float(sector_bits)


def conditional_fpr(words: np.ndarray, k: int, s: int, H: int, shard_bits: int,
                    layout: int = 0) -> float:
    """Expected false-positive rate of a random alien k-mer on this filter."""
    _, _, c = sector_layout(H, shard_bits, layout)
    f = sector_fill(words, H, shard_bits, layout)
    expo = (k - s + 1) * c
    used = expo > 0  # sectors no hash addresses (layout 1, H < 4) do not count
    with np.errstate(divide="ignore"):
        logp = (np.log(f[:, used]) * expo[None, used]).sum(axis=1)
    return float(np.exp(logp).mean())


def blocked_bloom_fpr(n: int, n_shards: int, H: int, shard_bits: int, layout: int = 0) -> float:
    """A-priori FPR of the s = k reduction: n distinct items in n_shards blocks.

    The load of a block is Poisson(n / n_shards); an item puts c_j bits into
    sector j, so a sector with load L is filled to 1 - (1 - 1/sector_bits)^(L c_j).
    """
    S, sector_bits, c = sector_layout(H, shard_bits, layout)
    lam = n / n_shards
    total = 0.0
    L = 0
    pmf = math.exp(-lam)
    while True:
        prob = 1.0
        for j in range(S):
            fill = 1.0 - (1.0 - 1.0 / sector_bits) ** (L * int(c[j]))
            prob *= fill ** int(c[j])
        total += pmf * prob
        L += 1
        pmf *= lam / L
        if L > lam and pmf < 1e-18:
            break
    return total


def binomial_two_sided_p(x: int, n: int, p: float) -> float:
    """Exact two-sided binomial p-value (sum of outcomes no more likely than x)."""
    from scipy.stats import binomtest

    return float(binomtest(int(x), int(n), float(p)).pvalue)
