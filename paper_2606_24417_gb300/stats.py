"""Filter statistics computed from a filter's bit array (host side).

expected_fpr: the false-positive rate a random alien k-mer is expected to
have on a built filter -- its shard is uniform, and hash i of each of its
k-s+1 s-mers tests a uniform bit of sector (i mod S), set with probability
fill[x, sector]; the k-mer is positive only if all (k-s+1)*H tests pass
(Findere, Eq. 2, made shard-aware).  Used by the parameter sweep to put the
measured rate beside the expected one.
"""
from __future__ import annotations

import numpy as np


def _popcount64(a: np.ndarray) -> np.ndarray:
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    b = a.view(np.uint8).reshape(a.shape + (8,))
    return np.unpackbits(b, axis=-1).sum(axis=-1).astype(np.int64)


def expected_fpr(words: np.ndarray, k: int, s: int, H: int, shard_bits: int,
                 layout: int = 0) -> float:
    """Layout 1 (the paper's) has one sector per 64-bit word; sectors no hash
    uses (H < 4) do not enter the product.  Under layout 1 an alien's shard is
    only close to uniform (it is the low bits of its minimizer key), so this
    is the uniform-shard approximation there."""
    w64 = shard_bits // 64
    sectors = min(H, w64)
    while sectors & (sectors - 1):   # largest power of two not above min(H, W)
        sectors &= sectors - 1
    if layout == 1:
        sectors = w64
    per_sector = _popcount64(np.asarray(words, dtype=np.uint64)).reshape(-1, sectors, w64 // sectors).sum(axis=2)
    fill = per_sector / float(shard_bits // sectors)
    uses = np.array([sum(1 for i in range(H) if i % sectors == j) for j in range(sectors)])
    used = uses > 0
    with np.errstate(divide="ignore"):
        logp = (np.log(fill[:, used]) * ((k - s + 1) * uses[used])[None, :]).sum(axis=1)
    return float(np.exp(logp).mean())
