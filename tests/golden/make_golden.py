"""Writes oracle_regression.json: digests of the oracle's filter and answers on
small seeded workloads.  Calls only the oracle and the input generators; it
records the oracle as pinned by tests/test_oracle_pins.py so that any later
change of its arithmetic shows up (and has to name its justification)."""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleSBF  # noqa: E402
from paper_2606_24417_gb300 import synth  # noqa: E402

CASES = [
    # name, k, m, s, H, bits, B, canonical
    ("uniform_1e5_31_16_28_4_512", 31, 16, 28, 4, 1 << 20, 512, True),
    ("uniform_1e5_31_16_28_4_256", 31, 16, 28, 4, 1 << 20, 256, True),
    ("uniform_1e5_31_20_24_8_512", 31, 20, 24, 8, 1 << 20, 512, True),
    ("uniform_1e5_9_5_6_2_256_fwd", 9, 5, 6, 2, 1 << 16, 256, False),
]


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def compute():
    g = synth.uniform_dna(100_000, 0)
    off = np.array([0, g.size], dtype=np.uint64)
    q, qoff = synth.mixed_query_reads(g, 500, 500, 150, 0.01, seed=3)
    out = {}
    for name, k, m, s, H, bits, B, canon in CASES:
        f = OracleSBF(k, m, s, H, bits, shard_bits=B, canonical=canon)
        f.insert(g, off)
        w = f.words()
        qb, qh = f.query(q, qoff)
        out[name] = {
            "params": [k, m, s, H, bits, B, int(canon)],
            "words_sha256": digest(w),
            "set_bits": int(np.unpackbits(w.view(np.uint8)).sum()),
            "query_bits_sha256": digest(qb),
            "query_hits_sum": int(qh.sum()),
        }
    return out


if __name__ == "__main__":
    res = {"generator": "tests/golden/make_golden.py (oracle + synth only)", "cases": compute()}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as fh:
        json.dump(res, fh, indent=1)
    print(json.dumps(res, indent=1))
