"""The multi-process oracle harness (oracle/parallel.py, used for the CPU
baseline) gives exactly the single-process oracle's filter and answers:
sliced insertion OR-merged, read chunks answered from the loaded words."""
import numpy as np

from oracle import OracleSBF
from oracle.parallel import OraclePool
from paper_2606_24417_gb300 import synth


def test_pool_matches_single_process(tmp_path):
    g = synth.bacterial_genome(300_000, seed=12)
    q, qoff = synth.mixed_query_reads(g, 3000, 3000, 150, 0.01, seed=13)
    params = (31, 16, 28, 4, 1 << 22)
    o = OracleSBF(*params)
    o.insert(g, np.array([0, g.size], dtype=np.uint64))
    _, hits = o.query(q, qoff)
    gp, qp, op, wp = (str(tmp_path / n) for n in ("g.npy", "q.npy", "o.npy", "w.npy"))
    np.save(gp, g)
    np.save(qp, q)
    np.save(op, qoff)
    pool = OraclePool(*params, workers=3)
    try:
        words = pool.insert(gp, g.size, str(tmp_path))
        assert np.array_equal(words, o.words())
        np.save(wp, words)
        assert pool.query_hits(wp, qp, op, qoff.size - 1, chunk_reads=1000) == int(hits.sum())
    finally:
        pool.close()
