"""Oracle parity of the batched and served workloads at their full sizes.

Batched: 256 filters of 2^20-2^28 bits built from 3.07 Gbp of genomes, 5M
reads of lognormal lengths, in the launch configuration the benchmark times
(tuned schedule, one persistent launch replayed from a CUDA graph).  Every
filter's words equal the oracle's; a seeded 1% of the reads plus every read
longer than 10 kb equal the oracle's answers bit for bit.

Served: the 3.1 Gbp human-shaped genome in a 2^35-bit (4 GiB) filter.  The
whole array equals the oracle's (compared in chunks by digest, with a count
of differing words on a mismatch); a seeded sample of the request pool is
answered identically alone, in a four-client mix, by a direct query and by
the oracle.

Integer work: the tolerance is zero everywhere (Alg. 1 and Alg. 2 fix every
bit)."""
import threading

import numpy as np
import pytest

from paper_2606_24417_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K, M, S, H, B = 31, 16, 28, 4, 512
PARAMS = (K, M, S, H, B, True)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_off(off):
    return dev(np.asarray(off, dtype=np.uint64).astype(np.int64))


def bits_at(words_u32, pos):
    """Answer bits at start positions `pos` of a uint32 answer array."""
    pos = np.asarray(pos, dtype=np.int64)
    return ((words_u32[pos >> 5] >> (pos & 31).astype(np.uint32)) & 1).astype(np.uint8)


def ranges(off, reads):
    """Concatenated positions [off[r], off[r+1]) of the given reads."""
    a = off[reads].astype(np.int64)
    L = (off[reads + 1] - off[reads]).astype(np.int64)
    base = np.repeat(a - np.concatenate([[0], np.cumsum(L)[:-1]]), L)
    return base + np.arange(int(L.sum()), dtype=np.int64)


def unpack(words_u32, n):
    return np.unpackbits(np.ascontiguousarray(words_u32).view(np.uint8), bitorder="little")[:n]


# ---------------------------------------------------------------------------
# batched: 256 filters, 5M reads
# ---------------------------------------------------------------------------
def test_batched_256_filters_full_size(tmp_path):
    from oracle_fullsize import ManyFilters
    from paper_2606_24417_gb300.sbf import BATCH_GRAPH, FilterBatch, SuperBloomFilter

    w = synth.batched_workload(n_filters=256, n_reads=5_000_000, seed=4)
    goff, off, group = w["goff"], w["off"], w["group"]
    filters = [SuperBloomFilter(K, M, S, H, b, shard_bits=B) for b in w["bits"]]
    batch = FilterBatch(filters)
    dg, dgo = dev(w["gseq"]), dev_off(goff)
    # the benchmark's configuration: tuned schedule, graph replay (re-inserting
    # the same genomes sets no new bit, so tuning leaves the filters exact)
    batch.tune(dg, dgo, goff, w["ggroup"], insert=True)
    batch.insert(dg, dgo, goff, w["ggroup"], mode=BATCH_GRAPH)
    torch.cuda.synchronize()
    del dg, dgo
    gpu_words = [f.words() for f in filters]

    pool = ManyFilters(PARAMS, w["gseq"], tmp_path)
    try:
        want = pool.insert_all(w["bits"], goff)
        bad = [f for f in range(len(filters)) if not np.array_equal(gpu_words[f], want[f])]
        assert not bad, f"filters differing from the oracle: {bad[:10]} ({len(bad)} in all)"
        for f in range(len(filters)):
            pool.save_words(f, want[f])

        dq, dqo = dev(w["seq"]), dev_off(off)
        bits = torch.empty((w["seq"].size + 31) // 32, dtype=torch.int32, device="cuda")
        hits = torch.empty(off.size - 1, dtype=torch.int32, device="cuda")
        batch.tune(dq, dqo, off, group, bits=bits, hits=hits)
        batch.query(dq, dqo, off, group, bits=bits, hits=hits, mode=BATCH_GRAPH)
        torch.cuda.synchronize()
        gbits = bits.cpu().numpy().view(np.uint32)
        ghits = hits.cpu().numpy().view(np.uint32)
        del dq, dqo

        # a seeded 1% of the reads and every read longer than 10 kb
        n_reads = off.size - 1
        lens = np.diff(off.astype(np.int64))
        rng = np.random.default_rng(4)
        sample = np.union1d(rng.choice(n_reads, n_reads // 100, replace=False),
                            np.nonzero(lens > 10_000)[0])
        owner = np.searchsorted(group.astype(np.int64), sample, side="right") - 1
        tasks = []
        for f in np.unique(owner):
            rs = sample[owner == f]
            seq = np.concatenate([w["seq"][int(off[r]):int(off[r + 1])] for r in rs])
            soff = np.concatenate([[0], np.cumsum(lens[rs])]).astype(np.uint64)
            tasks.append((int(f), int(w["bits"][f]), seq, soff))
        by_f = {t[0]: t for t in tasks}
        checked_reads = checked_bits = 0
        for f, obits, ohits in pool.query(tasks):
            rs = sample[owner == f]
            seq = by_f[f][2]
            assert np.array_equal(ghits[rs], ohits), f"hits of filter {f}"
            got = bits_at(gbits, ranges(off, rs))
            assert np.array_equal(got, unpack(obits, seq.size)), f"answer bits of filter {f}"
            checked_reads += rs.size
            checked_bits += seq.size
        assert checked_reads == sample.size
        assert checked_reads >= n_reads // 100
        assert int(ghits[sample].sum()) > 0
    finally:
        pool.close()
        batch.close()
        for f in filters:
            f.close()


# ---------------------------------------------------------------------------
# served: 3.1 Gbp genome in a 4 GiB filter, a sample of the request pool
# ---------------------------------------------------------------------------
def served_request(genome, i):
    """Request i of the served workload's pool: log-uniform 1 kb-10 Mbp of
    150 bp reads with 1% errors (the benchmark's pool uses the same seeds)."""
    sz = np.exp(np.log(1e3) + synth.uniform01(9, 1, i, 1)[0] * (np.log(1e7) - np.log(1e3)))
    n = max(1, int(sz) // 150)
    return synth.sample_reads(genome, n, 150, 0.01, seed=5000 + i)


def test_served_4gib_full_size(tmp_path):
    from oracle_fullsize import BigFilter, compare_in_chunks, workers_for
    from paper_2606_24417_gb300.sbf import FilterServer, SuperBloomFilter

    bits = 1 << 35
    genome = synth.human_like_genome(3_100_000_000, seed=5)
    fbytes = bits // 8
    # host memory: one oracle filter per worker, next to the device filter's
    # copy, the accumulator, the genome and its memory-mapped file
    workers = workers_for(fbytes + (1 << 28), reserve=2 * fbytes + 2 * genome.size + (12 << 30))
    if workers < 2:
        pytest.skip("host memory holds fewer than two 4 GiB oracle filters")

    f = SuperBloomFilter(K, M, S, H, bits, shard_bits=B)
    dg = dev(genome)
    f.insert(dg, dev_off(np.array([0, genome.size], dtype=np.uint64)))
    torch.cuda.synchronize()
    del dg
    gpu_words = f.words()

    big = BigFilter(PARAMS, bits, genome, tmp_path, workers)
    try:
        big.insert()
        bad = compare_in_chunks(gpu_words, big.words())
        assert not bad, f"4 GiB filter differs from the oracle in chunks {bad[:5]}"
        del gpu_words

        # a seeded sample of the pool's 200 requests
        picks = np.unique(synth.randint(9, 2, 24, 0, 200))
        reqs = [served_request(genome, int(i)) for i in picks]
        srv = FilterServer(f, read_budget_bytes=1 << 30, max_inflight=3)
        alone = []
        for seq, off in reqs:
            hits, qb, _ = srv.wait(srv.submit(seq, off, want_bits=True), 120)
            alone.append((hits.copy(), qb.copy()))
        mix = [None] * len(reqs)

        def client(idx):
            tickets = list(zip(idx, srv.submit_many([reqs[i] for i in idx], want_bits=True)))
            for i, t in tickets:
                hits, qb, _ = srv.wait(t, 120)
                mix[i] = (hits.copy(), qb.copy())

        ths = [threading.Thread(target=client, args=(list(range(c, len(reqs), 4)),))
               for c in range(4)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        assert srv.stats()["launches"] < 2 * len(reqs)   # the mix was coalesced
        srv.close()
        for i, (seq, off) in enumerate(reqs):
            db, dh = f.query(dev(seq), dev_off(off))
            direct = (dh.cpu().numpy().view(np.uint32), db.cpu().numpy().view(np.uint32))
            for got in (alone[i], mix[i]):
                assert np.array_equal(got[0], direct[0]) and np.array_equal(got[1], direct[1]), i

        tasks = [(i, seq, off) for i, (seq, off) in enumerate(reqs)]
        checked = 0
        for i, obits, ohits in big.query(tasks, workers=min(workers, len(tasks))):
            assert np.array_equal(alone[i][0], ohits), f"hits of request {picks[i]}"
            assert np.array_equal(alone[i][1], obits), f"answer bits of request {picks[i]}"
            checked += 1
        assert checked == len(reqs)
        assert sum(int(a[0].sum()) for a in alone) > 0
    finally:
        big.close()
        f.close()
