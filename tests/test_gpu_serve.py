"""Serving loop: continuous batching around a resident filter.  Each request's
answers are the same alone, in a concurrent mix and from a direct query."""
import threading

import numpy as np
import pytest

from oracle import OracleSBF
from paper_2606_24417_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def served():
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    g = synth.bacterial_genome(3_000_000, seed=21)
    f = SuperBloomFilter(31, 16, 28, 4, 1 << 26)
    f.insert(torch.from_numpy(g).cuda(),
             torch.from_numpy(np.array([0, g.size], dtype=np.int64)).cuda())
    o = OracleSBF(31, 16, 28, 4, 1 << 26)
    o.insert(g, np.array([0, g.size], dtype=np.uint64))
    # requests of 1 kb - 400 kb of 150 bp reads, half sampled with 1% errors
    sizes = np.exp(np.log(1000) + synth.uniform01(22, 1, 0, 40) * (np.log(400_000) - np.log(1000)))
    reqs = []
    for i, sz in enumerate(sizes):
        n = max(1, int(sz) // 150)
        if i % 2:
            seq, off = synth.sample_reads(g, n, 150, 0.01, seed=100 + i)
        else:
            seq, off = synth.random_reads(n, 150, seed=200 + i)
        reqs.append((seq, off))
    return f, o, g, reqs


def _direct(f, seq, off):
    b, h = f.query(torch.from_numpy(seq).cuda(), torch.from_numpy(off.astype(np.int64)).cuda())
    return b.cpu().numpy().view(np.uint32), h.cpu().numpy().view(np.uint32)


def test_alone_equals_mix_equals_direct(served):
    from paper_2606_24417_gb300.sbf import FilterServer

    f, o, g, reqs = served
    srv = FilterServer(f, read_budget_bytes=16 << 20, max_inflight=3)
    alone = []
    for seq, off in reqs:
        t = srv.submit(seq, off, want_bits=True)
        hits, bits, lat = srv.wait(t, 60)
        assert lat >= 0
        alone.append((hits.copy(), bits.copy()))
    # the same requests submitted together from four client threads
    mix = [None] * len(reqs)

    def client(idx):
        # each client queues its share in one call, so the worker finds several
        # requests waiting and serves them together
        tickets = list(zip(idx, srv.submit_many([reqs[i] for i in idx], want_bits=True)))
        for i, t in tickets:
            hits, bits, _ = srv.wait(t, 60)
            mix[i] = (hits.copy(), bits.copy())

    ths = [threading.Thread(target=client, args=(list(range(c, len(reqs), 4)),)) for c in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    st = srv.stats()
    assert st["completed"] == 2 * len(reqs)
    assert st["launches"] < 2 * len(reqs)          # the mix was coalesced
    assert 0 < st["p50_s"] <= st["p99_s"]
    for i, (seq, off) in enumerate(reqs):
        db, dh = _direct(f, seq, off)
        assert np.array_equal(alone[i][0], dh) and np.array_equal(alone[i][1], db), i
        assert np.array_equal(mix[i][0], dh) and np.array_equal(mix[i][1], db), i
    for i in (0, 1, 7):
        ob, oh = o.query(*reqs[i])
        assert np.array_equal(alone[i][0], oh) and np.array_equal(alone[i][1], ob)
    srv.close()


def test_admission_by_memory(served):
    from paper_2606_24417_gb300.sbf import FilterServer, SbfError

    f, _, _, reqs = served
    big = [(s, o) for s, o in reqs if 100_000 < s.size < 450_000][:6]
    srv = FilterServer(f, read_budget_bytes=1 << 20, max_inflight=2)  # a few requests at a time
    tickets = [srv.submit(s, o) for s, o in big]
    for (s, o), t in zip(big, tickets):
        hits, _, _ = srv.wait(t, 60)
        assert np.array_equal(hits, _direct(f, s, o)[1])
    huge = synth.random_reads(20_000, 150, seed=5)          # 3 MB > 1 MB budget
    with pytest.raises(SbfError) as ei:
        srv.submit(*huge)
    assert ei.value.code == -1
    srv.close()


def test_bounded_wait(served):
    from paper_2606_24417_gb300.sbf import FilterServer, SbfError

    f, _, _, reqs = served
    srv = FilterServer(f, read_budget_bytes=8 << 20, max_inflight=1)
    seq, off = max(reqs, key=lambda r: r[0].size)
    t = srv.submit(seq, off)
    try:
        srv.wait(t, 0.0)
    except SbfError as e:
        assert e.code == -5      # timed out, the request stays queued
        hits, _, _ = srv.wait(t, 60)
        assert np.array_equal(hits, _direct(f, seq, off)[1])
    srv.close()


def test_large_filter_served_equals_direct():
    """A 1 GiB filter is served by the bulk-copy query kernels: every request's
    answers equal a direct query's (checked against the oracle elsewhere) and
    no wait ran out."""
    from paper_2606_24417_gb300.sbf import FilterServer, SuperBloomFilter

    g = synth.bacterial_genome(2_000_000, seed=23)
    f = SuperBloomFilter(31, 16, 28, 4, 1 << 33)
    f.insert(torch.from_numpy(g).cuda(),
             torch.from_numpy(np.array([0, g.size], dtype=np.int64)).cuda())
    reqs = []
    for i in range(12):
        n = 50 + 700 * i
        if i % 2:
            reqs.append(synth.sample_reads(g, n, 150, 0.01, seed=300 + i))
        else:
            reqs.append(synth.random_reads(n, 150, seed=400 + i))
    srv = FilterServer(f, read_budget_bytes=16 << 20, max_inflight=3)
    tickets = [srv.submit(seq, off, want_bits=True) for seq, off in reqs]
    for (seq, off), t in zip(reqs, tickets):
        hits, bits, _ = srv.wait(t, 60)
        db, dh = _direct(f, seq, off)
        assert np.array_equal(hits, dh) and np.array_equal(bits, db)
    assert f.device_status() == 0
    srv.close()
    f.close()


def test_staged_and_in_place_inputs_and_batch_submission(served):
    """The same requests through a server that copies every input into its
    read arena, through one that reads host memory in place where the device
    can (pinned buffers always; pageable buffers when the device reads them
    through the host's page tables), and submitted all in one call: identical
    answers, equal to direct queries."""
    from paper_2606_24417_gb300.sbf import FilterServer

    f, _, _, reqs = served
    pinned = []
    for seq, off in reqs[:12]:
        ps = torch.from_numpy(seq).pin_memory().numpy()
        po = torch.from_numpy(off.view(np.int64)).pin_memory().numpy().view(np.uint64)
        pinned.append((ps, po))
    results = {}
    for name, stage, rq in (("staged", True, reqs), ("in_place", False, reqs),
                            ("pinned", False, pinned)):
        srv = FilterServer(f, read_budget_bytes=16 << 20, max_inflight=3, stage_inputs=stage)
        tickets = srv.submit_many(rq, want_bits=True)
        results[name] = [srv.wait(t, 60)[:2] for t in tickets]
        info = srv.breakdown()
        if stage:
            assert info["direct_requests"] == 0 and info["staged_requests"] == len(rq)
        if name == "pinned":   # page-locked memory is always read in place
            assert info["direct_requests"] == len(rq)
            # also when submitted from a thread that made no CUDA call before
            srv.reset_stats()
            out = []
            th = threading.Thread(target=lambda: out.extend(srv.submit_many(rq[:3])))
            th.start()
            th.join()
            for t in out:
                srv.wait(t, 60)
            assert srv.breakdown()["direct_requests"] == 3
        assert all(v >= 0 for v in info["p99_s"].values())
        srv.close()
    for i, (seq, off) in enumerate(reqs):
        db, dh = _direct(f, seq, off)
        for name in results:
            if i < len(results[name]):
                hits, bits = results[name][i]
                assert np.array_equal(hits, dh) and np.array_equal(bits, db), (name, i)


def test_batch_submission_refuses_all_or_nothing(served):
    from paper_2606_24417_gb300.sbf import FilterServer, SbfError

    f, _, _, reqs = served
    srv = FilterServer(f, read_budget_bytes=1 << 20, max_inflight=2)
    bad_off = reqs[1][1].copy()
    bad_off[1], bad_off[2] = bad_off[2], bad_off[1]        # offsets decrease
    with pytest.raises(SbfError) as ei:
        srv.submit_many([reqs[0], (reqs[1][0], bad_off)])
    assert ei.value.code == -1
    assert srv.stats()["completed"] == 0
    t = srv.submit_many([reqs[0]])
    hits, _, _ = srv.wait(t[0], 60)
    assert np.array_equal(hits, _direct(f, *reqs[0])[1])
    srv.close()
