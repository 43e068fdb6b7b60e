"""Batched scheduling: many filters in one persistent launch (and under a CUDA
graph) give exactly the bits of one launch per filter and of the oracle."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_off(off):
    return dev(np.asarray(off, dtype=np.uint64).astype(np.int64))


def unpack(bits_u32, n):
    return np.unpackbits(np.ascontiguousarray(bits_u32).view(np.uint8), bitorder="little")[:n]


PARAMS = [(31, 16, 28, 4, 512, True), (31, 20, 24, 8, 256, True), (31, 14, 26, 2, 512, False)]


@pytest.fixture(scope="module")
def workload():
    return synth.batched_workload(n_filters=12, exp_lo=14, exp_hi=21, genome_lo=20_000,
                                  genome_hi=400_000, n_reads=6000, seed=5, read_cap=30_000)


def _filters(params, bits):
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    k, m, s, H, B, canon = params
    return [SuperBloomFilter(k, m, s, H, b, shard_bits=B, canonical=canon) for b in bits]


@pytest.mark.parametrize("hits_pass", [True, False], ids=["hits_pass", "hits_in_kernel"])
@pytest.mark.parametrize("params", PARAMS, ids=lambda p: "_".join(map(str, p)))
def test_batched_insert_and_query_match_oracle(params, workload, hits_pass, monkeypatch):
    """hits_pass: the persistent launch leaves reads of at most 2048 positions
    to the short-read hit pass (forced onto this small batch by its knob);
    one launch per filter counts every read in the kernel either way."""
    from paper_2606_24417_gb300.sbf import BATCH_FUSED, BATCH_GRAPH, BATCH_PER_FILTER, FilterBatch

    if hits_pass:
        monkeypatch.setenv("SBF_HITS_PASS_MIN_POSITIONS", "0")
    else:
        monkeypatch.delenv("SBF_HITS_PASS_MIN_POSITIONS", raising=False)

    w = workload
    k, m, s, H, B, canon = params
    filters = _filters(params, w["bits"])
    batch = FilterBatch(filters)
    batch.insert(dev(w["gseq"]), dev_off(w["goff"]), w["goff"], w["ggroup"], mode=BATCH_GRAPH)
    oracles = []
    for f, g in enumerate(w["genomes"]):
        o = OracleSBF(k, m, s, H, w["bits"][f], shard_bits=B, canonical=canon)
        o.insert(g, np.array([0, g.size], dtype=np.uint64))
        assert np.array_equal(filters[f].words(), o.words()), f
        oracles.append(o)

    dseq, doff = dev(w["seq"]), dev_off(w["off"])
    outs = {}
    for mode in (BATCH_PER_FILTER, BATCH_FUSED, BATCH_GRAPH, BATCH_GRAPH):
        b_, h_ = batch.query(dseq, doff, w["off"], w["group"], mode=mode)
        outs.setdefault(mode, []).append((b_.cpu().numpy().view(np.uint32).copy(),
                                          h_.cpu().numpy().view(np.uint32).copy()))
    ref_bits, ref_hits = outs[BATCH_PER_FILTER][0]
    for mode, runs in outs.items():
        for bits, hits in runs:
            assert np.array_equal(bits, ref_bits) and np.array_equal(hits, ref_hits), mode

    # against the oracle, filter by filter
    ub = unpack(ref_bits, w["seq"].size)
    for f, o in enumerate(oracles):
        a, b = int(w["group"][f]), int(w["group"][f + 1])
        if a == b:
            continue
        p0, p1 = int(w["off"][a]), int(w["off"][b])
        oseq = w["seq"][p0:p1]
        ooff = w["off"][a:b + 1] - np.uint64(p0)
        obits, ohits = o.query(oseq, ooff)
        assert np.array_equal(ub[p0:p1], unpack(obits, p1 - p0)), f
        assert np.array_equal(ref_hits[a:b], ohits), f


def test_schedules_and_tuning_keep_the_bits(workload):
    from paper_2606_24417_gb300.sbf import BATCH_FUSED, BATCH_GRAPH, FilterBatch

    w = workload
    filters = _filters(PARAMS[0], w["bits"])
    batch = FilterBatch(filters)
    batch.insert(dev(w["gseq"]), dev_off(w["goff"]), w["goff"], w["ggroup"], mode=BATCH_FUSED)
    words = [f.words() for f in filters]
    dseq, doff = dev(w["seq"]), dev_off(w["off"])
    ref = None
    for sched in [(False, 1, 0), (True, 1, 0), (True, 7, 0), (True, 3, 5), (False, 1, 3)]:
        batch.set_schedule(*sched)
        assert batch.schedule() == sched
        b_, h_ = batch.query(dseq, doff, w["off"], w["group"], mode=BATCH_GRAPH)
        cur = (b_.cpu().numpy().copy(), h_.cpu().numpy().copy())
        if ref is None:
            ref = cur
        assert np.array_equal(cur[0], ref[0]) and np.array_equal(cur[1], ref[1]), sched
    ms = batch.tune(dseq, doff, w["off"], w["group"])
    assert ms > 0
    b_, h_ = batch.query(dseq, doff, w["off"], w["group"], mode=BATCH_GRAPH)
    assert np.array_equal(b_.cpu().numpy(), ref[0]) and np.array_equal(h_.cpu().numpy(), ref[1])
    # re-inserting with a tuned insert schedule changes no bit
    batch.tune(dev(w["gseq"]), dev_off(w["goff"]), w["goff"], w["ggroup"], insert=True)
    for f, wd in zip(filters, words):
        assert np.array_equal(f.words(), wd)


def test_graph_replay_sees_new_input(workload):
    from paper_2606_24417_gb300.sbf import BATCH_GRAPH, BATCH_PER_FILTER, FilterBatch

    w = workload
    filters = _filters(PARAMS[0], w["bits"])
    batch = FilterBatch(filters)
    batch.insert(dev(w["gseq"]), dev_off(w["goff"]), w["goff"], w["ggroup"], mode=BATCH_GRAPH)
    dseq, doff = dev(w["seq"]), dev_off(w["off"])
    b1, h1 = batch.query(dseq, doff, w["off"], w["group"], mode=BATCH_GRAPH)
    first = h1.cpu().numpy().copy()
    dseq.copy_(dev(synth.uniform_dna(w["seq"].size, 99)))  # same buffer, new reads
    b2, h2 = batch.query(dseq, doff, w["off"], w["group"], bits=b1, hits=h1, mode=BATCH_GRAPH)
    b3, h3 = batch.query(dseq, doff, w["off"], w["group"], mode=BATCH_PER_FILTER)
    assert torch.equal(b2, b3) and torch.equal(h2, h3)
    assert not np.array_equal(first, h2.cpu().numpy())
