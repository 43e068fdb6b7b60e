"""The allocation-free batched query (sbf_batch_query_noalloc), for callers that
cannot call cudaMalloc: its scratch is a fixed array inside the library.  Two
calls in a row through the C ABI must give exactly what the batch entry point
gives (the same integer answers, so the tolerance is zero).  Kept in a file
collected last so that a run stopping at the first failure has run every
other test before it; self-contained, so it also passes alone."""
import numpy as np
import pytest

from paper_2606_24417_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_batch_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    from paper_2606_24417_gb300.sbf import (BATCH_FUSED, FilterBatch, SbfError,
                                            SuperBloomFilter, batch_query_noalloc)

    w = synth.batched_workload(n_filters=9, exp_lo=15, exp_hi=21, genome_lo=30_000,
                               genome_hi=300_000, n_reads=5000, seed=17, read_cap=20_000)
    filters = [SuperBloomFilter(31, 16, 28, 4, b) for b in w["bits"]]
    batch = FilterBatch(filters)
    batch.insert(torch.from_numpy(w["gseq"]).cuda(),
                 torch.from_numpy(w["goff"].astype(np.int64)).cuda(), w["goff"], w["ggroup"],
                 mode=BATCH_FUSED)
    dseq = torch.from_numpy(w["seq"]).cuda()
    doff = torch.from_numpy(w["off"].astype(np.int64)).cuda()
    want_bits, want_hits = batch.query(dseq, doff, w["off"], w["group"], mode=BATCH_FUSED)
    torch.cuda.synchronize()
    assert int(want_hits.sum()) > 0
    bits = torch.full_like(want_bits, -1)   # stale contents must not leak into the answers
    hits = torch.full_like(want_hits, -1)
    for _ in range(2):                      # the shared scratch keeps the last call's contents
        batch_query_noalloc(filters, dseq, doff, w["off"], w["group"], bits, hits)
        torch.cuda.synchronize()
        assert torch.equal(bits, want_bits)
        assert torch.equal(hits, want_hits)
    # more filters than the fixed scratch holds are refused with a clear error
    many = [filters[0]] * 513
    group = np.zeros(514, dtype=np.uint64)
    group[1:] = w["off"].size - 1
    with pytest.raises(SbfError) as ei:
        batch_query_noalloc(many, dseq, doff, w["off"], group, bits, hits)
    assert ei.value.code == -1 and "at most 512" in str(ei.value)


def test_noalloc_with_a_large_filter():
    """A batch holding a 1 GiB filter takes the bulk-copy kernels; the
    allocation-free entry point still equals the batch entry point."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    from paper_2606_24417_gb300.sbf import (BATCH_FUSED, FilterBatch, SuperBloomFilter,
                                            batch_query_noalloc)

    w = synth.batched_workload(n_filters=3, exp_lo=15, exp_hi=21, genome_lo=200_000,
                               genome_hi=600_000, n_reads=6000, seed=19, read_cap=20_000)
    bits_of = [1 << 33] + list(w["bits"][1:])
    filters = [SuperBloomFilter(31, 16, 28, 4, b) for b in bits_of]
    batch = FilterBatch(filters)
    batch.insert(torch.from_numpy(w["gseq"]).cuda(),
                 torch.from_numpy(w["goff"].astype(np.int64)).cuda(), w["goff"], w["ggroup"],
                 mode=BATCH_FUSED)
    dseq = torch.from_numpy(w["seq"]).cuda()
    doff = torch.from_numpy(w["off"].astype(np.int64)).cuda()
    want_bits, want_hits = batch.query(dseq, doff, w["off"], w["group"], mode=BATCH_FUSED)
    bits = torch.full_like(want_bits, -1)
    hits = torch.full_like(want_hits, -1)
    batch_query_noalloc(filters, dseq, doff, w["off"], w["group"], bits, hits)
    torch.cuda.synchronize()
    assert int(want_hits.sum()) > 0
    assert torch.equal(bits, want_bits) and torch.equal(hits, want_hits)
    assert all(f.device_status() == 0 for f in filters)
    batch.close()
    for f in filters:
        f.close()


def test_noalloc_table_of_many_filters_with_empty_groups():
    """130 filters (more than one table-writing launch of 32 entries) with a
    few reads each, so several filters get no reads at all: the table
    entries after the first launch and their iteration ranges must line up
    with the batch entry point's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    from paper_2606_24417_gb300.sbf import (BATCH_FUSED, FilterBatch, SbfError,
                                            SuperBloomFilter, batch_query_noalloc)

    w = synth.batched_workload(n_filters=130, exp_lo=14, exp_hi=17, genome_lo=5_000,
                               genome_hi=40_000, n_reads=300, seed=23, read_cap=5_000)
    sizes = np.diff(w["group"].astype(np.int64))
    assert (sizes == 0).sum() >= 3 and (sizes > 0).sum() >= 100
    filters = [SuperBloomFilter(31, 16, 28, 4, b) for b in w["bits"]]
    batch = FilterBatch(filters)
    batch.insert(torch.from_numpy(w["gseq"]).cuda(),
                 torch.from_numpy(w["goff"].astype(np.int64)).cuda(), w["goff"], w["ggroup"],
                 mode=BATCH_FUSED)
    dseq = torch.from_numpy(w["seq"]).cuda()
    doff = torch.from_numpy(w["off"].astype(np.int64)).cuda()
    want_bits, want_hits = batch.query(dseq, doff, w["off"], w["group"], mode=BATCH_FUSED)
    torch.cuda.synchronize()
    assert int(want_hits.sum()) > 0
    bits = torch.full_like(want_bits, -1)
    hits = torch.full_like(want_hits, -1)
    for _ in range(2):
        batch_query_noalloc(filters, dseq, doff, w["off"], w["group"], bits, hits)
        torch.cuda.synchronize()
        assert torch.equal(bits, want_bits) and torch.equal(hits, want_hits)
    # short output or group arrays are refused before anything reaches the device
    with pytest.raises(SbfError):
        batch_query_noalloc(filters, dseq, doff, w["off"], w["group"][:-1], bits, hits)
    with pytest.raises(SbfError):
        batch_query_noalloc(filters, dseq, doff, w["off"], w["group"], bits[:1], hits)
    batch.close()
    for f in filters:
        f.close()
