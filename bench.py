"""Benchmark: Super Bloom filter insert + query on the bacterial-genome workload.

One step = clear the 2^30-bit filter, insert a 100 Mbp synthetic genome, then
query 20M 150 bp reads (10M sampled from the genome with 1% errors, 10M
random) -- the whole hot path, inputs resident in HBM.  value = (inserted +
queried k-mer positions) / time.  `e2e` repeats the step through the host
entry points of the C ABI (pinned host buffers, copies inside the timed
region).  The CPU oracle runs on a bounded sample as the reported baseline;
`--impl reference` times the oracle alone (there is no runnable reference
code for this paper).

Under torchrun each rank builds its own filter replica and queries its own
20M reads (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "insert/query k-mers/s (k=31,s=28,m=16,H=4), % HBM sector roofline; served p99"
K, M, S, H = 31, 16, 28, 4
FILTER_BITS = 1 << 30
SHARD_BITS = 512
GENOME_BP = 100_000_000
N_SAMPLED = 10_000_000
N_RANDOM = 10_000_000
READ_LEN = 150
WORKLOAD = ("bacterial-genome-shaped: insert a 100 Mbp order-3 Markov genome (GC 50%, 3% "
            "1-10 kb exact repeats) into a 2^30-bit filter of 512-bit shards; query 10M 150 bp "
            "reads sampled from it (1% substitutions, both strands) + 10M random 150 bp reads")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    job's time).  Ranks are independent filter replicas working on their own
    reads; this reduction of a few floats is the only cross-rank traffic."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def rank_read_seed(rank: int) -> int:
    """Seed of a rank's query reads: every rank queries its own batch (weak scaling)."""
    return 3 + 1000 * rank


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_workload(rank: int, small: bool = False):
    from paper_2606_24417_gb300 import synth

    t = time.time()
    genome = synth.bacterial_genome(GENOME_BP, seed=2)
    n_s, n_r = (N_SAMPLED // 10, N_RANDOM // 10) if small else (N_SAMPLED, N_RANDOM)
    reads, roff = synth.mixed_query_reads(genome, n_s, n_r, READ_LEN, 0.01,
                                          seed=rank_read_seed(rank))
    log(f"[bench] rank {rank}: workload generated in {time.time() - t:.1f}s")
    return genome, reads, roff


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("sbf_fused.cuh", "sbf_device.cuh")


def kernel_source_digest() -> str:
    """Digest of the fused kernels' sources (what the ncu traffic was taken on)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_24417_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_counter(kernel: str, key: str):
    """A per-launch ncu counter from the committed summary, if it was taken on
    the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(kernel)
    if not e or e.get("source_digest") != kernel_source_digest():
        return None
    return e.get(key)


def profiled_traffic(kernel: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return profiled_counter(kernel, "dram_bytes_per_launch")


def sector_bandwidth(dev, stream, buf_bytes: int, sector_bytes: int, rmw: bool, n: int,
                     reps: int = 5):
    """Median GB/s of the random-sector probe (n sectors per launch) over a
    buffer of buf_bytes: loaded bytes for a gather, read + written bytes for a
    read-modify-write."""
    import torch

    from paper_2606_24417_gb300.sbf import probe_sectors

    buf = torch.zeros(buf_bytes, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    for r in range(2):
        probe_sectors(buf, sector_bytes, n, seed=r, rmw=rmw, sink=sink, stream=stream)
    ms = []
    for r in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        probe_sectors(buf, sector_bytes, n, seed=100 + r, rmw=rmw, sink=sink, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    del buf
    moved = n * sector_bytes * (2 if rmw else 1)
    return moved / (statistics.median(ms) / 1e3) / 1e9


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def _read_sample(reads, roff, n_reads):
    """n_reads reads, half from the sampled and half from the random part."""
    n_all = roff.size - 1
    h = n_reads // 2
    parts = [(0, h), (n_all // 2, n_all // 2 + (n_reads - h))]
    seq = np.concatenate([reads[int(roff[a]):int(roff[b])] for a, b in parts])
    lens = np.concatenate([np.diff(roff[a:b + 1].astype(np.int64)) for a, b in parts])
    off = np.zeros(lens.size + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    return seq, off


def cpu_baseline(genome, reads, roff, budget_s: float = 15.0):
    """The oracle on the host: one core, and all cores through one process per
    core (sliced inserts OR-merged, read chunks in parallel)."""
    import tempfile

    from oracle import OracleSBF
    from oracle.parallel import OraclePool

    def single(n_gen, n_reads):
        f = OracleSBF(K, M, S, H, FILTER_BITS, shard_bits=SHARD_BITS)
        g = genome[:n_gen]
        q, qo = _read_sample(reads, roff, n_reads)
        t = time.perf_counter()
        f.insert(g, np.array([0, g.size], dtype=np.uint64))
        f.query(q, qo)
        dt = time.perf_counter() - t
        return (g.size - K + 1) + n_reads * (READ_LEN - K + 1), dt

    k1, t1 = single(1_000_000, 20_000)
    one = {"value": k1 / t1, "cores": 1,
           "sample": f"1 Mbp inserted, 20,000 reads queried ({k1} k-mer positions, {t1:.1f} s)"}
    pool = OraclePool(K, M, S, H, FILTER_BITS, shard_bits=SHARD_BITS, canonical=True)
    try:
        with tempfile.TemporaryDirectory(prefix="sbf_cpu_") as d:
            gp, wp = os.path.join(d, "g.npy"), os.path.join(d, "w.npy")
            qp, op = os.path.join(d, "q.npy"), os.path.join(d, "o.npy")
            np.save(gp, genome)
            t = time.perf_counter()
            words = pool.insert(gp, genome.size, d)
            np.save(wp, words)
            t_ins = time.perf_counter() - t
            # size the read sample by a calibration run so that the query
            # takes what is left of budget_s
            n_cal = 100_000
            q, qo = _read_sample(reads, roff, n_cal)
            np.save(qp, q)
            np.save(op, qo)
            t = time.perf_counter()
            pool.query_hits(wp, qp, op, n_cal)
            per_read = (time.perf_counter() - t) / n_cal
            n_reads = int(min(roff.size - 1, max(n_cal, (budget_s - t_ins) / per_read)))
            q, qo = _read_sample(reads, roff, n_reads)
            np.save(qp, q)
            np.save(op, qo)
            t = time.perf_counter()
            pool.query_hits(wp, qp, op, n_reads)
            dt = t_ins + (time.perf_counter() - t)
    finally:
        pool.close()
    kmers = (genome.size - K + 1) + n_reads * (READ_LEN - K + 1)
    return {"value": kmers / dt, "unit": "k-mers/s", "cores": pool.workers, "kind": "oracle",
            "sample": f"insert the whole {genome.size} bp genome, then query {n_reads} reads (half "
                      f"sampled, half random; {kmers} k-mer positions) in {dt:.1f} s with "
                      f"{pool.workers} single-threaded C oracles (one process per core: "
                      f"genome slices OR-merged, read chunks in parallel)",
            "single_core": one}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import tempfile

    from oracle.parallel import OraclePool

    genome, reads, roff = make_workload(0)
    n_reads = 1_000_000
    times = []
    pool = OraclePool(K, M, S, H, FILTER_BITS, shard_bits=SHARD_BITS, canonical=True)
    try:
        with tempfile.TemporaryDirectory(prefix="sbf_ref_") as d:
            gp, wp = os.path.join(d, "g.npy"), os.path.join(d, "w.npy")
            qp, op = os.path.join(d, "q.npy"), os.path.join(d, "o.npy")
            np.save(gp, genome)
            q, qo = _read_sample(reads, roff, n_reads)
            np.save(qp, q)
            np.save(op, qo)
            for i in range(args.warmup + args.steps):
                t = time.perf_counter()
                words = pool.insert(gp, genome.size, d)
                np.save(wp, words)
                pool.query_hits(wp, qp, op, n_reads)
                dt = time.perf_counter() - t
                if i >= args.warmup:
                    times.append(dt)
    finally:
        pool.close()
    kmers_step = (genome.size - K + 1) + n_reads * (READ_LEN - K + 1)
    total = sum(times)
    value = kmers_step * len(times) / total
    sample = (f"each step inserts the whole {genome.size} bp genome and queries {n_reads} reads "
              f"(half sampled, half random; {kmers_step} k-mer positions) with {pool.workers} "
              f"single-threaded C oracles, one process per core (genome slices OR-merged, read "
              f"chunks in parallel)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "k-mers/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "k": K, "m": M, "s": S, "H": H,
                       "filter_bits": FILTER_BITS, "shard_bits": SHARD_BITS},
            "cpu_baseline": {"value": value, "unit": "k-mers/s", "cores": pool.workers,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "k-mers/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2606_24417_gb300 import build_lib
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    build_lib.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

    genome, reads, roff = make_workload(rank, small=args.case == "small")
    n_reads = roff.size - 1
    goff = np.array([0, genome.size], dtype=np.uint64)
    ins_kmers = genome.size - K + 1
    q_kmers = n_reads * (READ_LEN - K + 1)
    kmers_step = ins_kmers + q_kmers

    d_genome = torch.from_numpy(genome).to(dev)
    d_goff = torch.from_numpy(goff.astype(np.int64)).to(dev)
    d_reads = torch.from_numpy(reads).to(dev)
    d_roff = torch.from_numpy(roff.astype(np.int64)).to(dev)
    d_bits = torch.empty((reads.size + 31) // 32, dtype=torch.int32, device=dev)
    d_hits = torch.empty(n_reads, dtype=torch.int32, device=dev)
    stats = torch.zeros(3, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    filter_bits = 1 << args.filter_log2
    f = SuperBloomFilter(K, M, S, H, filter_bits, shard_bits=SHARD_BITS)
    stream = torch.cuda.current_stream()

    # super-k-mer runs of the query batch (shard loads the method needs)
    f.clear()
    f.insert(d_genome, d_goff)
    f.query(d_reads, d_roff, bits=d_bits, hits=d_hits, stats=stats)
    torch.cuda.synchronize()
    valid_q, runs_q, pos_q = (int(x) for x in stats.cpu().tolist())
    stats.zero_()
    f.query(d_genome, d_goff, want_bits=False, want_hits=False, stats=stats)
    torch.cuda.synchronize()
    valid_i, runs_i, _ = (int(x) for x in stats.cpu().tolist())

    def step(ev):
        f.clear()
        ev[0].record(stream)
        f.insert(d_genome, d_goff)
        ev[1].record(stream)
        f.query(d_reads, d_roff, bits=d_bits, hits=d_hits)
        ev[2].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step([torch.cuda.Event(enable_timing=True) for _ in range(3)])
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local_rank)
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(1)  # L2 flush between timed steps (outside the events)
        step(evs[i])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if rank == 0 else None
    t_ins = [evs[i][0].elapsed_time(evs[i][1]) for i in range(args.steps)]
    t_q = [evs[i][1].elapsed_time(evs[i][2]) for i in range(args.steps)]
    total_ms = sum(t_ins) + sum(t_q)
    total_ms, ins_ms_sum, q_ms_sum = max_over_ranks([total_ms, sum(t_ins), sum(t_q)], dist, dev)
    value = world * kmers_step * args.steps / (total_ms / 1e3)

    if args.skip_extras:
        if rank == 0:
            print(json.dumps({"case": args.case, "query_ms": sum(t_q) / args.steps,
                              "insert_ms": sum(t_ins) / args.steps, "value": value}), flush=True)
        return 0

    # ---- e2e through the host entry points (pinned host buffers) ----------
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8)).pin_memory().numpy().view(a.dtype)

    h_genome = pinned(genome)
    h_goff = pinned(goff)
    h_reads = pinned(reads)
    h_roff = pinned(roff)
    h_bits = torch.empty((reads.size + 31) // 32, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    h_hits = torch.empty(n_reads, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(1):
        f.clear()
        f.insert_host(h_genome, h_goff)
        f.query_host(h_reads, h_roff, h_bits, h_hits)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        f.clear()
        f.insert_host(h_genome, h_goff)
        f.query_host(h_reads, h_roff, h_bits, h_hits)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks([e2e_s], dist, dev)[0]
    # e2e answers equal the device-resident answers
    same = bool(np.array_equal(h_bits, d_bits.cpu().numpy().view(np.uint32)) and
                np.array_equal(h_hits, d_hits.cpu().numpy().view(np.uint32)))
    e2e_value = world * kmers_step * e2e_steps / e2e_s
    h2d = genome.nbytes + goff.nbytes + reads.nbytes + roff.nbytes
    d2h = h_bits.nbytes + h_hits.nbytes

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel (query) --------------------------
    peak, peak_kind = measured_peaks()
    q_ms = q_ms_sum / args.steps
    ins_ms = ins_ms_sum / args.steps
    # algorithmic bytes per query launch: read bytes + offsets, one shard load
    # per super-k-mer run, the bit-packed answers and the per-read hits
    q_bytes = reads.nbytes + roff.nbytes + runs_q * (SHARD_BITS // 8) + (reads.size + 7) // 8 + 4 * n_reads
    # insert: genome bytes + a read-modify-write of one shard per run
    i_bytes = genome.nbytes + runs_i * 2 * (SHARD_BITS // 8)
    dominant = "query" if q_ms >= ins_ms else "insert"
    d_bytes, d_ms = (q_bytes, q_ms) if dominant == "query" else (i_bytes, ins_ms)
    achieved = d_bytes / (d_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic(dominant) if filter_bits == FILTER_BITS else None,
                "kernel": dominant, "peak_kind": f"{peak_kind} (copy bandwidth)",
                "algorithmic_bytes_per_launch": d_bytes, "launch_ms": d_ms}
    # ---- shard part against the random-sector probe; issue-slot bound -----
    sector_b = SHARD_BITS // 8
    big = 1 << 30  # 1 GiB >= 4x L2: every probe access goes to DRAM
    filt = filter_bits // 8
    bw = {"gather_dram": sector_bandwidth(dev, stream, big, sector_b, False, 1 << 27),
          "gather_filter_size": sector_bandwidth(dev, stream, filt, sector_b, False, 1 << 27),
          "rmw_dram": sector_bandwidth(dev, stream, big, sector_b, True, 1 << 25),
          "rmw_filter_size": sector_bandwidth(dev, stream, filt, sector_b, True, 1 << 25)}
    q_stream = q_bytes - runs_q * sector_b
    i_stream = genome.nbytes

    def bound(kmers, stream_bytes, shard_bytes, shard_gbs):
        t = stream_bytes / (peak * 1e9) + shard_bytes / (shard_gbs * 1e9)
        return kmers / t

    q_rate, i_rate = q_kmers / (q_ms / 1e3), ins_kmers / (ins_ms / 1e3)
    sector_roofline = {
        "unit": "k-mers/s",
        "probe_gbs": bw,
        "sector_bytes": sector_b,
        "query": {"bound_dram": bound(q_kmers, q_stream, runs_q * sector_b, bw["gather_dram"]),
                  "bound_filter_size": bound(q_kmers, q_stream, runs_q * sector_b,
                                             bw["gather_filter_size"]),
                  "achieved": q_rate},
        "insert": {"bound_dram": bound(ins_kmers, i_stream, runs_i * 2 * sector_b, bw["rmw_dram"]),
                   "bound_filter_size": bound(ins_kmers, i_stream, runs_i * 2 * sector_b,
                                              bw["rmw_filter_size"]),
                   "achieved": i_rate},
        "note": "streamed bytes at the copy peak plus shard bytes at the probe's random-sector "
                "bandwidth; 'dram' probes a 1 GiB buffer, 'filter_size' a buffer the size of "
                "the filter (part of it stays in L2)",
    }
    for part in ("query", "insert"):
        e = sector_roofline[part]
        e["frac_dram"] = e["achieved"] / e["bound_dram"]
        e["frac_filter_size"] = e["achieved"] / e["bound_filter_size"]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    issue_peak = n_sm * 4 * sm_mhz * 1e6  # 4 schedulers per SM, one warp instruction per cycle
    inst = profiled_counter(dominant, "warp_inst_per_launch") if filter_bits == FILTER_BITS else None
    alu = {"bound": "alu", "unit": "warp instructions/s", "kernel": dominant,
           "peak": issue_peak, "peak_kind": f"{n_sm} SMs x 4 schedulers x 1 instr/cycle x "
                                            f"{sm_mhz:.0f} MHz (median SM clock sampled)",
           "warp_inst_per_launch": inst,
           "achieved": inst / (d_ms / 1e3) if inst else None,
           "frac": inst / (d_ms / 1e3) / issue_peak if inst else None}
    # the oracle baseline is taken on the headline filter only (a 2^34-bit
    # oracle would hold 2 GiB per host process)
    cpu = cpu_baseline(genome, reads, roff) if world == 1 and filter_bits == FILTER_BITS else None
    # the same workload on filters far beyond the 129 MB L2 (1 GiB and 4 GiB),
    # each against the random-sector roofline of a buffer of its own size
    sizes = None
    if world == 1 and filter_bits == FILTER_BITS:
        del f
        sizes = {}
        for e in (33, 35):
            row = measure_filter_size(e, args.steps, dev, stream, genome, reads, roff, d_genome,
                                      d_goff, d_reads, d_roff, d_bits, d_hits, flush)
            sizes[f"2^{e}"] = {k: row[k] for k in (
                "filter_bytes", "insert_kmers_per_s", "query_kmers_per_s", "insert_ms", "query_ms",
                "insert_frac", "query_frac", "probe_gather_gbs", "probe_rmw_gbs",
                "device_status")}
            log(f"[bench] 2^{e} bits: query {row['query_kmers_per_s'] / 1e9:.1f} G/s "
                f"({row['query_frac']:.3f} of its sector bound), insert "
                f"{row['insert_kmers_per_s'] / 1e9:.1f} G/s ({row['insert_frac']:.3f})")
        sizes["note"] = ("median of max(steps, 3) steps per size; frac = k-mers/s over streamed "
                         "bytes at the copy peak plus one shard per super-k-mer run at the "
                         "random-sector probe's rate over a buffer of the filter's size")
    # the served workload (its own genome, filter and request pool), so that
    # the line carries served throughput and p50 / p99 latency
    served = None
    if world == 1 and filter_bits == FILTER_BITS and not args.no_served:
        del d_genome, d_reads, d_bits, d_hits
        torch.cuda.empty_cache()
        served = served_measurement(n_poisson=400)
        served["note"] = ("3.1 Gbp human-shaped genome in a 2^35-bit filter; 200 requests of "
                          "1 kb-10 Mbp of 150 bp reads (1% errors) in pinned host memory; "
                          "backlogs of 400 requests, 400 Poisson arrivals per load")
    line = {
        "metric": METRIC, "value": value, "unit": "k-mers/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "k": K, "m": M, "s": S, "H": H,
                   "filter_bits": filter_bits, "shard_bits": SHARD_BITS,
                   "insert_kmers": ins_kmers, "query_kmers": q_kmers,
                   "l2": "inputs larger than L2 (3.0 GB of reads per step) and a 256 MB L2 "
                         "flush between timed steps"},
        "insert_kmers_per_s": world * ins_kmers / (ins_ms / 1e3),
        "query_kmers_per_s": world * q_kmers / (q_ms / 1e3),
        "insert_ms": ins_ms, "query_ms": q_ms,
        "runs_per_kmer": {"query": runs_q / max(valid_q, 1), "insert": runs_i / max(valid_i, 1)},
        "roofline": roofline,
        "sector_roofline": sector_roofline,
        "alu": alu,
        "e2e": {"value": e2e_value, "unit": "k-mers/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "answers_match_device": same},
        # per step: the insert kernel, the query kernel and its short-read hit pass
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "filter_sizes": sizes,
        "served": served,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# batched workload: 256 filters, one persistent launch vs one launch per filter
# ---------------------------------------------------------------------------
def run_batched(args):
    import torch

    from paper_2606_24417_gb300 import build_lib, synth
    from paper_2606_24417_gb300.sbf import (BATCH_FUSED, BATCH_GRAPH, BATCH_PER_FILTER,
                                            FilterBatch, SuperBloomFilter, num_kmers)

    build_lib.build()
    torch.cuda.set_device(0)
    t = time.time()
    w = synth.batched_workload(n_filters=256, n_reads=5_000_000, seed=4)
    log(f"[bench] batched workload generated in {time.time() - t:.1f}s: "
        f"{w['gseq'].size / 1e9:.2f} Gbp genomes, {w['seq'].size / 1e9:.2f} Gbp reads")
    filters = [SuperBloomFilter(K, M, S, H, b, shard_bits=SHARD_BITS) for b in w["bits"]]
    batch = FilterBatch(filters)
    dg, dgo = torch.from_numpy(w["gseq"]).cuda(), torch.from_numpy(w["goff"].astype(np.int64)).cuda()
    dq, dqo = torch.from_numpy(w["seq"]).cuda(), torch.from_numpy(w["off"].astype(np.int64)).cuda()
    bits = torch.empty((w["seq"].size + 31) // 32, dtype=torch.int32, device="cuda")
    hits = torch.empty(w["off"].size - 1, dtype=torch.int32, device="cuda")
    ins_kmers = num_kmers(w["goff"], K)
    q_kmers = num_kmers(w["off"], K)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    tuned_ins_ms = batch.tune(dg, dgo, w["goff"], w["ggroup"], insert=True)
    for name, mode in [("per_filter", BATCH_PER_FILTER), ("graph", BATCH_GRAPH)]:
        res[f"insert_ms_{name}"] = timed(
            lambda: batch.insert(dg, dgo, w["goff"], w["ggroup"], mode=mode), args.steps)
    tuned_ms = batch.tune(dq, dqo, w["off"], w["group"], bits=bits, hits=hits)
    answers = {}
    for name, mode in [("per_filter", BATCH_PER_FILTER), ("fused", BATCH_FUSED), ("graph", BATCH_GRAPH)]:
        res[f"query_ms_{name}"] = timed(
            lambda: batch.query(dq, dqo, w["off"], w["group"], bits=bits, hits=hits, mode=mode),
            args.steps)
        torch.cuda.synchronize()
        answers[name] = (bits.clone(), hits.clone())
    same = all(torch.equal(answers[n][0], answers["per_filter"][0]) and
               torch.equal(answers[n][1], answers["per_filter"][1]) for n in answers)
    # a small batch (every 500th read, 10,000 reads over the same 256 filters),
    # where launch overhead is a visible part of the call: per-filter
    # launches, one fused launch, and the fused launch replayed from a graph
    sel = np.arange(0, w["off"].size - 1, 500)
    owner = np.searchsorted(w["group"].astype(np.int64), sel, side="right") - 1
    s_len = np.diff(w["off"].astype(np.int64))[sel]
    s_seq = np.concatenate([w["seq"][int(w["off"][r]):int(w["off"][r + 1])] for r in sel])
    s_off = np.concatenate([[0], np.cumsum(s_len)]).astype(np.uint64)
    s_group = np.searchsorted(owner, np.arange(len(filters) + 1)).astype(np.uint64)
    dsq = torch.from_numpy(s_seq).cuda()
    dso = torch.from_numpy(s_off.astype(np.int64)).cuda()
    sb = torch.empty((s_seq.size + 31) // 32, dtype=torch.int32, device="cuda")
    sh = torch.empty(sel.size, dtype=torch.int32, device="cuda")
    small = {"reads": int(sel.size), "kmers": num_kmers(s_off, K)}
    for name, mode in [("per_filter", BATCH_PER_FILTER), ("fused", BATCH_FUSED), ("graph", BATCH_GRAPH)]:
        small[f"query_ms_{name}"] = timed(
            lambda: batch.query(dsq, dso, s_off, s_group, bits=sb, hits=sh, mode=mode), 50)
    dyn, chunk, grid = batch.schedule()
    idyn, ichunk, igrid = batch.schedule(insert=True)
    line = {"workload": "batched: 256 filters of 2^20-2^28 bits (log-uniform sizes) built from "
                        "1-50 Mbp uniform genomes (log-uniform), 5M reads of lognormal lengths "
                        "(median 150 bp, sigma 1.5, cap 100 kb), half sampled with 1% errors",
            "insert_kmers": ins_kmers, "query_kmers": q_kmers,
            **{k: v for k, v in res.items()},
            "query_kmers_per_s_graph": q_kmers / (res["query_ms_graph"] / 1e3),
            "query_kmers_per_s_per_filter": q_kmers / (res["query_ms_per_filter"] / 1e3),
            "insert_kmers_per_s_graph": ins_kmers / (res["insert_ms_graph"] / 1e3),
            "insert_kmers_per_s_per_filter": ins_kmers / (res["insert_ms_per_filter"] / 1e3),
            "tuned_schedule": {"query": {"dynamic": dyn, "chunk": chunk, "grid_blocks": grid,
                                         "tuned_ms": tuned_ms},
                               "insert": {"dynamic": idyn, "chunk": ichunk, "grid_blocks": igrid,
                                          "tuned_ms": tuned_ins_ms}},
            "answers_identical_across_modes": same,
            "small_batch": small}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# served workload: resident 4 GiB filter, Poisson requests, p50/p99
# ---------------------------------------------------------------------------
def served_measurement(n_poisson: int = 1000):
    """The served workload: the 3.1 Gbp human-shaped genome in a 2^35-bit
    (4 GiB) filter resident in HBM; a pool of 200 requests of log-uniform
    1 kb-10 Mbp of 150 bp reads with 1% errors in pinned host memory.
    Measures, on the same requests: the kernel's rate when all of them are
    device-resident in one launch (the direct-query rate) and in one launch
    each; the server's backlog rate with one client submitting all requests
    in one call, one client submitting one call per request and four
    clients; one launch per request through the server; and Poisson arrivals
    at 0.5 / 0.8 / 0.95 of the one-client backlog rate (p50 / p99 latency,
    with the time per stage).  Returns a dict."""
    import torch

    from paper_2606_24417_gb300 import synth
    from paper_2606_24417_gb300.sbf import FilterServer, SuperBloomFilter

    t = time.time()
    genome = synth.human_like_genome(3_100_000_000, seed=5)
    log(f"[bench] human-shaped genome generated in {time.time() - t:.1f}s")
    f = SuperBloomFilter(K, M, S, H, 1 << 35, shard_bits=SHARD_BITS)
    dg = torch.from_numpy(genome).cuda()
    do = torch.from_numpy(np.array([0, genome.size], dtype=np.int64)).cuda()
    f.insert(dg, do)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    f.insert(dg, do)
    e1.record()
    torch.cuda.synchronize()
    insert_ms = e0.elapsed_time(e1)
    del dg
    n_pool = 200
    sizes = np.exp(np.log(1e3) + synth.uniform01(9, 1, 0, n_pool) * (np.log(1e7) - np.log(1e3)))
    pool = []
    for i, sz in enumerate(sizes):
        n = max(1, int(sz) // READ_LEN)
        seq, off = synth.sample_reads(genome, n, READ_LEN, 0.01, seed=5000 + i)
        pool.append((torch.from_numpy(seq).pin_memory().numpy(),
                     torch.from_numpy(off.view(np.int64)).pin_memory().numpy().view(np.uint64),
                     n * (READ_LEN - K + 1)))
    del genome
    pool_kmers = float(sum(p[2] for p in pool))
    mean_kmers = pool_kmers / n_pool
    log(f"[bench] {n_pool} requests, {sum(p[0].size for p in pool) / 1e6:.0f} Mbp, "
        f"mean {mean_kmers / 1e3:.0f}k k-mers")

    # the direct-query rate on the same requests, device-resident
    allseq = np.concatenate([p[0] for p in pool])
    alloff = np.concatenate([[0], np.cumsum([p[0].size for p in pool])])
    lens = np.concatenate([np.diff(p[1].astype(np.int64)) for p in pool])
    reads_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    d_all, d_alloff = torch.from_numpy(allseq).cuda(), torch.from_numpy(reads_off).cuda()
    d_reqs = [(d_all[int(alloff[i]):int(alloff[i + 1])],
               torch.from_numpy(p[1].view(np.int64)).cuda()) for i, p in enumerate(pool)]
    hits_all = torch.empty(reads_off.size - 1, dtype=torch.int32, device="cuda")

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps / 1e3

    one_launch_s = timed(lambda: f.query(d_all, d_alloff, want_bits=False, hits=hits_all))
    per_req_s = timed(lambda: [f.query(s_, o_, want_bits=False) for s_, o_ in d_reqs], reps=1)
    del d_all, d_reqs

    def backlog(srv, clients=1, batch=False, reps=2):
        """Every pool request `reps` times from `clients` threads, then waited for."""
        srv.reset_stats()
        work = [(p[0], p[1]) for _ in range(reps) for p in pool]
        tickets = [None] * len(work)

        def client(c):
            idx = list(range(c, len(work), clients))
            if batch:
                for i, tk in zip(idx, srv.submit_many([work[i] for i in idx])):
                    tickets[i] = tk
            else:
                for i in idx:
                    tickets[i] = srv.submit(*work[i])

        ths = [threading.Thread(target=client, args=(c,)) for c in range(clients)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for tk in tickets:
            srv.wait(tk, 600)
        st = srv.stats()
        st.update(clients=clients, one_call=batch, breakdown=srv.breakdown())
        return st

    out = {"insert_ms": insert_ms,
           "direct": {"one_launch_kmers_per_s": pool_kmers / one_launch_s,
                      "launch_per_request_kmers_per_s": pool_kmers / per_req_s}}
    srv = FilterServer(f, read_budget_bytes=1 << 30, max_inflight=3)
    backlog(srv, batch=True, reps=1)  # warm
    out["backlog_1_client_one_call"] = backlog(srv, batch=True)
    out["backlog_1_client"] = backlog(srv)
    out["backlog_4_clients"] = backlog(srv, clients=4)
    one = FilterServer(f, read_budget_bytes=1 << 30, max_inflight=3, max_per_launch=1)
    backlog(one, reps=1)
    out["one_launch_per_request"] = backlog(one)
    one.close()
    peak = out["backlog_1_client"]["kmers_per_s"]
    loads = {}
    for load in (0.5, 0.8, 0.95):
        rate = load * peak / mean_kmers  # requests per second
        arrivals = synth.poisson_arrivals(n_poisson, rate, seed=int(load * 100))
        srv.reset_stats()
        tickets = []
        t0 = time.perf_counter()
        for i in range(n_poisson):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            p = pool[i % n_pool]
            tickets.append(srv.submit(p[0], p[1]))
        for tk in tickets:
            srv.wait(tk, 600)
        st = srv.stats()
        st.update(offered_load=load, offered_requests_per_s=rate,
                  achieved_requests_per_s=n_poisson / (time.perf_counter() - t0),
                  breakdown=srv.breakdown())
        loads[str(load)] = st
    out["poisson"] = loads
    srv.close()
    f.close()
    direct = out["direct"]["one_launch_kmers_per_s"]
    out["served_over_direct"] = {k: out[k]["kmers_per_s"] / direct for k in
                                 ("backlog_1_client_one_call", "backlog_1_client",
                                  "backlog_4_clients", "one_launch_per_request")}
    out["p99_over_p50"] = {k: v["p99_s"] / v["p50_s"] if v["p50_s"] else None
                           for k, v in loads.items()}
    return out


def run_served(args):
    import torch

    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    out = served_measurement()
    line = {"workload": "served: 3.1 Gbp order-5 Markov genome (GC 41%, 45% interspersed repeat copies "
                        "of 500 families 300 bp-6 kb, 10% divergence) in a 2^35-bit filter resident in "
                        "HBM; requests of 1 kb-10 Mbp of 150 bp reads with 1% errors, Poisson arrivals",
            **out}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# parameter sweep: s x m x H x shard bits x bits per k-mer on the 100 Mbp genome
# ---------------------------------------------------------------------------
def run_sweep(args):
    import itertools

    import torch

    from paper_2606_24417_gb300 import build_lib, synth
    from paper_2606_24417_gb300.sbf import SuperBloomFilter
    from paper_2606_24417_gb300.stats import expected_fpr

    build_lib.build()
    torch.cuda.set_device(0)
    genome = synth.bacterial_genome(GENOME_BP, seed=2)
    n_s = n_r = 1_000_000
    reads, roff = synth.mixed_query_reads(genome, n_s, n_r, READ_LEN, 0.01, seed=3)
    dg = torch.from_numpy(genome).cuda()
    dgo = torch.from_numpy(np.array([0, genome.size], dtype=np.int64)).cuda()
    dq = torch.from_numpy(reads).cuda()
    dqo = torch.from_numpy(roff.astype(np.int64)).cuda()
    bits_out = torch.empty((reads.size + 31) // 32, dtype=torch.int32, device="cuda")
    hits = torch.empty(n_s + n_r, dtype=torch.int32, device="cuda")
    ins_kmers = genome.size - K + 1
    q_kmers = (n_s + n_r) * (READ_LEN - K + 1)
    rand_kmers = n_r * (READ_LEN - K + 1)
    points = []
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for s, m, h, b, bpk in itertools.product((24, 26, 28, 31), (12, 14, 16, 20), (1, 2, 4, 8),
                                             (256, 512), (8, 12, 16)):
        f = SuperBloomFilter(K, m, s, h, bpk * ins_kmers, shard_bits=b)
        f.insert(dg, dgo)   # warm (bits are idempotent)
        f.query(dq, dqo, bits=bits_out, hits=hits)
        e[0].record()
        f.insert(dg, dgo)
        e[1].record()
        f.query(dq, dqo, bits=bits_out, hits=hits)
        e[2].record()
        torch.cuda.synchronize()
        fp = int(hits[n_s:].sum().item())
        words = f.words()
        points.append({"s": s, "m": m, "H": h, "B": b, "bits_per_kmer": bpk, "fused": f.fused,
                       "insert_ms": e[0].elapsed_time(e[1]), "query_ms": e[1].elapsed_time(e[2]),
                       "insert_kmers_per_s": ins_kmers / (e[0].elapsed_time(e[1]) / 1e3),
                       "query_kmers_per_s": q_kmers / (e[1].elapsed_time(e[2]) / 1e3),
                       "fpr_measured": fp / rand_kmers, "fpr_expected": expected_fpr(words, K, s, h, b),
                       "fill": float(np.bitwise_count(words).sum() / (words.size * 64))
                       if hasattr(np, "bitwise_count") else None})
        f.close()
    os.makedirs(args.out, exist_ok=True)
    with open(os.path.join(args.out, "sweep.json"), "w") as fh:
        json.dump(points, fh)
    best = min((p for p in points if p["bits_per_kmer"] == 16), key=lambda p: p["fpr_measured"])
    print(json.dumps({"workload": "sweep: 100 Mbp bacterial-shaped genome, s in {24,26,28,31}, "
                      "m in {12,14,16,20}, H in {1,2,4,8}, shard bits {256,512}, 8/12/16 bits per "
                      "k-mer; 1M sampled + 1M random 150 bp query reads (FPR from the random half)",
                      "points": len(points), "lowest_fpr_at_16_bits": best,
                      "written": os.path.join(args.out, "sweep.json")}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the paper's parameter sweep (Sec. V-B, Fig. 5) on its literal layout
# ---------------------------------------------------------------------------
PAPER_SWEEP_CLAIMS = {
    # (numerator point, denominator point): ratios the paper quotes (Sec. V-B)
    "H8_vs_H4": ((28, 16, 8), (28, 16, 4), {"fpr": 2.0, "total_time": 1.076}),
    "H16_vs_H4": ((28, 16, 16), (28, 16, 4), {"fpr": 5.2, "total_time": 1.659}),
    "s28_vs_s16": ((28, 16, 4), (16, 16, 4), {"fpr": 1 - 0.374, "total_time": 1 - 0.291}),
    "s30_vs_s28": ((30, 16, 4), (28, 16, 4), {"fpr": 1.256}),
    "s31_vs_s28": ((31, 16, 4), (28, 16, 4), {"fpr": 2.29}),
    "m12_vs_m8": ((28, 12, 4), (28, 8, 4), {"fpr": 1 - 0.917}),
    "m16_vs_m12": ((28, 16, 4), (28, 12, 4), {"fpr": 1 - 0.908}),
    "m18_vs_m16": ((28, 18, 4), (28, 16, 4), {"fpr": 1.035, "total_time": 1.085}),
    "m31_vs_m16": ((28, 31, 4), (28, 16, 4), {"fpr": 4.8, "insert_time": 7.7}),
}


def paper_sweep_points():
    pts = [(28, 16, h) for h in (4, 8, 12, 16)]
    pts += [(s, 16, 4) for s in (16, 20, 24, 26, 27, 28, 29, 30, 31)]
    pts += [(28, m, 4) for m in (8, 10, 12, 14, 16, 18, 20, 24, 31)]
    pts += [(s, m, h) for s in (24, 26, 28, 30, 31) for m in (12, 14, 16, 20)
            for h in (4, 8, 12, 16)]
    seen, out = set(), []
    for p in pts:
        if p not in seen:
            seen.add(p)
            out.append(p)
    return out


def run_paper_sweep(args):
    """(s, m, H) at k = 31 on the paper's layout (256-bit shards, 2^P of them,
    shard = minimizer key & (2^P - 1), forward strand only) with its 256 MiB
    budget, on the 100 Mbp bacterial-shaped genome standing in for C. elegans.
    Every point is timed on the generic one-k-mer-per-thread kernels (the
    paper's thread mapping) and on the default kernels (fused where the grid
    has them, else rolling)."""
    import torch

    from paper_2606_24417_gb300 import build_lib, synth
    from paper_2606_24417_gb300.sbf import LAYOUT_PAPER, SuperBloomFilter
    from paper_2606_24417_gb300.stats import expected_fpr

    build_lib.build()
    torch.cuda.set_device(0)
    genome = synth.bacterial_genome(GENOME_BP, seed=2)
    n_s = n_r = 1_000_000
    reads, roff = synth.mixed_query_reads(genome, n_s, n_r, READ_LEN, 0.01, seed=3)
    dg = torch.from_numpy(genome).cuda()
    dgo = torch.from_numpy(np.array([0, genome.size], dtype=np.int64)).cuda()
    dq = torch.from_numpy(reads).cuda()
    dqo = torch.from_numpy(roff.astype(np.int64)).cuda()
    bits_out = torch.empty((reads.size + 31) // 32, dtype=torch.int32, device="cuda")
    hits = torch.empty(n_s + n_r, dtype=torch.int32, device="cuda")
    rand_kmers = n_r * (READ_LEN - K + 1)
    budget_bits = 256 * 8 * (1 << 20)  # 256 MiB
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def timed(f):
        f.clear()
        f.insert(dg, dgo)
        f.query(dq, dqo, bits=bits_out, hits=hits)   # warm
        f.clear()
        e[0].record()
        f.insert(dg, dgo)
        e[1].record()
        f.query(dq, dqo, bits=bits_out, hits=hits)
        e[2].record()
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])

    points = {}
    for (s, m, h) in paper_sweep_points():
        rec = {"s": s, "m": m, "H": h}
        for variant in ("generic", "default"):
            # generic: one k-mer per thread (the paper's thread mapping); the
            # default kernels are the fused ones where the grid has them, else
            # the rolling ones
            if variant == "generic":
                os.environ["SBF_FORCE_GENERIC"] = "1"
            else:
                os.environ.pop("SBF_FORCE_GENERIC", None)
            f = SuperBloomFilter(K, m, s, h, budget_bits, shard_bits=256, canonical=False,
                                 layout=LAYOUT_PAPER)
            variant = f.kernel_variant
            ins_ms, q_ms = timed(f)
            rec[variant] = {"insert_ms": ins_ms, "query_ms": q_ms, "total_ms": ins_ms + q_ms}
            if variant == "generic":
                fp = int(hits[n_s:].sum().item())
                words = f.words()
                rec["fpr_measured"] = fp / rand_kmers
                rec["false_positives"] = fp
                rec["fpr_expected_uniform_shard"] = expected_fpr(words, K, s, h, 256, layout=1)
            else:   # both kernels give the same answers
                assert int(hits[n_s:].sum().item()) == rec["false_positives"]
            f.close()
        points[(s, m, h)] = rec
    os.environ.pop("SBF_FORCE_GENERIC", None)

    # the same budget and points on this library's default layout (mixed
    # minimizer -> any shard), to show what the mask rule costs
    default_layout = {}
    for (s, m, h) in ((28, 16, 4), (28, 16, 8), (28, 12, 4), (31, 16, 4)):
        f = SuperBloomFilter(K, m, s, h, budget_bits, shard_bits=256, canonical=False)
        ins_ms, q_ms = timed(f)
        fp = int(hits[n_s:].sum().item())
        default_layout[f"{s},{m},{h}"] = {
            "fpr_measured": fp / rand_kmers, "false_positives": fp,
            "fpr_paper_layout": points[(s, m, h)]["fpr_measured"],
            "insert_ms": ins_ms, "query_ms": q_ms, "fused": f.fused}
        f.close()

    claims = {}
    for name, (num, den, paper) in PAPER_SWEEP_CLAIMS.items():
        a, b = points[num], points[den]
        got = {"fpr": a["fpr_measured"] / b["fpr_measured"] if b["fpr_measured"] else None}
        for kern in ("generic", "fused", "rolling"):
            if kern in a and kern in b:
                got[f"total_time_{kern}"] = a[kern]["total_ms"] / b[kern]["total_ms"]
                got[f"insert_time_{kern}"] = a[kern]["insert_ms"] / b[kern]["insert_ms"]
        claims[name] = {"ours": got, "paper": paper}
    os.makedirs(args.out, exist_ok=True)
    with open(os.path.join(args.out, "paper_sweep.json"), "w") as fh:
        json.dump({"points": list(points.values()), "claims": claims,
                   "default_layout": default_layout}, fh)
    print(json.dumps({"workload": "paper sweep: k=31, (s, m, H) axes through (28, 16, 4) and the "
                      "s x m x H grid with H in {4,8,12,16}; paper layout (256-bit shards, "
                      "key & (2^P - 1), forward strand), 256 MiB filter; 100 Mbp "
                      "bacterial-shaped genome; 1M sampled + 1M random 150 bp query reads "
                      "(FPR from the random half)",
                      "points": len(points), "claims": claims,
                      "default_layout_same_budget": default_layout,
                      "written": os.path.join(args.out, "paper_sweep.json")}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# host-resident FASTA / FASTQ input (Sec. IV-A streamed FASTX, Sec. V-F)
# ---------------------------------------------------------------------------
def run_fastx(args):
    """Insert the bacterial genome from a FASTA file and query 2M reads from a
    FASTQ file (plain and gzip) through the streaming reader; beside them the
    same work from host arrays and from device-resident inputs."""
    import gzip
    import shutil
    import tempfile

    import torch

    from paper_2606_24417_gb300 import build_lib, synth
    from paper_2606_24417_gb300.fastx import insert_fastx, query_fastx
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    build_lib.build()
    torch.cuda.set_device(0)
    genome = synth.bacterial_genome(GENOME_BP, seed=2)
    n_s = n_r = 1_000_000
    reads, roff = synth.mixed_query_reads(genome, n_s, n_r, READ_LEN, 0.01, seed=3)
    tmp = tempfile.mkdtemp(prefix="sbf_fastx_")
    try:
        t = time.perf_counter()
        fa = os.path.join(tmp, "genome.fa")
        with open(fa, "wb") as fh:
            fh.write(b">genome synthetic 100 Mbp\n")
            lines = np.full((genome.size + 59) // 60 * 61, ord("\n"), dtype=np.uint8)
            full = genome.size // 60
            lines[:full * 61].reshape(full, 61)[:, :60] = genome[:full * 60].reshape(full, 60)
            rest = genome.size - full * 60
            if rest:
                lines[full * 61:full * 61 + rest] = genome[full * 60:]
                lines = lines[:full * 61 + rest + 1]
            fh.write(lines.tobytes())
        fq = os.path.join(tmp, "reads.fq")
        n = roff.size - 1
        rec = np.empty((n, 3 + READ_LEN + 3 + READ_LEN + 1), dtype=np.uint8)
        rec[:, 0] = ord("@")
        rec[:, 1] = ord("r")
        rec[:, 2] = ord("\n")
        rec[:, 3:3 + READ_LEN] = reads.reshape(n, READ_LEN)
        rec[:, 3 + READ_LEN:6 + READ_LEN] = np.frombuffer(b"\n+\n", dtype=np.uint8)
        rec[:, 6 + READ_LEN:6 + 2 * READ_LEN] = ord("I")
        rec[:, -1] = ord("\n")
        with open(fq, "wb") as fh:
            fh.write(rec.tobytes())
        fqz = fq + ".gz"
        with open(fq, "rb") as src, gzip.open(fqz, "wb", compresslevel=1) as dst:
            shutil.copyfileobj(src, dst, 16 << 20)
        from paper_2606_24417_gb300.fastx import write_bgzf

        fqb = fq + ".bgz"
        with open(fq, "rb") as src, open(fqb, "wb") as dst:
            dst.write(write_bgzf(src.read(), level=1))
        log(f"[bench] FASTX files written in {time.perf_counter() - t:.1f}s")
        ins_kmers = genome.size - K + 1
        q_kmers = n * (READ_LEN - K + 1)
        f = SuperBloomFilter(K, M, S, H, FILTER_BITS, shard_bits=SHARD_BITS)

        def best(fn, reps=3):
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                out = fn()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            return min(ts), out

        res = {}
        t_ins, info = best(lambda: (f.clear(), insert_fastx(f, fa))[1])
        res["fasta_insert"] = {"kmers_per_s": ins_kmers / t_ins, "seconds": t_ins,
                               "text_bytes": info["text_bytes"],
                               "parse_seconds": info["parse_seconds"], "batches": info["batches"]}
        want = f.words()
        for name, path in (("fastq_query", fq), ("fastq_gz_query", fqz)):
            t_q, (hits, kmers, qi) = best(lambda: query_fastx(f, path))
            res[name] = {"kmers_per_s": q_kmers / t_q, "seconds": t_q,
                         "text_bytes": qi["text_bytes"], "parse_seconds": qi["parse_seconds"],
                         "batches": qi["batches"], "positives": int(hits.sum())}
        # the same files tokenised on the device (raw text over the link)
        from paper_2606_24417_gb300.fastx import DeviceFastx

        dfx = DeviceFastx(f)
        t_dins, dinfo = best(lambda: (f.clear(), dfx.insert(fa))[1])
        same_dev = bool(np.array_equal(f.words(), want))
        res["fasta_insert_device_parse"] = {"kmers_per_s": ins_kmers / t_dins, "seconds": t_dins,
                                            "text_bytes": os.path.getsize(fa),
                                            "host_fallback_chunks": dinfo["host_fallback_chunks"]}
        for name, path in (("fastq_query_device_parse", fq), ("fastq_gz_query_device_parse", fqz),
                           ("fastq_bgzf_query_device_parse", fqb)):
            t_q, (hits, kmers, qi) = best(lambda: dfx.query(path))
            res[name] = {"kmers_per_s": q_kmers / t_q, "seconds": t_q,
                         "positives": int(hits.sum()),
                         "host_fallback_chunks": qi["host_fallback_chunks"]}
        # the same work from host arrays and from device-resident inputs
        h_genome = torch.from_numpy(genome).pin_memory().numpy()
        h_goff = np.array([0, genome.size], dtype=np.uint64)
        h_reads = torch.from_numpy(reads).pin_memory().numpy()
        h_roff = torch.from_numpy(roff.view(np.int64)).pin_memory().numpy().view(np.uint64)
        t_hi, _ = best(lambda: (f.clear(), f.insert_host(h_genome, h_goff)))
        same = bool(np.array_equal(f.words(), want))
        t_hq, (_, hh) = best(lambda: f.query_host(h_reads, h_roff, want_bits=False))
        dg = torch.from_numpy(genome).cuda()
        dgo = torch.from_numpy(h_goff.astype(np.int64)).cuda()
        dq = torch.from_numpy(reads).cuda()
        dqo = torch.from_numpy(roff.astype(np.int64)).cuda()
        hits_d = torch.empty(n, dtype=torch.int32, device="cuda")
        t_di, _ = best(lambda: (f.clear(), f.insert(dg, dgo)))
        t_dq, _ = best(lambda: f.query(dq, dqo, hits=hits_d, want_bits=False))
        agree = int(hh.astype(np.int64).sum()) == res["fastq_query"]["positives"] == \
            res["fastq_gz_query"]["positives"] == int(hits_d.sum().item()) == \
            res["fastq_query_device_parse"]["positives"] == \
            res["fastq_gz_query_device_parse"]["positives"] == \
            res["fastq_bgzf_query_device_parse"]["positives"] and same_dev
        res["host_arrays"] = {"insert_kmers_per_s": ins_kmers / t_hi,
                              "query_kmers_per_s": q_kmers / t_hq}
        res["device_resident"] = {"insert_kmers_per_s": ins_kmers / t_di,
                                  "query_kmers_per_s": q_kmers / t_dq,
                                  "note": "wall clock around one launch (host timer)"}
        print(json.dumps({"workload": "fastx: 100 Mbp bacterial-shaped genome as FASTA (60-column "
                          "lines) inserted; 1M sampled + 1M random 150 bp reads as FASTQ (plain, "
                          "gzip level 1 and BGZF level 1) queried; per-record hits",
                          "results": res, "filters_identical": same, "answers_agree": agree,
                          "host_cores": os.cpu_count()}), flush=True)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return 0


# ---------------------------------------------------------------------------
# the other alphabets of Sec. IV-A on the generic kernels
# ---------------------------------------------------------------------------
def run_alphabets(args):
    """Protein filter (k=12, m=6, s=10, H=4 over 5-bit residues) on a 100M-
    residue synthetic proteome, and a DNA-triplet filter (k=10, m=5, s=8,
    H=4 over 6-bit codons) on the 100 Mbp genome read as codons; each queried
    with 1M sampled reads (1% substitutions) + 1M random reads."""
    import torch

    from paper_2606_24417_gb300 import build_lib, synth
    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    build_lib.build()
    torch.cuda.set_device(0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    n_s = n_r = 1_000_000
    out = {}
    cases = {
        "protein": dict(k=12, m=6, s=10, H=4, bits=1 << 31, alphabet="protein", sym=1),
        "dna_triplet": dict(k=10, m=5, s=8, H=4, bits=1 << 29, alphabet="dna_triplet", sym=3),
    }
    for name, c in cases.items():
        if name == "protein":
            ref = synth.protein_sequence(100_000_000, 7)
            q1, o1 = synth.sample_peptides(ref, n_s, 150, 0.01, 8)
            q2, o2 = synth.random_peptides(n_r, 150, 9)
            rlen = 150
        else:
            ref = synth.bacterial_genome(GENOME_BP, seed=2)
            q1, o1 = synth.sample_reads(ref, n_s, 450, 0.01, 8)
            q2, o2 = synth.random_reads(n_r, 450, 9)
            rlen = 450
        q = np.concatenate([q1, q2])
        qo = np.concatenate([o1, o2[1:] + o1[-1]]).astype(np.uint64)
        ins_kmers = ref.size // c["sym"] - c["k"] + 1
        q_kmers = (n_s + n_r) * (rlen // c["sym"] - c["k"] + 1)
        dr, dro = dev(ref), dev(np.array([0, ref.size], dtype=np.int64))
        dq, dqo = dev(q), dev(qo.astype(np.int64))
        hits = torch.empty(n_s + n_r, dtype=torch.int32, device="cuda")
        bits = torch.empty((q.size + 31) // 32, dtype=torch.int32, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        answers = {}
        for variant in ("rolling", "generic"):
            # the generic one-k-mer-per-thread kernels, for comparison
            if variant == "generic":
                os.environ["SBF_FORCE_GENERIC"] = "1"
            f = SuperBloomFilter(c["k"], c["m"], c["s"], c["H"], c["bits"], shard_bits=512,
                                 canonical=False, alphabet=c["alphabet"])
            os.environ.pop("SBF_FORCE_GENERIC", None)
            assert f.kernel_variant == variant
            ti, tq = [], []
            for rep in range(args.warmup + args.steps):
                f.clear()
                ev[0].record()
                f.insert(dr, dro)
                ev[1].record()
                f.query(dq, dqo, bits=bits, hits=hits)
                ev[2].record()
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    ti.append(ev[0].elapsed_time(ev[1]))
                    tq.append(ev[1].elapsed_time(ev[2]))
            h = hits.cpu().numpy()
            answers[variant] = (bits.cpu().numpy(), h, f.words())
            out[f"{name}_{variant}"] = {
                "k": c["k"], "m": c["m"], "s": c["s"], "H": c["H"], "filter_bits": c["bits"],
                "insert_kmers": ins_kmers, "query_kmers": q_kmers,
                "insert_ms": statistics.median(ti), "query_ms": statistics.median(tq),
                "insert_kmers_per_s": ins_kmers / (statistics.median(ti) / 1e3),
                "query_kmers_per_s": q_kmers / (statistics.median(tq) / 1e3),
                "sampled_hit_fraction": float(h[:n_s].sum()) / (n_s * (rlen // c["sym"] - c["k"] + 1)),
                "fpr_random": float(h[n_s:].sum()) / (n_r * (rlen // c["sym"] - c["k"] + 1)),
                "kernel": f.kernel_variant}
            f.close()
        out[f"{name}_identical"] = all(np.array_equal(a, b) for a, b in
                                       zip(answers["rolling"], answers["generic"]))
        out[f"{name}_speedup"] = {
            "insert": out[f"{name}_generic"]["insert_ms"] / out[f"{name}_rolling"]["insert_ms"],
            "query": out[f"{name}_generic"]["query_ms"] / out[f"{name}_rolling"]["query_ms"]}
    print(json.dumps({"workload": "alphabets: protein filter on a 100M-residue synthetic proteome "
                      "(150-residue peptides) and DNA-triplet filter on the 100 Mbp genome "
                      "(450 bp reads); 1M sampled (1% substitutions) + 1M random queries each",
                      "results": out}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# false positives against filter size (Sec. V-D, Fig. 7)
# ---------------------------------------------------------------------------
def run_fpr_curve(args):
    """Insert the 100 Mbp genome (stand-in for C. elegans) into filters of
    2^22 .. 2^39 bits for s in {28, 30, 31} (k=31, m=16, H=4, 512-bit shards)
    and count false positives among 10^9 independent random 31-mers (reads of
    exactly 31 bases, resident on the device).  Beside each count: the
    shard-aware closed form (Eq. 2 conditioned on the built filter) where the
    filter is small enough to copy to the host."""
    import torch

    from paper_2606_24417_gb300 import build_lib, synth
    from paper_2606_24417_gb300.sbf import SuperBloomFilter
    from paper_2606_24417_gb300.stats import expected_fpr

    build_lib.build()
    torch.cuda.set_device(0)
    n_alien = 1_000_000_000
    batch = 100_000_000
    genome = synth.bacterial_genome(GENOME_BP, seed=2)
    dg = torch.from_numpy(genome).cuda()
    dgo = torch.tensor([0, genome.size], dtype=torch.int64).cuda()
    t = time.time()
    aliens = []
    for b in range(n_alien // batch):
        a = synth.uniform_dna(batch * K, 1000 + b)
        aliens.append(torch.from_numpy(a).cuda())
    aoff = torch.arange(0, batch * K + 1, K, dtype=torch.int64, device="cuda")
    hits = torch.empty(batch, dtype=torch.int32, device="cuda")
    log(f"[bench] 10^9 random 31-mers on the device in {time.time() - t:.1f}s")
    rows = []
    for s_ in (28, 30, 31):
        for e in range(22, 40):
            f = SuperBloomFilter(K, M, s_, H, 1 << e, shard_bits=SHARD_BITS)
            f.insert(dg, dgo)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fp = 0
            for a in aliens:
                f.query(a, aoff, hits=hits, want_bits=False)
                fp += int(hits.sum().item())
            dt = time.perf_counter() - t0
            row = {"s": s_, "log2_bits": e, "false_positives": fp, "fpr": fp / n_alien,
                   "query_seconds": dt}
            if e <= 34:
                row["fpr_expected"] = expected_fpr(f.words(), K, s_, H, SHARD_BITS)
            rows.append(row)
            log(f"[bench] s={s_} 2^{e}: {fp} false positives")
            f.close()
    os.makedirs(args.out, exist_ok=True)
    with open(os.path.join(args.out, "fpr_curve.json"), "w") as fh:
        json.dump(rows, fh)
    print(json.dumps({"workload": "fpr_curve: 100 Mbp bacterial-shaped genome inserted into "
                      "2^22..2^39-bit filters (k=31, m=16, H=4, 512-bit shards), s in {28,30,31}; "
                      "false positives among 10^9 independent random 31-mers",
                      "rows": rows}), flush=True)
    return 0


def measure_filter_size(e, steps, dev, stream, genome, reads, roff, d_genome, d_goff, d_reads,
                        d_roff, d_bits, d_hits, flush):
    """One filter size of the bacterial workload: median insert and query
    times over max(steps, 3) steps after 3 warm-up steps (L2 flushed before
    each), each set against the random-sector roofline of a buffer of the
    filter's size (streamed bytes at the copy peak plus one shard per
    super-k-mer run at the probe's rate; read-modify-write for the insert)."""
    import torch

    from paper_2606_24417_gb300.sbf import SuperBloomFilter

    peak, _ = measured_peaks()
    sector_b = SHARD_BITS // 8
    n_reads = roff.size - 1
    ins_kmers = genome.size - K + 1
    q_kmers = n_reads * (READ_LEN - K + 1)
    stats = torch.zeros(3, dtype=torch.int64, device=dev)
    f = SuperBloomFilter(K, M, S, H, 1 << e, shard_bits=SHARD_BITS)
    # runs (one shard each) of the query and of the insert
    f.insert(d_genome, d_goff)
    f.query(d_reads, d_roff, bits=d_bits, hits=d_hits, stats=stats)
    torch.cuda.synchronize()
    runs_q = int(stats[1].item())
    stats.zero_()
    f.query(d_genome, d_goff, want_bits=False, want_hits=False, stats=stats)
    torch.cuda.synchronize()
    runs_i = int(stats[1].item())
    t_i, t_q = [], []
    for rep in range(3 + max(steps, 3)):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        flush.fill_(1)
        f.clear()
        ev[0].record(stream)
        f.insert(d_genome, d_goff)
        ev[1].record(stream)
        f.query(d_reads, d_roff, bits=d_bits, hits=d_hits)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if rep >= 3:
            t_i.append(ev[0].elapsed_time(ev[1]))
            t_q.append(ev[1].elapsed_time(ev[2]))
    ins_ms, q_ms = statistics.median(t_i), statistics.median(t_q)
    fbytes = f.nbytes
    status = f.device_status()
    g_gbs = sector_bandwidth(dev, stream, fbytes, sector_b, False, 1 << 27)
    r_gbs = sector_bandwidth(dev, stream, fbytes, sector_b, True, 1 << 25)
    q_stream = reads.nbytes + roff.nbytes + (reads.size + 7) // 8 + 4 * n_reads
    q_bound = q_kmers / (q_stream / (peak * 1e9) + runs_q * sector_b / (g_gbs * 1e9))
    i_bound = ins_kmers / (genome.nbytes / (peak * 1e9) + runs_i * 2 * sector_b / (r_gbs * 1e9))
    q_rate, i_rate = q_kmers / (q_ms / 1e3), ins_kmers / (ins_ms / 1e3)
    row = {"log2_bits": e, "filter_bytes": fbytes, "in_l2": fbytes <= (96 << 20),
           "insert_ms": ins_ms, "query_ms": q_ms,
           "insert_kmers_per_s": i_rate, "query_kmers_per_s": q_rate,
           "probe_gather_gbs": g_gbs, "probe_rmw_gbs": r_gbs,
           "query_sector_bound": q_bound, "insert_sector_bound": i_bound,
           "query_frac": q_rate / q_bound, "insert_frac": i_rate / i_bound,
           "positive_kmers": int(d_hits.sum().item()), "device_status": status}
    f.close()
    return row


def run_filter_sizes(args):
    """The bacterial workload (100 Mbp genome inserted, 20M 150 bp reads
    queried; k=31, m=16, s=28, H=4, 512-bit shards) on filters of 8 MiB to
    4 GiB: inside the 129 MB L2, around it and far beyond it.  Each size is
    set against its own random-sector roofline: streamed bytes at the copy
    peak plus one shard per super-k-mer run at the probe's measured rate
    over a buffer of the filter's size (served from L2 when it fits)."""
    import torch

    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    genome, reads, roff = make_workload(0, small=args.case == "small")
    n_reads = roff.size - 1
    d_genome = torch.from_numpy(genome).to(dev)
    d_goff = torch.tensor([0, genome.size], dtype=torch.int64, device=dev)
    d_reads = torch.from_numpy(reads).to(dev)
    d_roff = torch.from_numpy(roff.astype(np.int64)).to(dev)
    d_bits = torch.empty((reads.size + 31) // 32, dtype=torch.int32, device=dev)
    d_hits = torch.empty(n_reads, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peak, peak_kind = measured_peaks()
    rows = []
    for e in (26, 27, 28, 29, 30, 31, 32, 33, 35):
        row = measure_filter_size(e, args.steps, dev, stream, genome, reads, roff, d_genome,
                                  d_goff, d_reads, d_roff, d_bits, d_hits, flush)
        rows.append(row)
        log(f"[bench] 2^{e} bits: query {row['query_kmers_per_s'] / 1e9:.1f} G/s "
            f"({row['query_frac']:.2f} of bound), insert {row['insert_kmers_per_s'] / 1e9:.1f} G/s "
            f"({row['insert_frac']:.2f})")
    os.makedirs(args.out, exist_ok=True)
    with open(os.path.join(args.out, "filter_sizes.json"), "w") as fh:
        json.dump(rows, fh)
    print(json.dumps({"workload": "filter_sizes: 100 Mbp bacterial-shaped genome inserted, "
                      f"{n_reads} 150 bp reads queried (half sampled with 1% errors, half random), "
                      "k=31 m=16 s=28 H=4, 512-bit shards, filters of 2^26..2^35 bits; "
                      "256 MB L2 flush before each timed step",
                      "peak_gbs": peak, "peak_kind": peak_kind, "rows": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: 2M query reads (300 MB, still larger than L2) for profiling")
    ap.add_argument("--workload", default="bacterial",
                    choices=["bacterial", "batched", "served", "sweep", "paper_sweep", "fastx",
                             "alphabets", "fpr_curve", "filter_sizes"],
                    help="batched: the many-filter workload (its own JSON line)")
    ap.add_argument("--out", default=os.path.join(ROOT, "bench_results"),
                    help="directory for the per-point JSON of the sweep-type workloads")
    ap.add_argument("--filter-log2", type=int, default=30,
                    help="filter of 2^N bits for the default workload (30: the headline 128 MiB)")
    ap.add_argument("--no-served", action="store_true",
                    help="leave the served workload out of the default line")
    ap.add_argument("--skip-extras", action="store_true",
                    help="device-timed steps only (no e2e, no CPU baseline): profiling runs")
    args = ap.parse_args()
    if args.warmup < 3:
        log("[bench] warmup raised to 3")
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args) if rank == 0 else 0
    if args.workload == "served":
        return run_served(args) if rank == 0 else 0
    if args.workload == "sweep":
        return run_sweep(args) if rank == 0 else 0
    if args.workload == "paper_sweep":
        return run_paper_sweep(args) if rank == 0 else 0
    if args.workload == "fastx":
        return run_fastx(args) if rank == 0 else 0
    if args.workload == "alphabets":
        return run_alphabets(args) if rank == 0 else 0
    if args.workload == "fpr_curve":
        return run_fpr_curve(args) if rank == 0 else 0
    if args.workload == "filter_sizes":
        return run_filter_sizes(args) if rank == 0 else 0
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
