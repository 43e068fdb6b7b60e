"""Seeded synthetic genomic workloads (inputs only).

This module generates DNA sequences, read sets and request streams.  It holds
none of the filter's arithmetic: its random numbers come from a counter-based
generator built on the MurmurHash3 64-bit finaliser (Appleby), and reverse
strands are produced with a byte translation table.  Everything is
deterministic for a given seed and independent of the numpy version.

Workload shapes follow the filter's evaluation: uniform random DNA, Markov
genomes with a GC target and repeat copies (bacterial- and human-shaped),
reads sampled from either strand with substitution errors, uniform random
reads, lognormal read lengths and Poisson request arrivals.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np


def _parallel(fn, items):
    """Run fn over items on threads (numpy releases the GIL in its loops);
    threads, not processes, so it is safe after CUDA initialisation."""
    items = list(items)
    workers = min(len(items), os.cpu_count() or 1, 32)
    if workers <= 1:
        for it in items:
            fn(it)
        return
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(fn, items))

_ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
_COMPLEMENT = np.arange(256, dtype=np.uint8)
for _a, _b in zip(b"ACGTacgt", b"TGCAtgca"):
    _COMPLEMENT[_a] = _b

_M1 = np.uint64(0xFF51AFD7ED558CCD)
_M2 = np.uint64(0xC4CEB9FE1A85EC53)
_S33 = np.uint64(33)


def _fmix64(x: np.ndarray) -> np.ndarray:
    x = x ^ (x >> _S33)
    x = x * _M1
    x = x ^ (x >> _S33)
    x = x * _M2
    return x ^ (x >> _S33)


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _fmix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
        b = _fmix64(a ^ np.uint64(stream & 0xFFFFFFFFFFFFFFFF) ^ np.uint64(0x632BE59BD9B4E019))
    return b[0]


def u64(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """n counter-based 64-bit random words: element i depends only on (seed, stream, start+i)."""
    return u64_at(seed, stream, np.arange(start, start + n, dtype=np.uint64))


def u64_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based 64-bit random words at arbitrary counters idx."""
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        return _fmix64(np.asarray(idx, dtype=np.uint64) * np.uint64(0xD6E8FEB86659FD93) + key)


def uniform01(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) (53 bits)."""
    return (u64(seed, stream, start, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def randint(seed: int, stream: int, n: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi) (multiply-shift on 53-bit uniforms);
    element i uses counter start + i."""
    span = hi - lo
    return lo + np.floor(uniform01(seed, stream, start, n) * span).astype(np.int64)


# ----------------------------------------------------------------------------
# sequences
# ----------------------------------------------------------------------------
_BYTE_TO_BASES = _ACGT[(np.arange(256)[:, None] >> (2 * np.arange(4))[None, :]) & 3].astype(np.uint8)


def uniform_dna(n: int, seed: int) -> np.ndarray:
    """n uniform random bases (uint8 ASCII 'ACGT'): each random byte gives four
    bases (2 bits each, low bits first)."""
    out = np.empty(n, dtype=np.uint8)
    chunk = 1 << 24

    def fill(s):
        e = min(n, s + chunk)
        w = u64(seed, 1, s // 32, (e - s + 31) // 32)
        out[s:e] = _BYTE_TO_BASES[w.view(np.uint8)].reshape(-1)[: e - s]

    _parallel(fill, range(0, n, chunk))
    return out


def reverse_complement(x: np.ndarray) -> np.ndarray:
    """Reverse strand of an ASCII DNA array (non-ACGT bytes kept)."""
    return _COMPLEMENT[np.asarray(x, dtype=np.uint8)[::-1]]


# Concentration of the Dirichlet transition rows.  alpha = 5 gives an
# expected conditional entropy of about 1.9 bits per base, close to real
# genomes; alpha = 1 (about 1.56 bits) makes 16-mers so repetitive that a
# few thousand minimizers saturate their shards.
MARKOV_ALPHA = 5


def _markov_table(order: int, gc: float, seed: int, alpha: int = MARKOV_ALPHA) -> np.ndarray:
    """Transition table [4^order, 4]: Dirichlet(alpha) rows (normalised sums of
    alpha exponentials) tilted to a stationary GC fraction."""
    n_ctx = 4 ** order
    e = np.zeros((n_ctx, 4))
    for j in range(alpha):
        e += -np.log1p(-uniform01(seed, 7 + 100 * j, 0, n_ctx * 4)).reshape(n_ctx, 4)
    base = e / e.sum(axis=1, keepdims=True)
    is_gc = np.array([0.0, 1.0, 1.0, 0.0])

    def tilt(t):
        w = base * np.where(is_gc > 0, t, 1.0)[None, :]
        return w / w.sum(axis=1, keepdims=True)

    def stationary_gc(P):
        # power iteration on the 4^order context chain
        pi = np.full(n_ctx, 1.0 / n_ctx)
        nxt = (np.arange(n_ctx)[:, None] * 4 + np.arange(4)[None, :]) % n_ctx
        for _ in range(200):
            new = np.zeros(n_ctx)
            np.add.at(new, nxt.reshape(-1), (pi[:, None] * P).reshape(-1))
            pi = new
        return float((pi[:, None] * P * is_gc[None, :]).sum())

    lo, hi = 1e-3, 1e3
    for _ in range(60):  # bisection on the log of the tilt
        mid = math.sqrt(lo * hi)
        if stationary_gc(tilt(mid)) < gc:
            lo = mid
        else:
            hi = mid
    return tilt(math.sqrt(lo * hi))


def markov_dna(n: int, order: int, gc: float, seed: int, n_chains: int | None = None) -> np.ndarray:
    """Order-`order` Markov DNA of length n, run as n_chains independent
    segments (vectorised across segments, groups of segments on threads)
    that are concatenated.  The next base is looked up from the top 16 bits
    of a uniform draw in a per-context quantile table (probabilities resolved
    to 2^-16).  Step t of chain c draws counter t * n_chains + c, so the
    result does not depend on the thread grouping."""
    P = _markov_table(order, gc, seed)
    cum = np.cumsum(P, axis=1)
    cum[:, -1] = 1.0
    n_ctx = 4 ** order
    q = (np.arange(1 << 16, dtype=np.float64) + 0.5) / (1 << 16)
    table = np.empty((n_ctx, 1 << 16), dtype=np.uint8)
    for c in range(n_ctx):
        table[c] = np.searchsorted(cum[c], q, side="right")
    table = np.minimum(table, 3).reshape(-1)
    if n_chains is None:  # about 256 steps: large vector operations run well on threads
        n_chains = max(4096, -(-n // 256))
    n_chains = max(1, min(n_chains, n))
    seg = (n + n_chains - 1) // n_chains
    codes = np.empty((seg, n_chains), dtype=np.uint8)
    ctx0 = randint(seed, 11, n_chains, 0, n_ctx)
    n_groups = max(1, min(os.cpu_count() or 1, 32, n_chains // 1024))
    bounds = np.linspace(0, n_chains, n_groups + 1).astype(np.int64)
    s48 = np.uint64(48)

    def run(gi):
        c0, c1 = int(bounds[gi]), int(bounds[gi + 1])
        ctx = ctx0[c0:c1].astype(np.int64)
        for t in range(seg):
            u = (u64(seed, 12, t * n_chains + c0, c1 - c0) >> s48).astype(np.int64)
            c = table[ctx * (1 << 16) + u]
            codes[t, c0:c1] = c
            ctx = (ctx * 4 + c) % n_ctx

    _parallel(run, range(n_groups))
    return _ACGT[codes.T.reshape(-1)[:n]]


def gc_fraction(x: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.uint8)
    return float(np.isin(x, np.frombuffer(b"CGcg", dtype=np.uint8)).mean())


def add_exact_repeats(genome: np.ndarray, frac: float, min_len: int, max_len: int,
                      seed: int) -> np.ndarray:
    """Overwrite about frac of the genome with exact copies of other segments
    (uniform length in [min_len, max_len], uniform source/destination,
    random strand)."""
    g = genome.copy()
    n = g.size
    if n <= max_len * 2:
        return g
    mean = (min_len + max_len) / 2
    count = int(round(frac * n / mean))
    lens = randint(seed, 21, count, min_len, max_len + 1)
    src = randint(seed, 22, count, 0, n - max_len)
    dst = randint(seed, 23, count, 0, n - max_len)
    strand = randint(seed, 24, count, 0, 2)
    for L, a, b, st in zip(lens, src, dst, strand):
        piece = genome[a:a + L]
        g[b:b + L] = reverse_complement(piece) if st else piece
    return g


def add_diverged_repeats(genome: np.ndarray, frac: float, n_families: int, min_len: int,
                         max_len: int, divergence: float, seed: int, order: int = 5,
                         gc: float = 0.41) -> np.ndarray:
    """Interspersed repeats: n_families consensus sequences (log-uniform lengths,
    drawn from the same Markov chain), copied with independent substitutions
    and random strand until about frac of the genome is covered.  Copies are
    written in order (a later copy overwrites an earlier one)."""
    g = genome.copy()
    n = g.size
    ll = np.exp(np.log(min_len) + uniform01(seed, 31, 0, n_families)
                * (np.log(max_len) - np.log(min_len)))
    flen = np.maximum(min_len, ll.astype(np.int64))
    fam_src = markov_dna(int(flen.sum()), order, gc, seed + 1, n_chains=min(4096, n_families))
    fstart = np.concatenate([[0], np.cumsum(flen)[:-1]])
    mean = float(flen.mean())
    count = int(round(frac * n / mean))
    fam = randint(seed, 32, count, 0, n_families)
    dst = randint(seed, 33, count, 0, max(1, n - max_len))
    strand = randint(seed, 34, count, 0, 2).astype(bool)
    L = flen[fam]
    cum = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(L, out=cum[1:])
    # chunks of whole copies, about 2^23 bases each
    cuts = [0]
    while cuts[-1] < count:
        nxt = int(np.searchsorted(cum, cum[cuts[-1]] + (1 << 23), side="right")) - 1
        cuts.append(max(nxt, cuts[-1] + 1))
    chunks = list(zip(cuts[:-1], cuts[1:]))
    results = [None] * len(chunks)
    thr = np.uint64(int(divergence * 2.0 ** 32))

    def build(ci):
        a, b = chunks[ci]
        base = cum[a]
        m = int(cum[b] - base)
        owner = np.repeat(np.arange(a, b), L[a:b])
        within = np.arange(m, dtype=np.int64) - (cum[owner] - base)
        st = strand[owner]
        src = fstart[fam[owner]] + np.where(st, L[owner] - 1 - within, within)
        vals = fam_src[src]
        vals = np.where(st, _COMPLEMENT[vals], vals)
        u = u64(seed, 35, int(base), m)
        hit = np.nonzero((u >> np.uint64(32)) < thr)[0]
        if hit.size:
            sub = 1 + (((u[hit] & np.uint64(0xFFFFFFFF)) * np.uint64(3)) >> np.uint64(32)).astype(np.int64)
            code = np.searchsorted(_ACGT, vals[hit])
            vals[hit] = _ACGT[(code + sub) % 4]
        results[ci] = (dst[owner] + within, vals)

    step = max(1, min(32, os.cpu_count() or 1))
    for c0 in range(0, len(chunks), step):  # bounded memory: build a group, apply it in order
        ids = range(c0, min(len(chunks), c0 + step))
        _parallel(build, ids)
        for ci in ids:
            pos, vals = results[ci]
            g[pos] = vals
            results[ci] = None
    return g


# ----------------------------------------------------------------------------
# reads
# ----------------------------------------------------------------------------
def concat(reads) -> tuple[np.ndarray, np.ndarray]:
    """Concatenate a list of uint8 reads into (seq, off[n+1])."""
    lens = np.array([len(r) for r in reads], dtype=np.uint64)
    off = np.zeros(len(reads) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    seq = np.concatenate([np.asarray(r, dtype=np.uint8) for r in reads]) if reads else \
        np.zeros(0, dtype=np.uint8)
    return seq, off


def fixed_length_offsets(n_reads: int, length: int) -> np.ndarray:
    return (np.arange(n_reads + 1, dtype=np.uint64) * np.uint64(length))


def sample_reads(genome: np.ndarray, n_reads: int, length: int, error_rate: float,
                 seed: int, chunk: int = 1 << 18) -> tuple[np.ndarray, np.ndarray]:
    """n_reads reads of one length from uniform positions on a random strand,
    each base substituted with probability error_rate (uniform among the
    other three).  Returns (seq, off).  Generated in chunks of reads; the
    result does not depend on the chunk size."""
    n = genome.size
    out = np.empty(n_reads * length, dtype=np.uint8)
    thr = np.uint64(int(error_rate * 2.0 ** 32))
    lo32 = np.uint64(0xFFFFFFFF)
    windows = np.lib.stride_tricks.sliding_window_view(genome, length)

    def one(c0):
        c1 = min(n_reads, c0 + chunk)
        m = c1 - c0
        starts = randint(seed, 41, m, 0, n - length + 1, start=c0)
        reads = windows[starts]
        strand = randint(seed, 42, m, 0, 2, start=c0).astype(bool)
        if strand.any():
            reads[strand] = _COMPLEMENT[reads[strand][:, ::-1]]
        flat = reads.reshape(-1)
        base = c0 * length
        # base j of the batch is an error iff its 32-bit uniform (one half of
        # word j // 2) is below the rate; the substitute comes from counter j
        first = base // 2
        w = u64(seed, 43, first, (base + flat.size + 1) // 2 - first)
        halves = np.empty(w.size * 2, dtype=np.uint64)
        halves[0::2] = w >> np.uint64(32)
        halves[1::2] = w & lo32
        halves = halves[base - 2 * first: base - 2 * first + flat.size]
        idx = np.nonzero(halves < thr)[0]
        if idx.size:
            r = u64_at(seed, 44, idx.astype(np.uint64) + np.uint64(base))
            sub = 1 + (((r >> np.uint64(32)) * np.uint64(3)) >> np.uint64(32)).astype(np.int64)
            code = np.searchsorted(_ACGT, flat[idx])
            flat[idx] = _ACGT[(code + sub) % 4]
        out[base:base + flat.size] = flat

    _parallel(one, range(0, n_reads, chunk))
    return out, fixed_length_offsets(n_reads, length)


def random_reads(n_reads: int, length: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    return uniform_dna(n_reads * length, seed), fixed_length_offsets(n_reads, length)


def lognormal_lengths(n: int, median: float, sigma: float, lo: int, hi: int,
                      seed: int) -> np.ndarray:
    """clip(round(lognormal(ln median, sigma)), lo, hi) via Box-Muller."""
    u1 = uniform01(seed, 51, 0, n)
    u2 = uniform01(seed, 52, 0, n)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return np.clip(np.rint(np.exp(np.log(median) + sigma * z)), lo, hi).astype(np.int64)


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    gaps = -np.log1p(-uniform01(seed, 61, 0, n)) / rate_per_s
    return np.cumsum(gaps)


# ----------------------------------------------------------------------------
# the evaluation workloads
# ----------------------------------------------------------------------------
def bacterial_genome(n: int = 100_000_000, seed: int = 2) -> np.ndarray:
    """Order-3 Markov genome (Dirichlet(5) rows) at GC 50% with 3% of it overwritten by exact
    1-10 kb repeat copies (random strand)."""
    g = markov_dna(n, 3, 0.5, seed)
    return add_exact_repeats(g, 0.03, 1000, 10000, seed + 100)


def human_like_genome(n: int = 3_100_000_000, seed: int = 5) -> np.ndarray:
    """Order-5 Markov genome at GC 41% with 45% covered by interspersed copies
    of 500 repeat families (300 bp - 6 kb, 10% divergence, random strand)."""
    g = markov_dna(n, 5, 0.41, seed)
    return add_diverged_repeats(g, 0.45, 500, 300, 6000, 0.10, seed + 100)


def mixed_query_reads(genome: np.ndarray, n_sampled: int, n_random: int, length: int,
                      error_rate: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """n_sampled reads from the genome (with errors) followed by n_random uniform reads."""
    s1, _ = sample_reads(genome, n_sampled, length, error_rate, seed)
    s2, _ = random_reads(n_random, length, seed + 1)
    seq = np.concatenate([s1, s2])
    return seq, fixed_length_offsets(n_sampled + n_random, length)


def sample_variable_reads(genome: np.ndarray, lengths: np.ndarray, error_rate: float, seed: int,
                          stream_base: int = 0) -> np.ndarray:
    """Concatenated reads of the given lengths (each clipped to the genome)
    from uniform positions on a random strand with substitution errors."""
    n = genome.size
    lengths = np.minimum(np.asarray(lengths, dtype=np.int64), n)
    total = int(lengths.sum())
    out = np.empty(total, dtype=np.uint8)
    if total == 0:
        return out
    starts = randint(seed, 71 + stream_base, lengths.size, 0, 1 << 62) % (n - lengths + 1)
    strand = randint(seed, 72 + stream_base, lengths.size, 0, 2).astype(bool)
    cum = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=cum[1:])
    step = 1 << 24
    r0 = 0
    while r0 < lengths.size:
        r1 = int(np.searchsorted(cum, cum[r0] + step, side="right")) - 1
        r1 = max(r1, r0 + 1)
        L = lengths[r0:r1]
        base = cum[r0]
        rel = np.arange(int(cum[r1] - base), dtype=np.int64)
        owner = np.repeat(np.arange(r0, r1), L)
        within = rel - (cum[owner] - base)
        fwd = starts[owner] + within
        rev = starts[owner] + (lengths[owner] - 1 - within)
        sb = strand[owner]
        piece = genome[np.where(sb, rev, fwd)]
        piece = np.where(sb, _COMPLEMENT[piece], piece)
        out[base:base + piece.size] = piece
        r0 = r1
    u = u64(seed, 73 + stream_base, 0, total)
    idx = np.nonzero((u >> np.uint64(32)) < np.uint64(int(error_rate * 2.0 ** 32)))[0]
    if idx.size:
        sub = 1 + (((u[idx] & np.uint64(0xFFFFFFFF)) * np.uint64(3)) >> np.uint64(32)).astype(np.int64)
        code = np.searchsorted(_ACGT, out[idx])
        out[idx] = _ACGT[(code + sub) % 4]
    return out


def batched_workload(n_filters: int = 256, exp_lo: int = 20, exp_hi: int = 28,
                     genome_lo: float = 1e6, genome_hi: float = 50e6, n_reads: int = 5_000_000,
                     seed: int = 4, read_cap: int = 100_000):
    """Many independent filters queried in one launch.

    Filter sizes 2^e bits with e uniform in [exp_lo, exp_hi]; genome lengths
    log-uniform in [genome_lo, genome_hi] (uniform random DNA); both lists
    sorted ascending and paired so bits per k-mer stay in a sane range.  Read
    lengths clip(round(lognormal(ln 150, 1.5)), 1, read_cap); each read goes
    to a uniform filter; half are sampled from that filter's genome with 1%
    errors, half are random.  Reads are grouped by filter.

    Returns dict(bits, genomes, gseq, goff, ggroup, seq, off, group)."""
    exps = np.sort(randint(seed, 81, n_filters, exp_lo, exp_hi + 1))
    glen = np.sort(np.exp(np.log(genome_lo) + uniform01(seed, 82, 0, n_filters)
                          * (np.log(genome_hi) - np.log(genome_lo))).astype(np.int64))
    bits = [int(1) << int(e) for e in exps]
    genomes = [uniform_dna(int(L), seed * 1000 + f) for f, L in enumerate(glen)]
    lens = lognormal_lengths(n_reads, 150, 1.5, 1, read_cap, seed + 7)
    owner = randint(seed, 83, n_reads, 0, n_filters)
    sampled = randint(seed, 84, n_reads, 0, 2).astype(bool)
    order = np.argsort(owner, kind="stable")
    owner, lens, sampled = owner[order], lens[order], sampled[order]
    group = np.searchsorted(owner, np.arange(n_filters + 1)).astype(np.uint64)
    parts = [None] * n_filters

    def reads_of(f):
        a, b = int(group[f]), int(group[f + 1])
        if a == b:
            return
        L, smp = lens[a:b], sampled[a:b]
        piece_s = sample_variable_reads(genomes[f], L[smp], 0.01, seed + 11 * f + 1)
        piece_r = uniform_dna(int(L[~smp].sum()), seed * 7919 + f)
        # interleave in read order: sampled and random reads keep their slots
        Lc = np.minimum(L, np.where(smp, genomes[f].size, L))
        cum_s = np.concatenate([[0], np.cumsum(Lc[smp])])
        cum_r = np.concatenate([[0], np.cumsum(L[~smp])])
        src = np.empty(L.size, dtype=np.int64)     # start of each read in piece_s ++ piece_r
        src[smp] = cum_s[:-1]
        src[~smp] = piece_s.size + cum_r[:-1]
        dst = np.concatenate([[0], np.cumsum(Lc)])
        idx = np.repeat(src - dst[:-1], Lc) + np.arange(int(dst[-1]), dtype=np.int64)
        parts[f] = np.concatenate([piece_s, piece_r])[idx]
        lens[a:b] = Lc

    _parallel(reads_of, range(n_filters))
    parts = [p for p in parts if p is not None]
    seq = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    off = np.zeros(n_reads + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    gseq = np.concatenate(genomes)
    gl = np.array([g.size for g in genomes], dtype=np.uint64)
    goff = np.zeros(n_filters + 1, dtype=np.uint64)
    np.cumsum(gl, out=goff[1:])
    return dict(bits=bits, genomes=genomes, gseq=gseq, goff=goff,
                ggroup=np.arange(n_filters + 1, dtype=np.uint64), seq=seq, off=off, group=group)


# ----------------------------------------------------------------------------
# proteins (Sec. IV-A's 26-symbol alphabet; the 20 standard residues occur)
# ----------------------------------------------------------------------------
AMINO = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", dtype=np.uint8)
# residue frequencies in percent, rounded (typical of large protein databases)
_AMINO_PCT = np.array([8.3, 1.4, 5.5, 6.8, 3.9, 7.1, 2.3, 5.9, 5.8, 9.7,
                       2.4, 4.1, 4.7, 3.9, 5.5, 6.6, 5.4, 6.9, 1.1, 2.9])
_AMINO_CDF = np.cumsum(_AMINO_PCT / _AMINO_PCT.sum())


def protein_sequence(n: int, seed: int, dup_frac: float = 0.05) -> np.ndarray:
    """n residues drawn i.i.d. from the frequencies above, then dup_frac of
    them overwritten by copies of 50-300-residue segments (paralogous
    domains), each copy with 10% substitutions."""
    u = uniform01(seed, 11, 0, n)
    out = AMINO[np.minimum(np.searchsorted(_AMINO_CDF, u, side="right"), 19)]
    if dup_frac > 0 and n > 1000:
        budget = int(dup_frac * n)
        lens = randint(seed, 12, max(1, budget // 50), 50, 301)
        lens = lens[: max(1, int(np.searchsorted(np.cumsum(lens), budget)))]
        src = randint(seed, 13, lens.size, 0, n - 301)
        dst = randint(seed, 14, lens.size, 0, n - 301)
        for i, L in enumerate(lens):
            seg = out[src[i]:src[i] + L].copy()
            mut = uniform01(seed, 15, int(i) * 301, int(L)) < 0.10
            seg[mut] = AMINO[randint(seed, 16, int(mut.sum()), 0, 20, start=int(i) * 301)]
            out[dst[i]:dst[i] + L] = seg
    return out


def sample_peptides(proteome: np.ndarray, n: int, length: int, error_rate: float,
                    seed: int) -> tuple[np.ndarray, np.ndarray]:
    """n peptides of `length` residues from uniform positions, each residue
    substituted (uniformly among the 20) with probability error_rate."""
    starts = randint(seed, 21, n, 0, proteome.size - length + 1)
    idx = starts[:, None] + np.arange(length)[None, :]
    seq = proteome[idx].reshape(-1).copy()
    mut = uniform01(seed, 22, 0, seq.size) < error_rate
    seq[mut] = AMINO[randint(seed, 23, int(mut.sum()), 0, 20)]
    return seq, fixed_length_offsets(n, length)


def random_peptides(n: int, length: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """n peptides of i.i.d. residues (the same frequencies)."""
    return protein_sequence(n * length, seed, dup_frac=0.0), fixed_length_offsets(n, length)
