"""Pins of the oracle to facts outside itself (no GPU).

Each test ties the C oracle to the paper or to mathematics: closed forms of
the packing, the brute-force string-level filter, invariants of canonical
k-mers and of OR-insertion, the minimizer density of Sec. II-B, Eq. 1 / Eq. 2
and their shard-aware forms under an exact binomial test, the blocked-Bloom
reduction s = k, and the worked examples of Fig. 2 and Fig. 4.
"""
import json
import os
import random

import numpy as np
import pytest

from bruteforce import BruteSBF, revcomp
from oracle import OracleSBF
from oracle.fpr import (binomial_two_sided_p, blocked_bloom_fpr, bloom_fpr,
                        conditional_fpr, sector_fill, sector_layout)
from oracle.oracle import runs_of_keys
from paper_2606_24417_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def _reads_to_arrays(reads):
    return synth.concat([np.frombuffer(r.encode(), dtype=np.uint8) for r in reads])


def _random_dna(rng, n, alphabet="ACGT"):
    return "".join(rng.choice(alphabet) for _ in range(n))


# ---------------------------------------------------------------------------
# the 64-bit finaliser: known answers of the published SplitMix64 generator
# ---------------------------------------------------------------------------
def test_mix64_matches_published_splitmix64_outputs():
    """Every hash of the filter (shard choice and s-mer bits, Sec. IV-G) goes
    through the oracle's mix64, the output function of SplitMix64.  The
    generator's published first outputs for two seeds pin all five of its
    steps (three xor-shifts and two multipliers): a transposed constant or
    a wrong shift changes every output."""
    from oracle.oracle import mix64

    kat = _golden("splitmix64_kat.json")
    gamma = int(kat["gamma"], 16)
    for stream in kat["streams"]:
        want = stream.get("outputs") or [int(h, 16) for h in stream["outputs_hex"]]
        state = stream["seed"]
        for expected in want:
            state = (state + gamma) & 0xFFFFFFFFFFFFFFFF
            assert mix64(state) == expected


# ---------------------------------------------------------------------------
# packing and canonical values: closed forms of val = sum c_i 4^(L-1-i)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kmer,canonical,expected", [
    ("ACGT", True, 0b00011011),     # palindrome: rc(ACGT) = ACGT
    ("AAAA", True, 0),
    ("TTTT", True, 0),              # rc(TTTT) = AAAA
    ("TTTT", False, 255),
    ("CAAA", True, 64),             # fwd 1*4^3 = 64 < rc TTTG = 254
    ("TTTG", True, 64),
    ("GGGG", True, 85),             # rc = CCCC = 0b01010101
    ("acgt", True, 27),             # lower case is the same base
])
def test_packing_closed_form(kmer, canonical, expected):
    # with m = k the minimizer is the canonical k-mer itself (w = 1)
    f = OracleSBF(k=4, m=4, s=4, H=1, bits=512, canonical=canonical)
    mu, shard = f.kmer_info(np.frombuffer(kmer.encode(), dtype=np.uint8))
    assert mu == expected
    assert 0 <= shard < f.n_shards


def test_minimizer_is_min_over_windows_k32():
    # k = 32 uses all 64 bits of the packed k-mer
    rng = random.Random(3)
    f = OracleSBF(k=32, m=16, s=32, H=2, bits=1 << 16)
    b = BruteSBF(32, 16, 32, 2, 1 << 16)
    for _ in range(50):
        km = _random_dna(rng, 32)
        mu, shard = f.kmer_info(np.frombuffer(km.encode(), dtype=np.uint8))
        assert mu == b.minimizer(km)
        assert shard == b.shard(km)


# ---------------------------------------------------------------------------
# brute force on tiny inputs
# ---------------------------------------------------------------------------
CONFIGS = [
    # k, m, s, H, bits, B, canonical
    (9, 5, 6, 2, 4096, 256, True),        # Fig. 2 parameters
    (31, 16, 28, 4, 1 << 16, 512, True),  # the paper's operating point, 512-bit shards
    (31, 16, 28, 4, 1 << 15, 256, True),  # the paper's 256-bit layout
    (31, 12, 24, 8, 1 << 15, 256, True),
    (31, 20, 31, 1, 1 << 14, 512, True),  # m > 16: 64-bit order key; s = k
    (31, 14, 26, 2, 1 << 14, 512, False),  # forward-only (paper literal)
    (31, 16, 28, 16, 1 << 16, 512, True),  # q = 4 < b: salted multiply
    (21, 11, 17, 12, 5000, 512, True),     # non power-of-two shard count
    (32, 16, 30, 4, 1 << 15, 512, True),   # k = 32
    (31, 16, 28, 3, 1 << 15, 512, True),   # H = 3: two sectors
    (31, 16, 28, 6, 1 << 15, 256, True),   # H = 6: four sectors, two slices share one
    # the paper's literal layout (layout 1): 2^P shards, key & (N - 1), word sectors
    (31, 16, 28, 4, 1 << 15, 256, False, 1),  # the paper's operating point, forward only
    (31, 16, 28, 2, 3000 * 256, 256, False, 1),  # N rounded up; words 2, 3 unused
    (31, 16, 28, 12, 1 << 15, 256, True, 1),  # q = 5 < 6: salted multiply
    (31, 16, 28, 16, 1 << 15, 256, False, 1),  # q = 4
    (31, 20, 31, 8, 1 << 14, 256, True, 1),   # 64-bit order key
    (9, 5, 6, 2, 4096, 256, False, 1),        # Fig. 2 parameters
]


def _tiny_reads(rng, k):
    reads = [_random_dna(rng, rng.randint(0, 3 * k)) for _ in range(12)]
    reads.append(_random_dna(rng, 2 * k, "ACGTN"))       # invalid bases inside
    reads.append(_random_dna(rng, k - 1))                 # shorter than k
    reads.append("")                                      # empty read
    reads.append(_random_dna(rng, k).lower())             # lower case
    reads.append("A" * (2 * k))                           # homopolymer: one long run
    return reads


@pytest.mark.parametrize("cfg", CONFIGS)
def test_bruteforce_filter_and_answers(cfg):
    k, m, s, H, bits, B, canon, *rest = cfg
    layout = rest[0] if rest else 0
    rng = random.Random(hash(cfg) & 0xFFFF)
    reads = _tiny_reads(rng, k)
    seq, off = _reads_to_arrays(reads)
    f = OracleSBF(k, m, s, H, bits, shard_bits=B, canonical=canon, layout=layout)
    f.insert(seq, off)
    b = BruteSBF(k, m, s, H, bits, shard_bits=B, canonical=canon, layout=layout)
    for r in reads:
        b.insert_read(r)
    assert np.array_equal(f.words(), b.words())

    # queries: the inserted reads, their reverse complements, mutants, random reads
    qreads = list(reads) + [revcomp(r) for r in reads if r]
    for r in reads:
        if len(r) >= k:
            i = rng.randrange(len(r))
            qreads.append(r[:i] + rng.choice("ACGT") + r[i + 1:])
    qreads += [_random_dna(rng, rng.randint(k, 3 * k)) for _ in range(20)]
    qseq, qoff = _reads_to_arrays(qreads)
    bits_out, hits = f.query(qseq, qoff)
    bitset = b.bitset()
    for ri, r in enumerate(qreads):
        n_pos = 0
        for p in range(len(r)):
            gp = int(qoff[ri]) + p
            got = (int(bits_out[gp >> 5]) >> (gp & 31)) & 1
            km = r[p:p + k]
            want = 0
            if len(km) == k and all(ch in "ACGTacgt" for ch in km):
                want = int(b.query_kmer(km, bitset))
            assert got == want, (cfg, ri, p)
            n_pos += want
        assert hits[ri] == n_pos


def test_sparse_filter_exact_membership():
    """With s = k and a sparse filter, an alien k-mer is positive iff its
    (shard, s-mer) pair was inserted or its H bits collide in its shard; the
    brute force tells the two apart, and inserted k-mers are exact members."""
    k, m, s, H = 31, 16, 31, 4
    rng = random.Random(11)
    inserted = [_random_dna(rng, k) for _ in range(200)]
    seq, off = _reads_to_arrays(inserted)
    f = OracleSBF(k, m, s, H, 1 << 24)
    f.insert(seq, off)
    b = BruteSBF(k, m, s, H, 1 << 24)
    for r in inserted:
        b.insert_read(r)
    aliens = [_random_dna(rng, k) for _ in range(2000)]
    qseq, qoff = _reads_to_arrays(inserted + aliens)
    _, hits = f.query(qseq, qoff)
    assert hits[:200].tolist() == [1] * 200
    bitset = b.bitset()
    for j, a in enumerate(aliens):
        exact = b.query_kmer_exact(a)
        collide = b.query_kmer(a, bitset)
        assert hits[200 + j] == int(exact or collide)
        assert not exact  # random 31-mers are not in a set of 200


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def _genome(n, seed):
    return synth.uniform_dna(n, seed)


def test_no_false_negatives_and_revcomp_invariance():
    g = _genome(200_000, 4)
    off = np.array([0, g.size], dtype=np.uint64)
    f1 = OracleSBF(31, 16, 28, 4, 1 << 22)
    f1.insert(g, off)
    bits, hits = f1.query(g, off)
    assert int(hits[0]) == g.size - 31 + 1          # every inserted k-mer is positive
    # inserting the reverse strand gives the identical filter (canonical m/s-mers)
    rc = synth.reverse_complement(g)
    f2 = OracleSBF(31, 16, 28, 4, 1 << 22)
    f2.insert(rc, off)
    assert np.array_equal(f1.words(), f2.words())
    # query(rc(read)) = reversed answers of query(read)
    reads, roff = synth.sample_reads(g, 300, 150, 0.02, seed=9)
    rb, rh = f1.query(reads, roff)
    rcs = [synth.reverse_complement(reads[int(roff[i]):int(roff[i + 1])]) for i in range(300)]
    rseq, roff2 = synth.concat(rcs)
    qb, qh = f1.query(rseq, roff2)
    assert np.array_equal(rh, qh)
    ub = np.unpackbits(rb.view(np.uint8), bitorder="little")[: reads.size].reshape(300, 150)
    uq = np.unpackbits(qb.view(np.uint8), bitorder="little")[: rseq.size].reshape(300, 150)
    L = 150 - 31 + 1
    assert np.array_equal(ub[:, :L], uq[:, :L][:, ::-1])


def test_insert_order_split_and_idempotence():
    g = _genome(50_000, 5)
    off = np.array([0, g.size], dtype=np.uint64)
    ref = OracleSBF(31, 16, 28, 4, 1 << 20)
    ref.insert(g, off)
    # split into pieces overlapping by k-1, inserted in shuffled order, twice
    rng = random.Random(1)
    cuts = sorted(rng.sample(range(100, g.size - 100), 40))
    pieces = []
    start = 0
    for c in cuts + [g.size]:
        pieces.append(g[max(0, start - 30):c])
        start = c
    rng.shuffle(pieces)
    seq, poff = synth.concat(pieces)
    f = OracleSBF(31, 16, 28, 4, 1 << 20)
    f.insert(seq, poff)
    f.insert(seq, poff)
    assert np.array_equal(ref.words(), f.words())


def test_invalid_and_short_reads_give_zero():
    f = OracleSBF(31, 16, 28, 4, 1 << 20)
    good = synth.uniform_dna(100, 1)
    f.insert(good, np.array([0, 100], dtype=np.uint64))
    bad = good.copy()
    bad[50] = ord("N")
    seq, off = synth.concat([good[:30], bad, good[:0], good])
    bits, hits = f.query(seq, off)
    assert hits.tolist() == [0, 100 - 31 + 1 - 31, 0, 100 - 31 + 1]
    # no bit is set for a k-mer covering the N or crossing a read boundary
    u = np.unpackbits(bits.view(np.uint8), bitorder="little")[: seq.size]
    p0 = int(off[1])
    assert u[:p0].sum() == 0
    assert u[p0 + 20:p0 + 51].sum() == 0
    assert u[p0 + 70:p0 + 100].sum() == 0


# ---------------------------------------------------------------------------
# Sec. II-B: density of random minimizers, mean super-k-mer length (w+1)/2
# ---------------------------------------------------------------------------
def test_minimizer_density_matches_paper():
    gold = _golden("density.json")
    g = _genome(1_000_000, 0)
    off = np.array([0, g.size], dtype=np.uint64)
    for case in gold["cases"]:
        f = OracleSBF(gold["k"], case["m"], 28, 4, 1 << 24)
        valid, runs = f.count_runs(g, off)
        assert valid == g.size - 30
        mean_len = valid / runs
        assert abs(mean_len / case["mean_run_length"] - 1) < 0.03, (case, mean_len)


# ---------------------------------------------------------------------------
# Eq. 1, Eq. 2 and the shard-aware closed form, exact binomial tests
# ---------------------------------------------------------------------------
def _alien_kmers(n, seed, k=31):
    return synth.random_reads(n, k, seed)


@pytest.mark.parametrize("bits,H,B,s", [
    (1 << 22, 4, 512, 28),
    (1 << 23, 4, 512, 28),
    (1 << 22, 8, 256, 28),
    (1 << 21, 2, 512, 24),
    (1 << 22, 1, 512, 31),
])
def test_fpr_matches_conditional_closed_form(bits, H, B, s):
    g = _genome(1_000_000, 0)
    f = OracleSBF(31, 16, s, H, bits, shard_bits=B)
    f.insert(g, np.array([0, g.size], dtype=np.uint64))
    p_hat = conditional_fpr(f.words(), 31, s, H, B)
    Q = 1_000_000
    qseq, qoff = _alien_kmers(Q, seed=77)
    _, hits = f.query(qseq, qoff)
    X = int(hits.sum())
    assert p_hat > 1e-4
    assert binomial_two_sided_p(X, Q, p_hat) > 1e-4, (X, Q * p_hat)


def _paper_shards_numpy(qseq, Q, k, m, n_shards, canonical):
    """Shards of Q length-k reads under layout 1, vectorised in numpy from the
    definition (a third implementation, sharing nothing with the C oracle):
    minimizer = m-mer of least key (v * 0x9E3779B9) mod 2^32, shard = key & (N - 1)."""
    code = np.full(256, 0, dtype=np.uint64)
    for ch, c in zip(b"ACGTacgt", (0, 1, 2, 3, 0, 1, 2, 3)):
        code[ch] = c
    x = code[np.asarray(qseq, dtype=np.uint8).reshape(Q, k)]
    best_key = None
    for i in range(k - m + 1):
        fwd = np.zeros(Q, dtype=np.uint64)
        rc = np.zeros(Q, dtype=np.uint64)
        for j in range(m):
            fwd = (fwd << np.uint64(2)) | x[:, i + j]
            rc = rc | ((np.uint64(3) - x[:, i + j]) << np.uint64(2 * j))
        v = np.minimum(fwd, rc) if canonical else fwd
        key = (v * np.uint64(0x9E3779B9)) & np.uint64(0xFFFFFFFF)
        best_key = key if best_key is None else np.minimum(best_key, key)
    return (best_key & np.uint64(n_shards - 1)).astype(np.int64)


@pytest.mark.parametrize("bits,H,s,canonical", [
    (1 << 22, 4, 28, False),
    (1 << 22, 2, 28, True),
    (3 << 20, 8, 26, False),   # 12,288 shards rounded up to 16,384
])
def test_paper_layout_fpr_matches_conditional_closed_form(bits, H, s, canonical):
    """Layout 1 under the shard-aware form of Eq. 2, conditioned on each
    alien's shard: with shardIdx = minHash & (N - 1) an alien's shard is not
    uniform (minimizer suffixes are biased and the same bias loads those
    shards more), so the uniform-shard average understates the rate by a few
    percent.  Given the shards, the alien's s-mers are independent of the
    filter and X has mean sum_q g(x_q) and variance sum_q g(1 - g), with
    g(x) = prod_j f[x, j]^((k-s+1) c_j)."""
    g = _genome(1_000_000, 0)
    f = OracleSBF(31, 16, s, H, bits, shard_bits=256, canonical=canonical, layout=1)
    f.insert(g, np.array([0, g.size], dtype=np.uint64))
    Q = 1_000_000
    qseq, qoff = _alien_kmers(Q, seed=78)
    _, hits = f.query(qseq, qoff)
    X = int(hits.sum())
    _, _, c = sector_layout(H, 256, layout=1)
    fill = sector_fill(f.words(), H, 256, layout=1)
    used = c > 0
    gx = np.prod(fill[:, used] ** ((31 - s + 1) * c[None, used]), axis=1)
    shards = _paper_shards_numpy(qseq, Q, 31, 16, f.n_shards, canonical)
    mean = float(gx[shards].sum())
    sd = float((gx[shards] * (1 - gx[shards])).sum()) ** 0.5
    assert mean > 100
    assert abs(X - mean) <= 4.5 * sd + 3, (X, mean, sd)
    # the uniform-shard form is the same quantity averaged over all shards
    p_uniform = conditional_fpr(f.words(), 31, s, H, 256, layout=1)
    assert abs(p_uniform - float(gx.mean())) <= 1e-12 + 1e-9 * p_uniform


def test_paper_layout_shard_count_and_unused_words():
    """Sec. IV-B: 2^P shards (count rounded up), hash i in 64-bit word i mod 4,
    so with H < 4 words H..3 of every shard are never set."""
    g = _genome(100_000, 9)
    off = np.array([0, g.size], dtype=np.uint64)
    for H in (1, 2, 3, 4):
        f = OracleSBF(31, 16, 28, H, 5000 * 256, shard_bits=256, layout=1)
        assert f.n_shards == 8192
        f.insert(g, off)
        w = f.words().reshape(-1, 4)
        for j in range(4):
            assert (np.count_nonzero(w[:, j]) > 0) == (j < H), (H, j)


def test_paper_layout_shard_depends_on_minimizer_suffix():
    """shardIdx = minHash & (N - 1) with a multiplicative minHash (Alg. 1): the
    low P bits of v * C (C odd) depend only on the low P bits of v, so k-mers
    whose minimizers end in the same P/2 bases share a shard, and distinct
    minimizer suffixes map to distinct shards (C odd is invertible mod 2^P)."""
    rng = random.Random(11)
    f = OracleSBF(31, 16, 28, 4, 1 << 20, shard_bits=256, canonical=False, layout=1)
    P = f.n_shards.bit_length() - 1
    assert f.n_shards == 1 << P
    by_suffix = {}
    for _ in range(3000):
        km = _random_dna(rng, 31)
        mu, x = f.kmer_info(np.frombuffer(km.encode(), dtype=np.uint8))
        by_suffix.setdefault(mu & ((1 << P) - 1), set()).add(x)
    assert all(len(v) == 1 for v in by_suffix.values())
    shards = [next(iter(v)) for v in by_suffix.values()]
    assert len(set(shards)) == len(shards)


def test_blocked_bloom_reduction_s_equals_k():
    """s = k leaves one s-mer per k-mer: a blocked Bloom filter (Sec. II-A).
    Independent random k-mers have independent uniform shards, so the rate
    follows the Poisson-load blocked-Bloom formula."""
    n = 60_000
    for H, B, bits in [(1, 512, 1 << 16), (4, 512, 1 << 17), (2, 256, 1 << 16)]:
        seq, off = _alien_kmers(n, seed=5)
        f = OracleSBF(31, 16, 31, H, bits, shard_bits=B)
        f.insert(seq, off)
        prior = blocked_bloom_fpr(n, f.n_shards, H, B)
        Q = 200_000
        qseq, qoff = _alien_kmers(Q, seed=6)
        _, hits = f.query(qseq, qoff)
        X = int(hits.sum())
        # the filter's own fill fluctuates around the prior: allow the binomial
        # spread of X plus 3% for the fill's randomness
        sd = (Q * prior * (1 - prior)) ** 0.5
        assert abs(X - Q * prior) <= 4 * sd + 0.03 * Q * prior, (H, B, X, Q * prior)
        p_hat = conditional_fpr(f.words(), 31, 31, H, B)
        assert binomial_two_sided_p(X, Q, p_hat) > 1e-4


def test_eq1_single_shard_standard_bloom():
    """One shard, s = k, H = 1: a standard Bloom filter with M = 512 bits; its
    fill fraction is Eq. 1's eps = 1 - exp(-n/M) up to the fill's binomial spread."""
    for n in (100, 300, 800):
        seq, off = _alien_kmers(n, seed=n)
        f = OracleSBF(31, 16, 31, 1, 512)
        f.insert(seq, off)
        fill = np.unpackbits(f.words().view(np.uint8)).mean()
        eps = bloom_fpr(1, n, 512)
        assert abs(fill - eps) < 4 * (eps * (1 - eps) / 512) ** 0.5 + 0.01


def test_findere_ordering_and_almost_aliens():
    """Sec. V-D ordering at a fixed budget: s = 28 beats s = 30 beats s = 31;
    and (Sec. II-B) a one-base mutant of an inserted k-mer is positive far more
    often than a random alien when the mutation sits in a single s-mer."""
    g = _genome(500_000, 8)
    off = np.array([0, g.size], dtype=np.uint64)
    Q = 300_000
    qseq, qoff = _alien_kmers(Q, seed=12)
    rates = {}
    for s in (28, 30, 31):
        f = OracleSBF(31, 16, s, 4, 1 << 22)
        f.insert(g, off)
        rates[s] = float(f.query(qseq, qoff)[1].mean())
    assert rates[28] < rates[30] < rates[31]
    f = OracleSBF(31, 16, 28, 4, 1 << 22)
    f.insert(g, off)
    mseq, moff = synth.sample_reads(g, 100_000, 31, 0.0, seed=13)
    mseq = mseq.reshape(-1, 31).copy()
    acgt = np.frombuffer(b"ACGT", dtype=np.uint8)
    col = 0   # an end base lies in one s-mer only: the mutant keeps z of z+1
    code = np.searchsorted(acgt, mseq[:, col])
    mseq[:, col] = acgt[(code + 1) % 4]
    mut_rate = float(f.query(mseq.reshape(-1), moff)[1].mean())
    assert mut_rate > 10 * rates[28]


# ---------------------------------------------------------------------------
# worked examples of the paper
# ---------------------------------------------------------------------------
def test_fig2_worked_example_counts():
    gold = _golden("fig2_minimizer_findere.json")
    k, m, s = gold["k"], gold["m"], gold["s"]
    f = OracleSBF(k, m, s, 2, 4096, shard_bits=256)
    seq = np.frombuffer(gold["sequence"].encode(), dtype=np.uint8)
    valid, runs = f.count_runs(seq, np.array([0, seq.size], dtype=np.uint64))
    assert valid == len(gold["kmers"])
    b = BruteSBF(k, m, s, 2, 4096, shard_bits=256)
    for p, km in enumerate(gold["kmers"]):
        assert gold["sequence"][p:p + k] == km
        assert len(b.smers(km)) == gold["smers_per_kmer"] == k - s + 1
        assert k - m + 1 == gold["mmers_per_kmer"]
    assert 1 <= runs <= valid


def test_fig4_segmented_reduction_counts():
    gold = _golden("fig4_segmented_reduction.json")
    ids = {"A": 1, "B": 2, "C": 3, "sentinel": 99}
    keys = [ids[x] for x in gold["lane_shards"]]
    runs = runs_of_keys(keys, gold["active"])
    assert runs == gold["runs"]
    W = gold["words_per_shard"]
    assert sum(gold["active"]) * W == gold["atomics_without_reduction"]
    assert runs * W == gold["atomics_with_reduction"]


def test_oracle_regression_digests():
    """The oracle still produces the digests its committed script recorded."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    stored = _golden("oracle_regression.json")["cases"]
    assert mod.compute() == stored


# ---------------------------------------------------------------------------
# other alphabets (Sec. IV-A): protein (26 symbols, 5 bits) and DNA triplets
# (64 symbols, 6 bits, three bytes each)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("alphabet,kmer,expected", [
    ("protein", "ACD", 0 * 1024 + 2 * 32 + 3),     # A=0, C=2, D=3 in 5-bit digits
    ("protein", "acd", 0 * 1024 + 2 * 32 + 3),     # either case
    ("protein", "ZZZ", 25 * 1024 + 25 * 32 + 25),
    ("dna_triplet", "AAAACG", 0 * 64 + 6),         # AAA = 0, ACG = 16*0 + 4*1 + 2
    ("dna_triplet", "TTTTTT", 63 * 64 + 63),
])
def test_alphabet_packing_closed_form(alphabet, kmer, expected):
    k = 3 if alphabet == "protein" else 2
    f = OracleSBF(k, k, k, 1, 512, canonical=False, alphabet=alphabet)
    mu, _ = f.kmer_info(np.frombuffer(kmer.encode(), dtype=np.uint8))
    assert mu == expected


def _protein_reads(rng, k):
    letters = "ACDEFGHIKLMNPQRSTVWYXBZUOJ"
    reads = ["".join(rng.choice(letters) for _ in range(rng.randint(0, 4 * k))) for _ in range(12)]
    reads.append("".join(rng.choice(letters + "*-.1") for _ in range(3 * k)))  # invalid symbols
    reads.append("".join(rng.choice(letters) for _ in range(k - 1)))           # shorter than k
    reads.append("")
    reads.append("".join(rng.choice(letters) for _ in range(2 * k)).lower())
    reads.append("W" * (3 * k))
    return reads


def _triplet_reads(rng, k):
    reads = [_random_dna(rng, rng.randint(0, 12 * k)) for _ in range(12)]  # lengths not multiples of 3
    reads.append(_random_dna(rng, 9 * k, "ACGTN"))
    reads.append(_random_dna(rng, 3 * k - 1))                               # one byte short
    reads.append("")
    reads.append(_random_dna(rng, 6 * k).lower())
    return reads


ALPHA_CONFIGS = [
    # k, m, s, H, bits, B, layout, alphabet
    (12, 6, 10, 4, 1 << 15, 512, 0, 1),
    (12, 7, 12, 1, 1 << 14, 512, 0, 1),    # s = k; 35-bit m-mers: 64-bit key
    (10, 4, 8, 8, 1 << 15, 256, 0, 1),
    (12, 6, 9, 16, 1 << 15, 512, 0, 1),    # salted multiply
    (12, 6, 10, 4, 1 << 15, 256, 1, 1),    # the paper's layout
    (10, 5, 8, 4, 1 << 15, 512, 0, 2),
    (10, 6, 10, 2, 1 << 14, 512, 0, 2),    # 36-bit m-mers: 64-bit key
    (8, 4, 6, 4, 1 << 14, 256, 1, 2),
]


@pytest.mark.parametrize("cfg", ALPHA_CONFIGS, ids=lambda c: "_".join(map(str, c)))
def test_alphabet_bruteforce_filter_and_answers(cfg):
    k, m, s, H, bits, B, layout, alphabet = cfg
    rng = random.Random(hash(cfg) & 0xFFFF)
    reads = _protein_reads(rng, k) if alphabet == 1 else _triplet_reads(rng, k)
    seq, off = _reads_to_arrays(reads)
    f = OracleSBF(k, m, s, H, bits, shard_bits=B, canonical=False, layout=layout, alphabet=alphabet)
    f.insert(seq, off)
    b = BruteSBF(k, m, s, H, bits, shard_bits=B, canonical=False, layout=layout, alphabet=alphabet)
    for r in reads:
        b.insert_read(r)
    assert np.array_equal(f.words(), b.words())
    # queries: the reads, one-symbol mutants, shifted copies and random reads
    qreads = list(reads)
    for r in reads:
        if len(r) > 3:
            i = rng.randrange(len(r))
            qreads.append(r[:i] + rng.choice("ACGT") + r[i + 1:])
            qreads.append(r[1:])  # a triplet read out of frame
    qreads += (_protein_reads(rng, k) if alphabet == 1 else _triplet_reads(rng, k))
    qseq, qoff = _reads_to_arrays(qreads)
    bits_out, hits = f.query(qseq, qoff)
    bitset = b.bitset()
    for ri, r in enumerate(qreads):
        want = {p: int(b.query_kmer(km, bitset)) for p, km in b.kmers_of(r)}
        for p in range(len(r)):
            gp = int(qoff[ri]) + p
            got = (int(bits_out[gp >> 5]) >> (gp & 31)) & 1
            assert got == want.get(p, 0), (cfg, ri, p)
        assert hits[ri] == sum(want.values())
    # every inserted k-mer is positive (no false negatives)
    _, ih = f.query(seq, off)
    assert [int(x) for x in ih] == [sum(1 for _ in b.kmers_of(r)) for r in reads]


def test_triplet_frame_and_valid_counts():
    """Triplet k-mers start at a read's first byte and every third byte after
    (Sec. IV-A multi-byte symbols): runs counted by the oracle match the
    string-level reading frame."""
    rng = random.Random(5)
    reads = [_random_dna(rng, n) for n in (29, 30, 31, 32, 90, 91, 92, 300)]
    seq, off = _reads_to_arrays(reads)
    f = OracleSBF(10, 5, 8, 4, 1 << 16, canonical=False, alphabet="dna_triplet")
    b = BruteSBF(10, 5, 8, 4, 1 << 16, canonical=False, alphabet=2)
    valid, _ = f.count_runs(seq, off)
    assert valid == sum(max(0, len(r) // 3 - 10 + 1) for r in reads)
    assert valid == sum(1 for r in reads for _ in b.kmers_of(r))
    f.insert(seq, off)
    bits_out, hits = f.query(seq, off)
    for ri, r in enumerate(reads):
        for p in range(len(r)):
            gp = int(off[ri]) + p
            bit = (int(bits_out[gp >> 5]) >> (gp & 31)) & 1
            assert bit == int(p % 3 == 0 and p + 30 <= len(r)), (ri, p)


def test_protein_fpr_matches_conditional_closed_form():
    """Eq. 2 made shard-aware holds for 5-bit symbols: random aliens against a
    filter built from a random 'proteome'."""
    from paper_2606_24417_gb300 import synth as sy

    letters = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", dtype=np.uint8)
    prot = letters[sy.randint(8, 1, 400_000, 0, 20)]
    f = OracleSBF(12, 6, 10, 4, 1 << 21, canonical=False, alphabet="protein")
    f.insert(prot, np.array([0, prot.size], dtype=np.uint64))
    p_hat = conditional_fpr(f.words(), 12, 10, 4, 512)
    Q = 300_000
    q = letters[sy.randint(9, 1, Q * 12, 0, 20)]
    qoff = np.arange(0, Q * 12 + 1, 12, dtype=np.uint64)
    _, hits = f.query(q, qoff)
    X = int(hits.sum())
    assert p_hat > 1e-4
    assert binomial_two_sided_p(X, Q, p_hat) > 1e-4, (X, Q * p_hat)
