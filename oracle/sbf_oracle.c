/*
 * sbf_oracle.c -- plain single-threaded CPU Super Bloom filter (the oracle).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.
 *
 * Every k-mer is handled on its own, in the order of Alg. 1 (insert) and
 * Alg. 2 (query) of the cuSBF paper: pack the k-mer, scan its k-m+1 m-mer
 * windows for the minimizer, pick the shard from the minimizer, then visit
 * its k-s+1 s-mers (Findere, Sec. II-B, Eq. 2) and set or test H bits of
 * each in that shard.  No rolling, no run sharing, no batching.
 *
 * Definition of the filter (the paper gives the structure but not the hash
 * constants; these readings are fixed here and in the CUDA library alike):
 *   code:      A/a=0, C/c=1, G/g=2, T/t=3, every other byte invalid.
 *   pack:      val(x_0..x_{L-1}) = sum c_i 4^(L-1-i), first base most
 *              significant (shift-and-OR, Sec. IV-C).
 *   canonical: every m-mer and every s-mer is replaced by min(val, val of
 *              its reverse complement); with canonical = 0 the forward value
 *              is used (the paper's literal behaviour).
 *   order key: minimizer order = one multiplicative mix (Sec. IV-G):
 *              (v * 0x9E3779B9) mod 2^32 when 2m <= 32, else
 *              (v * 0x9E3779B97F4A7C15) mod 2^64.  Both are bijections on the
 *              m-mer domain, so two different m-mers never tie.
 *   mix64:     the SplitMix64 finaliser (Steele, Lea, Flood 2014).
 *   shard:     x = floor(mix64(mu ^ 0x14057B7EF767814F) * N / 2^64).
 *   paper layout (layout = 1, Sec. IV-B and Alg. 1/2 taken literally):
 *              256-bit shards, N rounded up to a power of two, shard =
 *              order key of mu AND (N - 1), and every 64-bit word is its
 *              own sector (hash i in word i mod 4, b = 6), so for H < 4 some
 *              words of each shard stay unused.
 *   s-mer:     h = mix64(v ^ 0x5851F42D4C957F2D) (the stronger mix, Sec. IV-G).
 *   layout:    shard x owns bits [x*B, (x+1)*B) of a little-endian array of
 *              64-bit words.  W = B/64 words, S = the largest power of two
 *              not above min(H, W) sectors of B/S bits; hash i uses sector
 *              i mod S (Sec. IV-B: four equal sectors, hash i in sector i mod 4).
 *   bit:       b = log2(B/S), q = floor(64/H).  If q >= b, hash i takes bits
 *              [i*q, i*q+b) of h (bit-slicing); otherwise the top b bits of
 *              h * (0x9E3779B97F4A7C15 * (2i+1)) mod 2^64 (salted multiply,
 *              Sec. IV-G).
 *   insert:    set all (k-s+1)*H bits of every valid k-mer.
 *   query:     a valid k-mer is positive iff all its (k-s+1)*H bits are set
 *              (Findere rule; Contains of Alg. 2).
 *   valid:     a k-mer is valid iff its k bytes lie in one read and all are
 *              A/C/G/T (Sec. IV-C validity, Sec. IV-F separators).
 *   alphabets (Sec. IV-A: DNA 2 bits, protein 26 symbols in 5 bits, DNA
 *              triplets 64 symbols in 6 bits over 3 bytes): a symbol is one
 *              byte (DNA, protein: A..Z either case -> 0..25) or three
 *              (triplet: 16 c0 + 4 c1 + c2 of three DNA codes); the packed
 *              value, the sub-windows and the order key's width (32-bit when
 *              m symbols fit 32 bits) use the symbol width; a read's k-mers
 *              start at its first byte and then every symbol; the answer bit
 *              is the k-mer's first byte; non-DNA alphabets are forward only.
 */
#include "sbf_oracle.h"

#include <stdlib.h>
#include <string.h>

#define ORACLE_GOLDEN64 0x9E3779B97F4A7C15ULL
#define ORACLE_GOLDEN32 0x9E3779B9U
#define ORACLE_SPLITMIX_M1 0xBF58476D1CE4E5B9ULL
#define ORACLE_SPLITMIX_M2 0x94D049BB133111EBULL
#define ORACLE_SMER_KEY 0x5851F42D4C957F2DULL
#define ORACLE_SHARD_KEY 0x14057B7EF767814FULL

struct oracle_sbf {
  int k, m, s, H, B, canonical, layout;
  int alphabet;   /* 0 DNA, 1 protein, 2 DNA triplets */
  int sym_bits;   /* 2, 5, 6 */
  int sym_bytes;  /* 1, 1, 3 */
  uint64_t N;      /* shards */
  uint64_t words;  /* 64-bit words = N * B / 64 */
  uint64_t* bits;
};

static int base_code(uint8_t ch) {
  switch (ch) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
  }
}

/* Mask of the low `nbits` bits. */
static uint64_t bit_mask(int nbits) { return nbits >= 64 ? ~0ULL : ((1ULL << nbits) - 1ULL); }

/* Code of the symbol starting at x, or -1 if it is not in the alphabet. */
static int symbol_code(const oracle_sbf* f, const uint8_t* x) {
  if (f->alphabet == 1) {
    if (x[0] >= 'A' && x[0] <= 'Z') return x[0] - 'A';
    if (x[0] >= 'a' && x[0] <= 'z') return x[0] - 'a';
    return -1;
  }
  if (f->alphabet == 2) {
    int a = base_code(x[0]), b = base_code(x[1]), c = base_code(x[2]);
    if (a < 0 || b < 0 || c < 0) return -1;
    return 16 * a + 4 * b + c;
  }
  return base_code(x[0]);
}

/* PackKmer: shift-and-OR, first symbol most significant. */
static uint64_t pack_forward(const oracle_sbf* f, const uint8_t* x, int len) {
  uint64_t v = 0;
  for (int i = 0; i < len; ++i)
    v = (v << f->sym_bits) | (uint64_t)symbol_code(f, x + (size_t)i * (size_t)f->sym_bytes);
  return v;
}

/* Packed value of the reverse complement of x[0..len) (DNA only). */
static uint64_t pack_revcomp(const oracle_sbf* f, const uint8_t* x, int len) {
  if (f->alphabet != 0) return 0;
  uint64_t v = 0;
  for (int i = len - 1; i >= 0; --i) v = (v << 2) | (uint64_t)(3 - base_code(x[i]));
  return v;
}

/* Subwindow(packed, i, len) of Alg. 1: the len-mer at symbols [i, i+len). */
static uint64_t subwindow(const oracle_sbf* f, uint64_t packed, int i, int len) {
  return (packed >> (f->sym_bits * (f->k - len - i))) & bit_mask(f->sym_bits * len);
}

/* Reverse complement of bases [i, i+len), read off the reverse-complemented k-mer. */
static uint64_t subwindow_rc(uint64_t packed_rc, int i, int len) {
  return (packed_rc >> (2 * i)) & bit_mask(2 * len);
}

static uint64_t canonical_of(const oracle_sbf* f, uint64_t fwd, uint64_t rc) {
  if (!f->canonical) return fwd;
  return fwd < rc ? fwd : rc;
}

static uint64_t order_key(uint64_t v, int m_bits) {
  if (m_bits <= 32) return (uint64_t)((uint32_t)v * ORACLE_GOLDEN32);
  return v * ORACLE_GOLDEN64;
}

static uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= ORACLE_SPLITMIX_M1;
  x ^= x >> 27;
  x *= ORACLE_SPLITMIX_M2;
  x ^= x >> 31;
  return x;
}

static uint64_t order_key(uint64_t v, int m_bits);

static uint64_t shard_of(const oracle_sbf* f, uint64_t mu) {
  if (f->layout == 1) return order_key(mu, f->m * f->sym_bits) & (f->N - 1);  /* minHash & (NumShards - 1) */
  unsigned __int128 prod = (unsigned __int128)mix64(mu ^ ORACLE_SHARD_KEY) * f->N;
  return (uint64_t)(prod >> 64);
}

static int log2_exact(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return b;
}

/* Bit index inside the shard for hash function i of s-mer hash h. */
static int sector_count(const oracle_sbf* f, int H, int W) {
  if (f->layout == 1) return W;  /* one 64-bit word per sector */
  int lim = H < W ? H : W;
  int S = 1;
  while (2 * S <= lim) S *= 2;
  return S;
}

static uint64_t bit_in_shard(const oracle_sbf* f, uint64_t h, int i) {
  int W = f->B / 64;
  int S = sector_count(f, f->H, W);
  int sector_bits = f->B / S;
  int b = log2_exact(sector_bits);
  int q = 64 / f->H;
  uint64_t p;
  if (q >= b) {
    p = (h >> (i * q)) & (uint64_t)(sector_bits - 1);
  } else {
    uint64_t salt = ORACLE_GOLDEN64 * (uint64_t)(2 * i + 1);
    p = (h * salt) >> (64 - b);
  }
  return (uint64_t)(i % S) * (uint64_t)sector_bits + p;
}

/* Minimizer of the k-mer: the canonical m-mer with the smallest order key. */
static uint64_t minimizer(const oracle_sbf* f, uint64_t fwd, uint64_t rc) {
  uint64_t best_key = 0, mu = 0;
  for (int i = 0; i <= f->k - f->m; ++i) {
    uint64_t v = canonical_of(f, subwindow(f, fwd, i, f->m), subwindow_rc(rc, i, f->m));
    uint64_t key = order_key(v, f->m * f->sym_bits);
    if (i == 0 || key < best_key) {
      best_key = key;
      mu = v;
    }
  }
  return mu;
}

static uint64_t smer_hash(const oracle_sbf* f, uint64_t fwd, uint64_t rc, int t) {
  uint64_t v = canonical_of(f, subwindow(f, fwd, t, f->s), subwindow_rc(rc, t, f->s));
  return mix64(v ^ ORACLE_SMER_KEY);
}

static void insert_kmer(oracle_sbf* f, const uint8_t* x) {
  uint64_t fwd = pack_forward(f, x, f->k);
  uint64_t rc = pack_revcomp(f, x, f->k);
  uint64_t shard = shard_of(f, minimizer(f, fwd, rc));
  for (int t = 0; t <= f->k - f->s; ++t) {
    uint64_t h = smer_hash(f, fwd, rc, t);
    for (int i = 0; i < f->H; ++i) {
      uint64_t bit = shard * (uint64_t)f->B + bit_in_shard(f, h, i);
      f->bits[bit >> 6] |= 1ULL << (bit & 63);
    }
  }
}

static int query_kmer(const oracle_sbf* f, const uint8_t* x) {
  uint64_t fwd = pack_forward(f, x, f->k);
  uint64_t rc = pack_revcomp(f, x, f->k);
  uint64_t shard = shard_of(f, minimizer(f, fwd, rc));
  for (int t = 0; t <= f->k - f->s; ++t) {
    uint64_t h = smer_hash(f, fwd, rc, t);
    for (int i = 0; i < f->H; ++i) {
      uint64_t bit = shard * (uint64_t)f->B + bit_in_shard(f, h, i);
      if (!((f->bits[bit >> 6] >> (bit & 63)) & 1ULL)) return 0;
    }
  }
  return 1;
}

/* Bytes of a k-mer. */
static uint64_t kmer_bytes(const oracle_sbf* f) { return (uint64_t)f->k * (uint64_t)f->sym_bytes; }

/* A k-mer starting at p is valid iff it ends inside its read and all its
 * symbols are in the alphabet. */
static int kmer_valid(const oracle_sbf* f, const uint8_t* seq, uint64_t p, uint64_t read_end) {
  if (p + kmer_bytes(f) > read_end) return 0;
  for (int i = 0; i < f->k; ++i)
    if (symbol_code(f, seq + p + (uint64_t)i * (uint64_t)f->sym_bytes) < 0) return 0;
  return 1;
}

oracle_sbf* oracle_create(int k, int m, int s, int H, int shard_bits, int canonical,
                          uint64_t bits) {
  return oracle_create_layout(k, m, s, H, shard_bits, canonical, bits, 0);
}

oracle_sbf* oracle_create_layout(int k, int m, int s, int H, int shard_bits, int canonical,
                                 uint64_t bits, int layout) {
  return oracle_create_full(k, m, s, H, shard_bits, canonical, bits, layout, 0);
}

oracle_sbf* oracle_create_full(int k, int m, int s, int H, int shard_bits, int canonical,
                               uint64_t bits, int layout, int alphabet) {
  static const int sym_bits[3] = {2, 5, 6}, sym_bytes[3] = {1, 1, 3};
  if (alphabet < 0 || alphabet > 2) return NULL;
  if (alphabet != 0 && canonical) return NULL;               /* no reverse complement */
  if (k * sym_bits[alphabet] > 64) return NULL;              /* one 64-bit packed k-mer */
  if (layout != 0 && layout != 1) return NULL;
  if (layout == 1 && shard_bits != 256) return NULL;
  if (k < 1 || k > 32 || m < 1 || m > k || s < 1 || s > k || H < 1 || H > 16) return NULL;
  if (shard_bits != 256 && shard_bits != 512) return NULL;
  if (bits < (uint64_t)shard_bits) return NULL;
  oracle_sbf* f = (oracle_sbf*)calloc(1, sizeof(oracle_sbf));
  if (!f) return NULL;
  f->k = k; f->m = m; f->s = s; f->H = H; f->B = shard_bits; f->canonical = canonical ? 1 : 0;
  f->layout = layout;
  f->alphabet = alphabet;
  f->sym_bits = sym_bits[alphabet];
  f->sym_bytes = sym_bytes[alphabet];
  f->N = (bits + (uint64_t)shard_bits - 1) / (uint64_t)shard_bits;
  if (layout == 1) { /* round the shard count up to a power of two */
    uint64_t n = 1;
    while (n < f->N) n <<= 1;
    f->N = n;
  }
  f->words = f->N * (uint64_t)(shard_bits / 64);
  f->bits = (uint64_t*)calloc(f->words, sizeof(uint64_t));
  if (!f->bits) {
    free(f);
    return NULL;
  }
  return f;
}

void oracle_destroy(oracle_sbf* f) {
  if (!f) return;
  free(f->bits);
  free(f);
}

uint64_t oracle_num_shards(const oracle_sbf* f) { return f->N; }
uint64_t oracle_num_words(const oracle_sbf* f) { return f->words; }
uint64_t* oracle_words(oracle_sbf* f) { return f->bits; }

void oracle_insert(oracle_sbf* f, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                   uint64_t n_reads) {
  (void)seq_len;
  for (uint64_t r = 0; r < n_reads; ++r)
    for (uint64_t p = off[r]; p + kmer_bytes(f) <= off[r + 1]; p += (uint64_t)f->sym_bytes)
      if (kmer_valid(f, seq, p, off[r + 1])) insert_kmer(f, seq + p);
}

void oracle_query(const oracle_sbf* f, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                  uint64_t n_reads, uint32_t* out_bits, uint32_t* out_hits) {
  if (out_bits) memset(out_bits, 0, ((seq_len + 31) / 32) * sizeof(uint32_t));
  for (uint64_t r = 0; r < n_reads; ++r) {
    uint32_t hits = 0;
    for (uint64_t p = off[r]; p + kmer_bytes(f) <= off[r + 1]; p += (uint64_t)f->sym_bytes) {
      if (kmer_valid(f, seq, p, off[r + 1]) && query_kmer(f, seq + p)) {
        ++hits;
        if (out_bits) out_bits[p >> 5] |= 1U << (p & 31);
      }
    }
    if (out_hits) out_hits[r] = hits;
  }
}

/* Index of the read holding position p: the last r with off[r] <= p. */
static uint64_t read_of(const uint64_t* off, uint64_t n_reads, uint64_t p) {
  uint64_t lo = 0, hi = n_reads;  /* answer in [lo, hi) */
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

void oracle_query_positions(const oracle_sbf* f, const uint8_t* seq, uint64_t seq_len,
                            const uint64_t* off, uint64_t n_reads, const uint64_t* pos,
                            uint64_t n_pos, uint8_t* out) {
  for (uint64_t i = 0; i < n_pos; ++i) {
    uint64_t p = pos[i];
    out[i] = 0;
    if (p >= seq_len || n_reads == 0) continue;
    uint64_t r = read_of(off, n_reads, p);
    if (p < off[r] || p >= off[r + 1]) continue;
    if ((p - off[r]) % (uint64_t)f->sym_bytes != 0) continue;  /* not a symbol start */
    if (kmer_valid(f, seq, p, off[r + 1])) out[i] = (uint8_t)query_kmer(f, seq + p);
  }
}

void oracle_count_runs(const oracle_sbf* f, const uint8_t* seq, uint64_t seq_len,
                       const uint64_t* off, uint64_t n_reads, uint64_t* out_valid,
                       uint64_t* out_runs) {
  (void)seq_len;
  uint64_t valid = 0, runs = 0;
  for (uint64_t r = 0; r < n_reads; ++r) {
    int have_prev = 0;
    uint64_t prev_mu = 0;
    for (uint64_t p = off[r]; p + kmer_bytes(f) <= off[r + 1]; p += (uint64_t)f->sym_bytes) {
      if (!kmer_valid(f, seq, p, off[r + 1])) {
        have_prev = 0;
        continue;
      }
      uint64_t mu = minimizer(f, pack_forward(f, seq + p, f->k), pack_revcomp(f, seq + p, f->k));
      ++valid;
      if (!have_prev || mu != prev_mu) ++runs;
      have_prev = 1;
      prev_mu = mu;
    }
  }
  *out_valid = valid;
  *out_runs = runs;
}

void oracle_kmer_info(const oracle_sbf* f, const uint8_t* x, uint64_t* out_minimizer,
                      uint64_t* out_shard) {
  uint64_t mu = minimizer(f, pack_forward(f, x, f->k), pack_revcomp(f, x, f->k));
  *out_minimizer = mu;
  *out_shard = shard_of(f, mu);
}

uint64_t oracle_runs_of_keys(const uint64_t* keys, const uint8_t* active, uint64_t n) {
  uint64_t runs = 0;
  for (uint64_t i = 0; i < n; ++i) {
    if (!active[i]) continue;
    if (i == 0 || !active[i - 1] || keys[i - 1] != keys[i]) ++runs;
  }
  return runs;
}

uint64_t oracle_mix64(uint64_t x) { return mix64(x); }
