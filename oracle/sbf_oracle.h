/*
 * sbf_oracle.h -- plain single-threaded CPU Super Bloom filter (the oracle).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant with the CUDA library; the two are written separately from the same
 * definition of the filter (cuSBF paper: Sec. II-B, Sec. IV-B, Alg. 1, Alg. 2,
 * Sec. IV-G bit-slicing).
 *
 * Sequences are byte strings.  A batch of reads is one concatenated byte array
 * `seq` of length `seq_len` plus `n_reads + 1` offsets: read r is
 * seq[off[r], off[r+1]).  Offsets must be non-decreasing with off[0] = 0 and
 * off[n_reads] = seq_len.
 *
 * Query answers are bit-packed by start position in `seq`: bit p of the
 * uint32 array (word p >> 5, bit p & 31) is the answer for the k-mer starting
 * at p; it is 0 where no valid k-mer starts.  hits[r] counts the positive
 * k-mers of read r.
 */
#ifndef SBF_ORACLE_H
#define SBF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_sbf oracle_sbf;

/* Returns NULL on invalid parameters (same domain as the library). */
oracle_sbf* oracle_create(int k, int m, int s, int H, int shard_bits, int canonical,
                          uint64_t bits);
/* layout 0: this library's layout (the default); layout 1: the paper's
 * literal layout (256-bit shards only; N rounded up to a power of two, shard
 * = minimizer order key & (N - 1), hash i in 64-bit word i mod 4). */
oracle_sbf* oracle_create_layout(int k, int m, int s, int H, int shard_bits, int canonical,
                                 uint64_t bits, int layout);
/* alphabet 0: DNA (2-bit symbols, one byte each, the default); 1: protein
 * (A..Z either case, 5-bit symbols); 2: DNA triplets (three DNA bytes per
 * 6-bit symbol; a read's k-mers start at its first byte and every third
 * byte after).  Non-DNA alphabets need canonical = 0 and k * bits <= 64. */
oracle_sbf* oracle_create_full(int k, int m, int s, int H, int shard_bits, int canonical,
                               uint64_t bits, int layout, int alphabet);
void oracle_destroy(oracle_sbf* f);

uint64_t oracle_num_shards(const oracle_sbf* f);
uint64_t oracle_num_words(const oracle_sbf* f);     /* 64-bit words */
uint64_t* oracle_words(oracle_sbf* f);               /* the bit array */

void oracle_insert(oracle_sbf* f, const uint8_t* seq, uint64_t seq_len,
                   const uint64_t* off, uint64_t n_reads);

/* out_bits: ceil(seq_len / 32) words (overwritten); out_hits: n_reads (overwritten).
 * Either may be NULL. */
void oracle_query(const oracle_sbf* f, const uint8_t* seq, uint64_t seq_len,
                  const uint64_t* off, uint64_t n_reads, uint32_t* out_bits,
                  uint32_t* out_hits);

/* Answers for chosen start positions only (sampled parity at large sizes).
 * out[i] = answer for the k-mer starting at pos[i] (0 if none valid). */
void oracle_query_positions(const oracle_sbf* f, const uint8_t* seq, uint64_t seq_len,
                            const uint64_t* off, uint64_t n_reads, const uint64_t* pos,
                            uint64_t n_pos, uint8_t* out);

/* Super-k-mer statistics: valid k-mers and maximal runs of consecutive valid
 * k-mers of one read that share a minimizer (Sec. II-B). */
void oracle_count_runs(const oracle_sbf* f, const uint8_t* seq, uint64_t seq_len,
                       const uint64_t* off, uint64_t n_reads, uint64_t* out_valid,
                       uint64_t* out_runs);

/* Minimizer (canonical m-mer value) and shard of the k-mer at x[0..k). */
void oracle_kmer_info(const oracle_sbf* f, const uint8_t* x, uint64_t* out_minimizer,
                      uint64_t* out_shard);

/* Run count of a lane sequence as in the segmented reduction of Fig. 4:
 * keys[i] is lane i's shard, active[i] its validity; a run is a maximal span
 * of consecutive active lanes with equal keys. */
uint64_t oracle_runs_of_keys(const uint64_t* keys, const uint8_t* active, uint64_t n);

/* The 64-bit finaliser every hash of the filter goes through (the SplitMix64
 * output function of Steele, Lea and Flood, 2014; Sec. IV-G's "stronger mix
 * with an additional xorshift").  Exported so that tests can pin it to the
 * published generator's outputs. */
uint64_t oracle_mix64(uint64_t x);

#ifdef __cplusplus
}
#endif

#endif
