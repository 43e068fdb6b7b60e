/*
 * sbf.h -- C ABI of the GB300 Super Bloom filter library (libsbf.so).
 *
 * A Super Bloom filter (SBF; cuSBF paper, Sec. II-B) stores DNA k-mers.  A
 * k-mer's minimizer (the m-mer of smallest order key among its k-m+1 windows)
 * picks one shard of shard_bits bits; each of the k-mer's k-s+1 s-mers sets
 * (insert) or tests (query) H bits inside that shard; a query is positive only
 * if every one of those (k-s+1)*H bits is set (Findere, Eq. 2).  Shards are
 * split into S sectors, S the largest power of two not above
 * min(H, shard_bits/64), and hash i addresses sector i mod S (Sec. IV-B; for
 * H = 3 on 512-bit shards S = 2); bit positions come from slices of a 64-bit s-mer hash
 * (bit-slicing, Sec. IV-G).  The exact hash functions, the canonical-k-mer
 * rule and the 512-bit layout are fixed by this library (see the sbf_create
 * notes below); they are what the parity tests check bit for bit.
 *
 * Conventions shared by every call:
 *  - Sequences are ASCII bytes.  A/C/G/T (either case) are bases; any other
 *    byte is invalid and no k-mer covering it exists (Sec. IV-C validity,
 *    Sec. IV-F separators).
 *  - A batch of reads is one concatenated byte array `seq` of `seq_len` bytes
 *    and `n_reads + 1` offsets: read r is seq[off[r], off[r+1]).  Offsets are
 *    non-decreasing, off[0] = 0 and off[n_reads] = seq_len.  K-mers never
 *    span two reads.  Offsets are not checked one by one (on the device that
 *    would need a synchronisation, on the host a pass over all reads); only
 *    the first and last (and group boundaries) are.  Offsets outside
 *    [0, seq_len] are clamped, so a malformed table gives wrong answers but
 *    no out-of-bounds access.
 *  - Query answers are bit-packed by START POSITION in `seq` (as Alg. 2
 *    writes output[blockStartKmer + localIdx]): bit p of a uint32 array
 *    (word p >> 5, bit p & 31) is 1 iff a valid k-mer starts at p and is
 *    positive.  The array has ceil(seq_len / 32) words and is fully written.
 *    read_hits[r] is the number of positive k-mers of read r.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    taking device pointers are asynchronous and stream-ordered like the
 *    paper's device-facing entry points (Sec. IV-A); calls with a `_host`
 *    suffix take host pointers and synchronise before returning.
 *  - Every call returns SBF_OK or a negative status; on error nothing is
 *    launched, outputs are untouched and sbf_last_error() (per thread) says
 *    why.  Device faults are reported as SBF_ECUDA.
 *  - Concurrent queries of one filter are safe.  An insert that overlaps a
 *    query on the device makes the query see some subset of the inserted
 *    bits (insertion is a monotone OR).
 */
#ifndef SBF_H
#define SBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbf_filter sbf_filter;
typedef void* sbf_stream_t; /* cudaStream_t */

enum {
  SBF_OK = 0,
  SBF_EINVAL = -1,        /* bad argument */
  SBF_ENOMEM = -2,        /* device or host allocation failed */
  SBF_ECUDA = -3,         /* a CUDA call failed */
  SBF_EUNSUPPORTED = -4,  /* parameters outside the compiled set */
  SBF_ETIMEOUT = -5,      /* a bounded device wait gave up */
  SBF_EBUSY = -6          /* resource in use (server admission) */
};

/* ---------------------------------------------------------------------------
 * Filter lifetime.
 *
 * sbf_create: 512-bit shards, canonical k-mers.  sbf_create_ex adds the shard
 * size (256 or 512 bits) and `canonical` (1: every m-mer and s-mer is replaced
 * by the smaller of its value and its reverse complement's, so a k-mer and
 * its reverse complement are the same key; 0: forward strand only, the
 * paper's literal behaviour).
 *
 * Parameters (Sec. IV-A, the paper's compile-time Config): 1 <= k <= 32,
 * 1 <= m <= k, 1 <= s <= k, k - m + 1 <= 32, k - s <= 15, 1 <= H <= 16,
 * bits >= shard_bits.  The number of shards is N = ceil(bits / shard_bits)
 * (the paper rounds to a power of two; any N is valid here because the shard
 * is chosen by a multiply-high, Sec. IV-B).  Returns SBF_EUNSUPPORTED for a
 * parameter set without a compiled kernel.  The filter owns N * shard_bits / 8
 * bytes of device memory on the current device, zeroed, and a 4-byte status
 * word (sbf_device_status).
 * ------------------------------------------------------------------------- */
int sbf_create(int k, int m, int s, int H, uint64_t bits, sbf_filter** out);
int sbf_create_ex(int k, int m, int s, int H, uint64_t bits, int shard_bits, int canonical,
                  sbf_filter** out);

/* Shard layouts.  SBF_LAYOUT_DEFAULT is the layout described above (any N,
 * shard = multiply-high of a mixed minimizer, min(H, W) sectors rounded down
 * to a power of two).  SBF_LAYOUT_PAPER is Sec. IV-B with Alg. 1/2 taken
 * literally: shard_bits must be 256, N is rounded UP to a power of two,
 * the shard is the minimizer's order key & (N - 1) (so it depends only on
 * the minimizer's last log2(N)/2 bases), and hash i sets a bit of 64-bit word
 * i mod 4 (b = 6; for H < 4 words H..3 stay zero; bit-slicing while
 * floor(64/H) >= 6, the salted multiply beyond, Sec. IV-G).  sbf_create_ex is
 * sbf_create_layout with SBF_LAYOUT_DEFAULT.  The fused kernels serve the
 * paper layout for H in {4, 8}; other H use the generic kernels. */
enum { SBF_LAYOUT_DEFAULT = 0, SBF_LAYOUT_PAPER = 1 };
int sbf_create_layout(int k, int m, int s, int H, uint64_t bits, int shard_bits, int canonical,
                      int layout, sbf_filter** out);
/* The filter's layout (SBF_LAYOUT_*), or SBF_EINVAL for NULL. */
int sbf_layout(const sbf_filter* f);

/* Alphabets (Sec. IV-A).  SBF_ALPHABET_DNA: the 2-bit bases above.
 * SBF_ALPHABET_PROTEIN: 26 symbols A..Z (either case) -> 0..25 in 5 bits,
 * one byte each; any other byte is invalid.  SBF_ALPHABET_DNA_TRIPLET: 64
 * symbols of three DNA bytes each (16 c0 + 4 c1 + c2, 6 bits); a triplet with
 * a non-ACGT byte is invalid, and a read's k-mers start at its first byte and
 * every third byte after (a trailing partial triplet is ignored).  For both:
 * k symbols are packed first-symbol-most-significant into 64 bits (k * bits
 * <= 64: k <= 12 for protein, k <= 10 for triplets), the order key is 32-bit
 * when m symbols fit 32 bits, k-mers are forward only (canonical must be 0),
 * and a query's answer bit is the k-mer's first byte.  Hashes and layouts are
 * those of the DNA filter.  These filters use the generic kernels (batches
 * and the server need the fused DNA kernels).  sbf_create_layout is
 * sbf_create_full with SBF_ALPHABET_DNA. */
enum { SBF_ALPHABET_DNA = 0, SBF_ALPHABET_PROTEIN = 1, SBF_ALPHABET_DNA_TRIPLET = 2 };
int sbf_create_full(int k, int m, int s, int H, uint64_t bits, int shard_bits, int canonical,
                    int layout, int alphabet, sbf_filter** out);
/* The filter's alphabet (SBF_ALPHABET_*), or SBF_EINVAL for NULL. */
int sbf_alphabet(const sbf_filter* f);
/* Frees the device memory.  NULL is a no-op.  Must not be called while work
 * on the filter is in flight. */
void sbf_destroy(sbf_filter* f);

/* Any output pointer may be NULL. */
int sbf_info(const sbf_filter* f, int* k, int* m, int* s, int* H, int* shard_bits,
             int* canonical, uint64_t* n_shards);
/* Number of 64-bit words of the bit array (N * shard_bits / 64). */
uint64_t sbf_num_words(const sbf_filter* f);
/* Device address of the bit array (uint64 words, shard x = words
 * [x*W, (x+1)*W), W = shard_bits / 64).  Owned by the filter. */
const uint64_t* sbf_device_words(const sbf_filter* f);

/* Which kernels serve this filter: 1 = the fused kernels (DNA, compiled grid
 * w = k-m+1 in {12, 16, 18, 20}, H in {1, 2, 4, 8}); 2 = the rolling kernels
 * (every other parameter set and alphabet: one thread per 32 start
 * positions, a rolling k-mer, s-mers shared by the k-mers of a run of one
 * shard); 0 = the generic one-k-mer-per-thread kernels, used only when the
 * environment variable SBF_FORCE_GENERIC is set at sbf_create (a second,
 * independent path for tests).  All give identical bits. */
int sbf_kernel_variant(const sbf_filter* f);

/* Device status of the filter's kernels: *status = 0 while every launch ran
 * to completion.  The fused query waits on a shard-copy barrier (filters of
 * 1 GiB and more); a wait bounded at one second of the GPU's global timer
 * that ran out sets bit 0, and that warp stopped early, so answers of the
 * launches since the last clear are incomplete.  Batched and served launches
 * report to the first filter of their batch or to their filter.  Reads the
 * word (synchronous, after the work queued before on any stream has been
 * ordered by the caller); clear != 0 resets it.  SBF_EINVAL on NULL. */
int sbf_device_status(const sbf_filter* f, uint32_t* status, int clear);

/* Zero all bits (stream-ordered). */
int sbf_clear(sbf_filter* f, sbf_stream_t stream);

/* Copy the bit array to / from host memory (sbf_num_words uint64 words);
 * synchronous.  This is also the checkpoint format's payload. */
int sbf_get_bits(const sbf_filter* f, uint64_t* h_words);
int sbf_set_bits(sbf_filter* f, const uint64_t* h_words);
/* Device-to-device copy of the filter's words [word_begin, word_begin +
 * n_words) to d_words (to_filter = 0) or from it (to_filter = 1), on
 * `stream`.  Used to combine filters that inserted disjoint read sets: the
 * filter after inserting everything is the OR of their words (Alg. 1). */
int sbf_copy_bits_device(sbf_filter* f, uint64_t* d_words, uint64_t word_begin, uint64_t n_words,
                         int to_filter, sbf_stream_t stream);

/* Word-wise OR of n_parts device arrays of n_words uint64 words each, laid
 * out back to back in d_in (piece j at d_in + j * n_words):
 * d_out[i] = OR over j of d_in[j * n_words + i].  Filters that inserted
 * disjoint read shares combine this way (Alg. 1: a filter is the OR of the
 * bits its k-mers set); the multi-process insert runs it on each rank's
 * slice of the words after an all-to-all exchange.  Both pointers are
 * caller-owned device memory, 16-byte aligned, and must not overlap; n_words
 * must be even when n_parts > 1 (every piece 16-byte aligned).  Asynchronous
 * on `stream`; SBF_EINVAL for a NULL pointer, misalignment or n_parts < 1. */
int sbf_or_reduce_device(uint64_t* d_out, const uint64_t* d_in, uint64_t n_words, int n_parts,
                         sbf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Insert and query (Alg. 1 and Alg. 2).  Device pointers.
 *
 * sbf_insert_seqs: sets the bits of every valid k-mer of every read
 *   (Alg. 1).  d_seq: seq_len bytes; d_off: n_reads + 1 uint64.
 * sbf_query_seqs: d_kmer_bits: ceil(seq_len/32) uint32 (may be NULL);
 *   d_read_hits: n_reads uint32 (may be NULL).  Both are overwritten.
 *   d_read_hits[r] is the number of set answer bits at read r's start
 *   positions.  With both outputs on the fused kernels and at least 2^26
 *   start positions, reads of at most 2048 positions are counted from the
 *   answer words by a second small kernel on the same stream; longer reads
 *   (and every read otherwise) are counted in the query kernel.
 * sbf_query_seqs_ex: as sbf_query_seqs, and if d_stats != NULL adds into
 *   d_stats[0] the number of valid k-mers, d_stats[1] the number of
 *   super-k-mer runs (maximal spans of consecutive valid k-mers of one read
 *   with one minimizer: the shard loads the method needs, Sec. II-B) and
 *   d_stats[2] the number of positive k-mers (three uint64 the caller zeroes).
 * ------------------------------------------------------------------------- */
int sbf_insert_seqs(sbf_filter* f, const uint8_t* d_seq, uint64_t seq_len,
                    const uint64_t* d_off, uint64_t n_reads, sbf_stream_t stream);
int sbf_query_seqs(const sbf_filter* f, const uint8_t* d_seq, uint64_t seq_len,
                   const uint64_t* d_off, uint64_t n_reads, uint32_t* d_kmer_bits,
                   uint32_t* d_read_hits, sbf_stream_t stream);
int sbf_query_seqs_ex(const sbf_filter* f, const uint8_t* d_seq, uint64_t seq_len,
                      const uint64_t* d_off, uint64_t n_reads, uint32_t* d_kmer_bits,
                      uint32_t* d_read_hits, uint64_t* d_stats, sbf_stream_t stream);

/* Host-resident input (Sec. V-F): the same operations on host buffers.  The
 * input is copied to the device in chunks on two streams so that copies
 * overlap the kernels; outputs are copied back.  Pinned host memory gives
 * full link speed, pageable memory works.  Synchronous.  A query on a
 * filter of 1 GiB or more returns SBF_ETIMEOUT if a bounded shard-copy wait
 * ran out (see sbf_device_status). */
int sbf_insert_seqs_host(sbf_filter* f, const uint8_t* h_seq, uint64_t seq_len,
                         const uint64_t* h_off, uint64_t n_reads);
int sbf_query_seqs_host(const sbf_filter* f, const uint8_t* h_seq, uint64_t seq_len,
                        const uint64_t* h_off, uint64_t n_reads, uint32_t* h_kmer_bits,
                        uint32_t* h_read_hits);

/* ---------------------------------------------------------------------------
 * Batches: many filters, one launch (scheduling only; the bits are those of
 * the single-filter calls).  Not in the paper: its library serves one filter
 * per call.
 *
 * A batch groups filters with equal (k, m, s, H, shard bits, canonical) and a
 * fused kernel (sbf_kernel_variant = 1); sizes may differ.  The filters stay
 * owned by the caller and must outlive the batch.  Reads are grouped by
 * filter: filter f serves reads [h_group[f], h_group[f+1]) (h_group has
 * n_filters + 1 entries, h_group[0] = 0, h_group[n_filters] = n_reads).
 * Both the device offsets d_off and a host copy h_off are needed (the host
 * copy sizes the per-filter work without a synchronisation).  Outputs are
 * laid out as in sbf_query_seqs over the whole batch.
 *
 * mode: SBF_BATCH_PER_FILTER launches once per filter; SBF_BATCH_FUSED runs
 * one persistent launch over a device table of all filters; SBF_BATCH_GRAPH
 * captures that launch (with its memsets) into a CUDA graph on the first call
 * and replays it while the arguments stay the same.  The batch owns a small
 * device table and a work counter; calls on one batch must not overlap.
 * ------------------------------------------------------------------------- */
typedef struct sbf_batch sbf_batch;
enum { SBF_BATCH_PER_FILTER = 0, SBF_BATCH_FUSED = 1, SBF_BATCH_GRAPH = 2 };

int sbf_batch_create(sbf_filter* const* filters, int n_filters, sbf_batch** out);
void sbf_batch_destroy(sbf_batch* b);
int sbf_batch_insert(sbf_batch* b, const uint8_t* d_seq, uint64_t seq_len, const uint64_t* d_off,
                     const uint64_t* h_off, uint64_t n_reads, const uint64_t* h_group, int mode,
                     sbf_stream_t stream);
int sbf_batch_query(sbf_batch* b, const uint8_t* d_seq, uint64_t seq_len, const uint64_t* d_off,
                    const uint64_t* h_off, uint64_t n_reads, const uint64_t* h_group,
                    uint32_t* d_kmer_bits, uint32_t* d_read_hits, int mode, sbf_stream_t stream);
/* Schedule of the persistent query (insert = 0) or insert (insert = 1)
 * launch: dynamic = 0 splits the iterations (496 start positions each) into
 * one contiguous share per warp; dynamic = 1 lets warps claim `chunk`
 * iterations at a time from a device counter; grid_blocks caps the blocks
 * (0 = full occupancy). */
int sbf_batch_set_schedule(sbf_batch* b, int insert, int dynamic, uint32_t chunk,
                           uint32_t grid_blocks);
int sbf_batch_get_schedule(const sbf_batch* b, int insert, int* dynamic, uint32_t* chunk,
                           uint32_t* grid_blocks);
/* Autotuner: times candidate schedules on this exact call (insert != 0: the
 * insert) with CUDA events -- first the static split and dynamic chunks of 4
 * to 1024 iterations at full occupancy, then the best of those with the grid
 * capped at 1, 2 and 3 blocks per SM -- keeps the fastest for that operation
 * and returns its time in *best_ms.  Synchronises; the call's outputs are
 * left as a normal call leaves them. */
int sbf_batch_tune(sbf_batch* b, int insert, const uint8_t* d_seq, uint64_t seq_len,
                   const uint64_t* d_off, const uint64_t* h_off, uint64_t n_reads,
                   const uint64_t* h_group, uint32_t* d_kmer_bits, uint32_t* d_read_hits,
                   sbf_stream_t stream, float* best_ms);

/* Batched query without any allocation.  The paper has no counterpart: it is
 * an entry point for callers that cannot call cudaMalloc -- for instance a
 * process whose framework allocator has already reserved almost all GPU
 * memory, or a latency-critical path that cannot take cudaMalloc's implicit
 * device synchronisation.  It answers exactly like sbf_batch_query in
 * SBF_BATCH_FUSED mode (same arguments, the filters passed directly instead of
 * a batch object), but its scratch (a work counter and the per-filter table)
 * lives in a fixed array compiled into the library: 45,312 bytes (a 256-byte
 * header and 512 table entries of 88 bytes) that every GPU loading the
 * library holds until the process exits.  Hence at most 512 filters per call
 * (more: SBF_EINVAL).  No device or pinned memory is allocated; the table
 * reaches the array in the parameters of small kernels (32 entries each), so
 * the call does not wait on the host for earlier work on its stream.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  All calls on a device
 * share the array and each call
 * resets what it needs, so calls whose work overlaps on the GPU (other
 * streams, other host threads without ordering) race: order them. */
int sbf_batch_query_noalloc(sbf_filter* const* filters, int n_filters, const uint8_t* d_seq,
                            uint64_t seq_len, const uint64_t* d_off, const uint64_t* h_off,
                            uint64_t n_reads, const uint64_t* h_group, uint32_t* d_kmer_bits,
                            uint32_t* d_read_hits, sbf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Serving: a request loop around one resident filter (continuous batching).
 * Not in the paper.
 *
 * sbf_server_create: the filter (with a fused kernel) stays resident; the
 *   server takes read_budget_bytes as its budget of request reads in flight
 *   and owns device memory for it (a read arena of that size, offsets and
 *   results of a quarter and three eighths of it), a pinned mirror of the
 *   result memory where results land before they are copied to the callers'
 *   buffers (so result buffers may be pageable), and a worker thread.
 *   Queued requests are admitted while that memory and budget have room,
 *   every request admitted at one moment (at most max_per_launch of them,
 *   1..65536) is served by ONE kernel launch (one segment each), and up to
 *   max_inflight (1..16) launches run at once on separate streams, so
 *   requests that arrive while others run overlap with them.  A launch takes
 *   no further request once its reads reach read_budget_bytes /
 *   (max_inflight + 1), so a deep queue becomes several launches whose
 *   result copies overlap the next one's kernel.
 *   max_per_launch = 1 gives one launch per request, the baseline continuous
 *   batching is measured against.
 *   Inputs the device can read in place are not copied: page-locked host
 *   memory mapped for the device, and any host memory when the device reads
 *   pageable memory through the host's page tables (GB300 over NVLink-C2C).
 *   The kernel then reads the request's bytes and offsets where they are;
 *   they still count against read_budget_bytes while in flight.  Other
 *   requests are copied into the read arena first.
 * sbf_server_create_ex: flags = SBF_SERVER_STAGE_INPUTS copies every
 *   request into the read arena (never reads host memory in place).
 * sbf_server_submit: queue one request of host reads (offsets as in
 *   sbf_query_seqs, off[0] = 0).  h_read_hits (n_reads, may be NULL) and
 *   h_kmer_bits (ceil(seq_len/32) words, may be NULL) receive exactly what
 *   sbf_query_seqs would write.  All host buffers must stay valid and
 *   unchanged until the request is waited for (the device may read them at
 *   any time before).  A request larger than the budget, or with offsets that
 *   decrease, is refused (SBF_EINVAL).  Thread-safe.
 * sbf_server_submit_batch: n requests in one call (arrays of the arguments
 *   above; h_read_hits and h_kmer_bits may be NULL arrays); tickets[i] is
 *   request i's.  If any request is refused, none is queued.
 * sbf_server_wait: block until the request is done or timeout_s passes
 *   (SBF_ETIMEOUT); on success the ticket is released and *latency_s (may be
 *   NULL) is the time from submission to completion.
 * sbf_server_stats: latency percentiles of the requests completed since the
 *   last reset, and k-mers served per second from the first submission to
 *   the last completion.
 * sbf_server_breakdown: p50 and p99 (arrays of 4) of the time requests spent
 *   queued (submission to admission), being launched (admission to the end
 *   of the launch calls), on the device (to the worker seeing the launch
 *   complete) and in delivery (copies to the callers' buffers), since the
 *   last reset; and how many requests were read in place and how many staged.
 * sbf_server_destroy: finishes queued and running requests, then frees.
 * ------------------------------------------------------------------------- */
typedef struct sbf_server sbf_server;
enum { SBF_SERVER_STAGE_INPUTS = 1 };

int sbf_server_create(const sbf_filter* f, uint64_t read_budget_bytes, int max_inflight,
                      uint32_t max_per_launch, sbf_server** out);
int sbf_server_create_ex(const sbf_filter* f, uint64_t read_budget_bytes, int max_inflight,
                         uint32_t max_per_launch, uint32_t flags, sbf_server** out);
void sbf_server_destroy(sbf_server* s);
int sbf_server_submit(sbf_server* s, const uint8_t* h_seq, uint64_t seq_len, const uint64_t* h_off,
                      uint64_t n_reads, uint32_t* h_read_hits, uint32_t* h_kmer_bits,
                      uint64_t* ticket);
int sbf_server_submit_batch(sbf_server* s, uint64_t n, const uint8_t* const* h_seqs,
                            const uint64_t* seq_lens, const uint64_t* const* h_offs,
                            const uint64_t* n_reads, uint32_t* const* h_read_hits,
                            uint32_t* const* h_kmer_bits, uint64_t* tickets);
int sbf_server_wait(sbf_server* s, uint64_t ticket, double timeout_s, double* latency_s);
int sbf_server_stats(sbf_server* s, uint64_t* completed, double* p50_s, double* p99_s,
                     double* mean_s, double* kmers_per_s, uint64_t* launches);
int sbf_server_breakdown(sbf_server* s, double* p50_s, double* p99_s, uint64_t* direct,
                         uint64_t* staged);
int sbf_server_reset_stats(sbf_server* s);

/* Number of k-mer start positions sum_r max(0, len_r - k + 1) of a host
 * offset table (valid or not): the number of k-mers a batch presents, the
 * unit of every k-mers/s figure.  It does not size a query output, whose
 * answer words are indexed by start position in seq (ceil(seq_len / 32)
 * words, see above); a position where no k-mer starts has a 0 bit. */
int sbf_num_kmers(const uint64_t* h_off, uint64_t n_reads, int k, uint64_t* out);

/* ---------------------------------------------------------------------------
 * FASTA / FASTQ input (host side; Sec. IV-A streamed FASTX input, Sec. IV-F
 * sequence-native records).
 *
 * An incremental parser that turns FASTX text, fed in chunks of any size,
 * into read batches for sbf_*_seqs_host: sequence bytes of one or more
 * records back to back, `n_pieces + 1` offsets, and for each piece the index
 * of its record (0, 1, ... in file order; FASTA '>' and FASTQ '@' records may
 * be mixed).  Header lines, FASTQ '+' lines and qualities are skipped; line
 * breaks, CR, spaces and tabs inside sequence lines are dropped; every other
 * byte is copied (non-ACGT bytes such as N are invalid and break k-mers,
 * Sec. IV-F).  A record that does not fit the output buffer is split: its
 * next piece (in the next call) starts with the record's last k-1 bases, so
 * each k-mer of a record lies in exactly one piece.  Summing the per-read
 * hits of sbf_query_seqs_host over a record's pieces gives the record's hits.
 *
 * sbf_fastx_create: k sets the k-1 bases carried into a split record's next
 *   piece.  The parser owns no caller memory.
 * sbf_fastx_parse: parses text[0, *consumed) into seq (capacity seq_cap
 *   bytes, at least 2(k-1) + 64), off (pieces_cap + 1 entries) and rec
 *   (pieces_cap entries).  It stops early when either output is full; the
 *   caller feeds text[*consumed, text_len) again (with the next chunk
 *   appended if it likes).  final = 1 marks text_len as the end of the input
 *   (the open record ends).  A record may yield zero-length pieces.
 * ------------------------------------------------------------------------- */
typedef struct sbf_fastx sbf_fastx;
int sbf_fastx_create(int k, sbf_fastx** out);
void sbf_fastx_destroy(sbf_fastx* p);
int sbf_fastx_parse(sbf_fastx* p, const uint8_t* text, uint64_t text_len, int final,
                    uint8_t* seq, uint64_t seq_cap, uint64_t* off, uint64_t* rec,
                    uint64_t pieces_cap, uint64_t* n_pieces, uint64_t* seq_len,
                    uint64_t* consumed);

/* FASTA / FASTQ on the device.  sbf_fastx_parse_device turns a chunk of
 * whole records in device memory (d_text, 16-byte aligned, text_len bytes,
 * starting at a record's header line and ending with '\n') into a read batch
 * in device memory: d_seq receives the records' sequence bytes back to back
 * (at most text_len bytes), d_off the n + 1 record offsets (max_records + 1
 * entries).  fastq = 0: FASTA (records start at lines beginning with '>';
 * sequence lines lose '\r', ' ' and '\t'); fastq = 1: four-line FASTQ
 * records.  The bytes kept are exactly those sbf_fastx_parse keeps.  On
 * return (the call synchronises `stream`) h_result[0] = records, [1] =
 * sequence bytes, [2] = 1 if the chunk is outside these shapes (a FASTA line
 * starting with '@', a FASTQ record not of four lines, a quality line of
 * another length): then nothing usable was written and the chunk should go
 * through sbf_fastx_parse.  d_scratch (16-byte aligned) needs
 * sbf_fastx_device_scratch(text_len) bytes (about 9 per text byte). */
int sbf_fastx_device_scratch(uint64_t text_len, uint64_t* scratch_bytes);
int sbf_fastx_parse_device(const uint8_t* d_text, uint64_t text_len, int fastq, uint8_t* d_seq,
                           uint64_t* d_off, uint64_t max_records, void* d_scratch,
                           uint64_t scratch_bytes, uint64_t* h_result, sbf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Random-sector bandwidth probe.  Measurement only; not a step of the method.
 *
 * Inserts and queries touch one shard of shard_bits/8 bytes per super-k-mer
 * run at a hashed position (Alg. 1 flush, Alg. 2 shard load), so their shard
 * traffic is bounded by the bandwidth of random sector-sized accesses, not by
 * a streaming copy.  This call measures that ceiling on the caller's buffer:
 *  rmw = 0: n loads of one whole random sector each (sector_bytes / 16 lanes
 *           of 16 bytes, sector-aligned);
 *  rmw = 1: n read-modify-writes, one 64-bit atomicOr of a nonzero mask into
 *           every word of a random sector (the buffer's bits change).
 * Sector i of the sequence is floor(mix64(seed + i) * (buf_bytes /
 * sector_bytes) / 2^64) with mix64 the SplitMix64 finaliser, so a run with the
 * same arguments touches the same sectors.  d_buf: device, 64-byte aligned,
 * buf_bytes >= sector_bytes; sector_bytes: 32 or 64; d_sink: one device
 * uint64 the gather may add to (keeps its loads live; contents meaningless).
 * Asynchronous on `stream`; time it with events.  Algorithmic bytes: n *
 * sector_bytes (gather), 2 * n * sector_bytes (read-modify-write).
 * ------------------------------------------------------------------------- */
int sbf_probe_sectors(void* d_buf, uint64_t buf_bytes, int sector_bytes, uint64_t n,
                      uint64_t seed, int rmw, uint64_t* d_sink, sbf_stream_t stream);

/* Human-readable reason of the calling thread's last failure ("" if none). */
const char* sbf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SBF_H */
