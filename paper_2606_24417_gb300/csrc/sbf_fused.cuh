// sbf_fused.cuh -- fused sequence-native insert / query kernels for sm_103a.
//
// What they compute is Alg. 1 (insert) and Alg. 2 (query) of the cuSBF
// paper; how is designed for GB300 rather than taken from the paper:
//
//  * Warp-private pipeline, no block-wide barriers.  A warp owns a contiguous
//    range of start positions and walks it in iterations of U*16 positions
//    (U = 31 or 30 "useful" lanes; the last lane(s) only compute values their
//    left neighbours need).
//  * Staging: each lane loads 16 raw bytes (one 128-bit non-coherent load),
//    encodes them ONCE into a 2-bit word (first base most significant), its
//    reverse complement and a 16-bit invalid-base mask in shared memory.
//    Consecutive iterations overlap by the words their windows share; those
//    are carried in shared memory, so every iteration after a range's first
//    encodes exactly U new words (one per useful lane, no divergent pass).
//  * Lane chunks: lane l owns positions [16l, 16l+16).  From three staged words
//    it extracts every m-mer and s-mer by static funnel shifts (no per-k-mer
//    re-packing, Sec. IV-C / IV-E amortisation taken to the whole chunk).
//  * Minimizer: the sliding minimum of the order keys over w windows is the
//    van Herk / Gil-Werman block decomposition over the lane's keys and its
//    neighbour's (shuffled).  The order key is a bijection, so the minimizer
//    value is recovered from the minimum key by one multiplication with the
//    modular inverse -- no argmin is tracked.
//  * Runs (super-k-mers, Sec. II-B): run heads are compacted warp-wide into
//    slots; the shard of each run is computed once and loaded once into
//    shared memory (query: cp.async, and for filters of 1 GiB or more partly
//    TMA bulk copies on a per-warp mbarrier), or zeroed there (insert).
//  * Findere with pair deduplication: k-mer j needs its k-s+1 s-mers tested
//    in its run's shard.  Every position t tests its own pair (t, shard(t));
//    every run end e adds the z = k-s pairs (e+d, shard(e)).  A word-parallel
//    sliding AND inside runs plus a kill mask from the extra pairs gives the
//    Findere answers bit-packed, without any per-k-mer re-hashing.
//  * Insert ORs the same pairs' bits into the run's slot (shared atomics) and
//    flushes each slot with coalesced 64-bit atomicOr (Alg. 1's head-only
//    atomics, one per word per run).
#pragma once

#include <cstdint>
#include <type_traits>

#include "sbf_internal.h"

namespace sbf {
namespace fused {

constexpr int kLanePos = 16;        // start positions per lane
constexpr int kWarps = 4;           // warps per block
constexpr int kThreads = 32 * kWarps;
constexpr int kSlotCap = 64;        // runs per iteration with a shard copy in shared memory
// Windows of 12 or less (m = 20 at k = 31) give about 2/(w+1) * 496 = 76 runs
// per iteration, more than 64 slots; runs past the last slot set their bits
// with global atomics (insert) or test them with global loads (query).
// Inserts with such windows keep 96 slots in shared memory (m = 20, H = 8
// inserts 3.6x faster on 512-bit shards, 2.3x on 256-bit), and so do the
// queries on 512-bit shards, which run 3 blocks per SM either way; the
// 256-bit-shard queries (4 blocks per SM) would lose a block to the array.
template <int W, bool INSERT, int B>
constexpr int slot_cap() { return (W <= 12 && (INSERT || B == 512)) ? 96 : kSlotCap; }
constexpr int kStage = 34;          // staged 16-base words per iteration (544 bases)
constexpr unsigned kFull = 0xFFFFFFFFu;

// Shard copies of the query.  Below kTmaMinBytes of filter every slot is
// loaded with 16-byte cp.async.  From there on, slots kTmaFromSlot.. are
// loaded by the TMA engine instead (one cp.async.bulk of B/8 bytes each,
// completing on the warp's mbarrier): beyond L2 nearly every cp.async misses
// L2 and the TLB and holds the load/store pipe that all shared-memory loads
// and shuffles of the SM also use (short-scoreboard stalls tripled on a
// 2 GiB filter), while the bulk copies' fixed cost makes them slower than
// cp.async on filters that L2 serves.  Measured on GB300 (2M reads, k=31,
// m=16, s=28, H=4, 512-bit shards): 4 GiB 2.99 -> 2.49 ms, 1 GiB 2.57 ->
// 2.42 ms, 512 MiB 2.27 -> 2.40 ms; so the switch is at 1 GiB.
constexpr uint64_t kTmaMinBytes = 1ull << 30;
constexpr uint32_t kTmaFromSlot = 32;
// Bound of every wait on that barrier: one second of the global timer.  Each
// try_wait may suspend the thread for up to kSuspendHintNs instead of
// returning at once (it resumes when the phase completes), so a waiting warp
// issues few instructions (queries on a 4 GiB filter 0.5-1% faster).
constexpr uint64_t kWaitLimitNs = 1000000000ull;
constexpr uint32_t kSuspendHintNs = 20000;

// Modular inverses of the odd golden-ratio multipliers (Newton iteration).
__host__ __device__ constexpr uint32_t inv32(uint32_t a) {
  uint32_t x = a;
  for (int i = 0; i < 5; ++i) x *= 2u - a * x;
  return x;
}
__host__ __device__ constexpr uint64_t inv64(uint64_t a) {
  uint64_t x = a;
  for (int i = 0; i < 6; ++i) x *= 2ull - a * x;
  return x;
}
static_assert(inv32(kGolden32) * kGolden32 == 1u, "inverse");
static_assert(inv64(kGolden64) * kGolden64 == 1ull, "inverse");

template <int W>
struct Shape {
  // lanes whose chunk is only read by neighbours: windows reach up to
  // position 15 + W - 1 of the chunk, i.e. into lane l+1 (W <= 17) or l+2
  static constexpr int kHelpers = (15 + W - 1 >= 32) ? 2 : 1;
  static constexpr int kUseful = 32 - kHelpers;
  static constexpr int kAdvance = kUseful * kLanePos;
};

// Bit-address packs: H in-shard addresses of one s-mer, one per byte (H <= 4)
// or the masked hash itself (H = 8).
template <int H, int B>
struct Layout {
  static constexpr int W64 = B / 64;
  static constexpr int S = H < W64 ? H : W64;       // sectors (H is a power of two)
  static constexpr int SB = B / S;                   // sector bits
  static constexpr int b = (SB == 64) ? 6 : (SB == 128) ? 7 : (SB == 256) ? 8 : 9;
  static constexpr int q = 64 / H;                   // slice width (>= b for H <= 8)
  static constexpr int W32 = B / 32;                 // 32-bit words per shard
  static constexpr int SW32 = SB / 32;               // 32-bit words per sector
  // slot stride in shared memory: W32 + 4 words keeps 16-byte alignment for
  // cp.async and spreads consecutive slots over different banks
  static constexpr int SLOT = W32 + 4;
  using Pack = typename std::conditional<(H == 8), uint64_t, uint32_t>::type;
  static_assert(q >= b, "bit-slicing only");
};

template <int H, int B>
__device__ __forceinline__ typename Layout<H, B>::Pack make_pack(uint64_t h) {
  using L = Layout<H, B>;
  const uint32_t lo = (uint32_t)h, hi = (uint32_t)(h >> 32);
  constexpr uint32_t m = (1u << L::b) - 1u;
  if constexpr (H == 1) {
    return lo & m;
  } else if constexpr (H == 2) {
    return __byte_perm(lo, hi, 0x0040) & (m | (m << 8));
  } else if constexpr (H == 4) {
    return __byte_perm(lo, hi, 0x6420) & (m * 0x01010101u);
  } else {
    return h & ((uint64_t)m * 0x0101010101010101ull);
  }
}

template <int H, int B>
__device__ __forceinline__ uint32_t pack_addr(typename Layout<H, B>::Pack pk, int i) {
  if constexpr (H == 1) {
    return (uint32_t)pk;
  } else if constexpr (H == 8) {
    return (uint32_t)(pk >> (8 * i)) & 0xFFu;
  } else {
    return ((uint32_t)pk >> (8 * i)) & 0xFFu;
  }
}

// One filter's share of a launch: the filter, the reads it serves (a slice
// of the offset table, absolute positions) and the positions to cover.
// Shared-memory bit test / set of one s-mer's H addresses in a shard slot.
// The byte offset of hash i's 32-bit word inside its sector is
// ((p_i >> 5) << 2) = (p_i >> 3) & ~3, masked to the sector: one shift and
// mask yield it for all packed bytes at once, a byte permute picks one.  The
// funnel shift uses only the low 5 bits of its amount, so p_i itself (the
// pack shifted to byte i) serves as the bit index.
template <int H, int B>
__device__ __forceinline__ uint32_t test_slot(const uint32_t* slot_words,
                                              typename Layout<H, B>::Pack pk) {
  using L = Layout<H, B>;
  constexpr uint32_t SBY = L::SB / 8;          // sector bytes
  constexpr uint32_t OM = (SBY - 1u) & ~3u;   // word byte-offset mask
  const char* base = reinterpret_cast<const char*>(slot_words);
  uint32_t acc = 1u;
  if constexpr (H == 1) {
    const uint32_t p = (uint32_t)pk;
    const uint32_t w = *reinterpret_cast<const uint32_t*>(base + ((p >> 3) & OM));
    acc &= __funnelshift_r(w, w, p);
  } else if constexpr (H <= 4) {
    const uint32_t v = ((uint32_t)pk >> 3) & (OM * 0x01010101u);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const uint32_t off = __byte_perm(v, 0u, 0x4440u | (uint32_t)i);
      const uint32_t sh = i == 0 ? (uint32_t)pk : __byte_perm((uint32_t)pk, 0u, 0x4440u | (uint32_t)i);
      const uint32_t w = *reinterpret_cast<const uint32_t*>(base + (i % L::S) * SBY + off);
      acc &= __funnelshift_r(w, w, sh);
    }
  } else {
    const uint32_t lo = (uint32_t)pk, hi = (uint32_t)(pk >> 32);
    const uint32_t vlo = (lo >> 3) & (OM * 0x01010101u), vhi = (hi >> 3) & (OM * 0x01010101u);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const uint32_t src = i < 4 ? vlo : vhi;
      const uint32_t srp = i < 4 ? lo : hi;
      const uint32_t off = __byte_perm(src, 0u, 0x4440u | (uint32_t)(i & 3));
      const uint32_t sh = __byte_perm(srp, 0u, 0x4440u | (uint32_t)(i & 3));
      const uint32_t w = *reinterpret_cast<const uint32_t*>(base + (i % L::S) * SBY + off);
      acc &= __funnelshift_r(w, w, sh);
    }
  }
  return acc & 1u;
}

// Insert: the H bits, hash (ii + rot) mod H at step ii, so that lanes of one
// run (consecutive lanes, rot = lane mod H) set bits in different sectors at
// the same time instead of queueing on the same shared words.
template <int H, int B>
__device__ __forceinline__ void set_slot_rot(uint32_t* slot_words, typename Layout<H, B>::Pack pk,
                                             uint32_t rot) {
  using L = Layout<H, B>;
  constexpr uint32_t SBY = L::SB / 8;
  constexpr uint32_t OM = (SBY - 1u) & ~3u;
  char* base = reinterpret_cast<char*>(slot_words);
#pragma unroll
  for (int ii = 0; ii < H; ++ii) {
    const uint32_t i = ((uint32_t)ii + rot) & (uint32_t)(H - 1);
    uint32_t p;
    if constexpr (H == 1) {
      p = (uint32_t)pk;   // one address of up to 9 bits, not a byte
    } else if constexpr (H == 8) {
      p = (uint32_t)(pk >> (8 * i)) & 0xFFu;
    } else {
      p = ((uint32_t)pk >> (8 * i)) & 0xFFu;
    }
    atomicOr(reinterpret_cast<uint32_t*>(base + (i & (uint32_t)(L::S - 1)) * SBY + ((p >> 3) & OM)),
             1u << (p & 31u));
  }
}


// One share of a launch: a filter, the bytes and reads it serves and where
// its answers go.  Positions are relative to `seq`; the offsets use the same
// positions.
struct Segment {
  uint64_t* words;        // the filter's bit array
  uint64_t n_shards;
  const uint8_t* seq;     // bytes; positions index this pointer
  uint64_t seq_len;       // positions >= seq_len read as invalid bytes
  const uint64_t* off;    // n_reads + 1 offsets (positions in seq)
  uint64_t n_reads;
  uint32_t* bits;         // query: answer words indexed by position >> 5 (zeroed), or NULL
  uint32_t* hits;         // query: counts of these reads (zeroed by the launcher), or NULL
  uint64_t p_begin;       // first position covered (multiple of 16)
  uint64_t iter_begin;    // index of the segment's first iteration in the launch
  uint64_t iters;         // iterations of kAdvance positions
};

struct Params {
  Geom g;                 // shared k, m, s, H, shard bits, canonical, layout
  uint64_t* stats;        // query: valid k-mers, runs, positives, or NULL
  const Segment* segs;    // NULL: the launch is the single segment seg0
  uint32_t n_segs;
  Segment seg0;
  uint64_t iters;         // iterations over all segments
  unsigned long long* work;  // dynamic scheduling counter (zeroed), or NULL for a static split
  uint32_t chunk;         // iterations per dynamically claimed work item
  uint32_t grid_blocks;   // blocks to launch (0: enough for the work, capped at full occupancy)
  uint32_t big;           // a segment's filter has kTmaMinBytes or more (query: BULK kernels)
  uint32_t hits_above;    // query: the kernel counts hits of reads longer than this (0: of every
                          // read); shorter reads are counted afterwards from the answer words
};

template <int SC, int H, int B, bool KEY64>
struct alignas(16) WarpSmem {
  using L = Layout<H, B>;
  using Pack = typename L::Pack;
  // minimizer key, then shard index, per slot (32-bit unless the key is 64-bit;
  // the 32-bit form needs fewer than 2^32 shards)
  using SlotT = typename std::conditional<KEY64, uint64_t, uint32_t>::type;
  static constexpr int kHsStride = sizeof(Pack) == 4 ? 34 : 33;  // bank-conflict-free transposes
  uint32_t shard[SC * L::SLOT];          // shard copies (query) or masks (insert)
  SlotT slot_x[512];
  Pack hs[kLanePos * kHsStride];         // s-mer bit-address packs, [j][lane]
  uint16_t slot_of[kLanePos * 34];       // slot of each valid position, [j][lane]
  uint16_t end_list[512];                // run-end positions (end i closes slot i)
  uint32_t fwd[kStage];                  // staged 2-bit words
  uint32_t rcw[kStage];                  // their reverse complements
  uint32_t bad[kStage];                  // 16-bit invalid masks
  uint32_t valid_w[17];                  // position-space bit words (+1 zero word)
  uint32_t end_w[17];
  uint32_t own_w[17];
  uint32_t kill_w[17];
  uint32_t k_w[17];
  uint32_t pref_w[17];
  unsigned long long bar;                // query: the shard copies' mbarrier
};

// Waits for the completion of phase `parity` of the mbarrier at shared
// address bar, at most kWaitLimitNs of the global timer; false if it did not
// complete in that time.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity) {
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(parity), "n"(kSuspendHintNs) : "memory");
    if (done) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > kWaitLimitNs) return false;
  }
}

__device__ __forceinline__ uint32_t pairswap(uint32_t x) {
  return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

// 16 bytes at pos (bytes past seq_len read as 'N').
__device__ __forceinline__ uint4 load16(const uint8_t* seq, uint64_t pos, uint64_t seq_len,
                                        bool aligned) {
  if (aligned && pos + 16 <= seq_len) return __ldg(reinterpret_cast<const uint4*>(seq + pos));
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint32_t v = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      uint64_t p = pos + 4 * i + b;
      uint32_t ch = p < seq_len ? (uint32_t)seq[p] : (uint32_t)'N';
      v |= ch << (8 * b);
    }
    w[i] = v;
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Encode 4 ASCII bytes: 8-bit group of 2-bit codes (byte 0 most significant)
// and a 4-bit invalid mask (bit b = byte b not A/C/G/T in either case).
__device__ __forceinline__ void encode4(uint32_t x, uint32_t& code8, uint32_t& bad4) {
  uint32_t t = ((x >> 1) ^ (x >> 2)) & 0x03030303u;
  code8 = (t * 0x40100401u) >> 24;
  uint32_t sel = (t & 0x3u) | ((t >> 4) & 0x30u) | ((t >> 8) & 0x300u) | ((t >> 12) & 0x3000u);
  uint32_t expect = __byte_perm(0x54474341u, 0u, sel);  // 'A','C','G','T' by code
  uint32_t diff = expect ^ (x & 0xDFDFDFDFu);            // 0 byte <=> valid
  uint32_t nz = (((diff & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | diff) & 0x80808080u;
  bad4 = ((nz >> 7) * 0x00204081u >> 21) & 0xFu;
}

// Read the warp's position range [lo, hi) of start positions holding the
// reads: last r with off[r] <= p (32-ary search, warp-uniform result).
__device__ __forceinline__ uint64_t warp_find_read(const uint64_t* off, uint64_t n_reads,
                                                   uint64_t p, int lane) {
  uint64_t lo = 0, hi = n_reads;  // answer in [lo, hi)
  while (hi - lo > 1) {
    uint64_t step = (hi - lo + 31) / 32;
    uint64_t c = lo + (uint64_t)lane * step;
    bool pred = c < hi && off[c] <= p;
    unsigned bal = __ballot_sync(kFull, pred);
    if (bal == 0) return lo;  // off[lo] > p: before the first read
    int i = 31 - __clz(bal);
    uint64_t nlo = lo + (uint64_t)i * step;
    uint64_t nhi = nlo + step < hi ? nlo + step : hi;
    lo = nlo;
    hi = nhi;
  }
  return lo;
}

template <typename KeyT>
__device__ __forceinline__ KeyT key_of(uint64_t v) {
  if constexpr (sizeof(KeyT) == 4) {
    return (uint32_t)v * kGolden32;
  } else {
    return v * kGolden64;
  }
}

// Minimizer order key and validity of the k-mer at position p, straight from
// global memory (only for exact run-head statistics at a warp's first position).
template <typename KeyT>
__device__ bool prev_kmer_key(const Geom& g, const uint8_t* seq, uint64_t seq_len,
                              const uint64_t* off, uint64_t n_reads, uint64_t p, KeyT& key) {
  if (n_reads == 0) return false;
  uint64_t lo = 0, hi = n_reads;
  while (hi - lo > 1) {
    uint64_t mid = lo + ((hi - lo) >> 1);
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  uint64_t end = off[lo + 1] < seq_len ? off[lo + 1] : seq_len;
  if (off[lo] > p || p + (uint64_t)g.k > end) return false;
  uint64_t fwd = 0, rc = 0;
  for (int i = 0; i < g.k; ++i) {
    uint32_t ch = seq[p + i];
    if (!base_valid(ch)) return false;
    uint32_t c = base_code(ch);
    fwd = (fwd << 2) | c;
    rc |= (uint64_t)(3u - c) << (2 * i);
  }
  KeyT best = 0;
  for (int i = 0; i <= g.k - g.m; ++i) {
    uint64_t f = (fwd >> (2 * (g.k - g.m - i))) & len_mask(g.m);
    uint64_t r = (rc >> (2 * i)) & len_mask(g.m);
    uint64_t v = g.canonical ? (f < r ? f : r) : f;
    KeyT kk = key_of<KeyT>(v);
    if (i == 0 || kk < best) best = kk;
  }
  key = best;
  return true;
}

// Iterations [it0, it1) of one segment, walked by one warp.  False if a
// wait for shard copies ran out (the filter's status word is set).  BULK:
// the kernel variant for launches with a filter of kTmaMinBytes or more.
template <int W, int H, int B, bool KEY64, bool INSERT, bool BULK>
__device__ __forceinline__ bool run_range(WarpSmem<slot_cap<W, INSERT, B>(), H, B, KEY64>& S,
                                          const Params& P,
                                          const Segment& seg, uint64_t it0, uint64_t it1,
                                          int lane, unsigned long long& st_valid,
                                          unsigned long long& st_runs,
                                          unsigned long long& st_pos, uint32_t& bar_phase) {
  using L = Layout<H, B>;
  using Pack = typename L::Pack;
  using KeyT = typename std::conditional<KEY64, uint64_t, uint32_t>::type;
  using Sm = WarpSmem<slot_cap<W, INSERT, B>(), H, B, KEY64>;
  constexpr int U = Shape<W>::kUseful;
  constexpr int ADV = Shape<W>::kAdvance;
  constexpr int HS = Sm::kHsStride;
  constexpr int SC = slot_cap<W, INSERT, B>();  // runs of an iteration with a slot in shared memory
  // Queries test own pairs without masks or a global fallback when all runs of
  // an iteration have a slot.  That pays where the runs (about 2/(W+1) of
  // the 496 positions) usually fit the slots: W >= 16 with 64 slots, W = 12
  // with 96; at W = 12 with 64 slots (average 76 runs) the second loop only
  // adds code (2-5% slower there).
  constexpr bool kFastOwn = !INSERT && (W > 12 || SC > kSlotCap);
  Geom g = P.g;
  g.words = seg.words;
  g.n_shards = seg.n_shards;
  const int k = g.k, m = g.m, s = g.s, z = g.k - g.s;
  const bool canon = g.canonical != 0;

  const uint64_t seq_len = seg.seq_len;
  const uint64_t* off = seg.off;
  const uint64_t n_reads = seg.n_reads;
  // start positions outside [lo_pos, hi_pos) belong to no read
  uint64_t lo_pos = 0, hi_pos = 0;
  if (n_reads > 0) {
    lo_pos = off[0] < seq_len ? off[0] : seq_len;
    hi_pos = off[n_reads] < seq_len ? off[n_reads] : seq_len;
  }
  const bool aligned = (reinterpret_cast<uintptr_t>(seg.seq) & 15u) == 0;
  const uint64_t smask = (s >= 32) ? ~0ull : ((1ull << (2 * s)) - 1ull);
  const uint64_t mmask = (m >= 32) ? ~0ull : ((1ull << (2 * m)) - 1ull);
  uint32_t* words32 = reinterpret_cast<uint32_t*>(g.words);

  // end of read q (clamped), or "infinity" past the last read
  auto read_end = [&](uint64_t q) -> uint64_t {
    if (q >= n_reads) return ~0ull;
    uint64_t e = off[q + 1];
    return e < seq_len ? e : seq_len;
  };

  uint64_t p0 = seg.p_begin + it0 * (uint64_t)ADV;
  uint64_t r_cur = n_reads > 0 ? warp_find_read(off, n_reads, p0, lane) : 0;
  uint64_t r_cur_start = 0;                              // start of read r_cur (clamped)
  if (n_reads > 0) r_cur_start = off[r_cur] < seq_len ? off[r_cur] : seq_len;
  uint64_t e_batch = read_end(r_cur + lane);              // prefetched first batch of read ends
  // prefetched raw bytes of the first iteration
  uint4 raw_a = load16(seg.seq, p0 + 16ull * lane, seq_len, aligned);
  uint4 raw_b = make_uint4(0, 0, 0, 0);
  if (lane < kStage - 32) raw_b = load16(seg.seq, p0 + 16ull * (lane + 32), seq_len, aligned);

  // run-head carry: validity and minimizer key of position p0 - 1
  bool carry_valid = false;
  KeyT carry_key = 0;
  if (!INSERT && P.stats && p0 > 0) {
    KeyT kk = 0;
    bool v = false;
    if (lane == 0) v = prev_kmer_key<KeyT>(g, seg.seq, seq_len, off, n_reads, p0 - 1, kk);
    carry_valid = __shfl_sync(kFull, v, 0);
    if constexpr (KEY64) {
      carry_key = ((uint64_t)__shfl_sync(kFull, (uint32_t)(kk >> 32), 0) << 32) |
                  __shfl_sync(kFull, (uint32_t)kk, 0);
    } else {
      carry_key = __shfl_sync(kFull, kk, 0);
    }
  }

  // Staging: encode the 16 bases of word wi at p (bytes raw) once.
  auto stage = [&](uint64_t p, int wi, const uint4& raw) {
    const uint64_t pos = p + 16ull * wi;
    uint32_t c8, b4, fw, bad;
    encode4(raw.x, c8, b4); fw = c8;             bad = b4;
    encode4(raw.y, c8, b4); fw = (fw << 8) | c8; bad |= b4 << 4;
    encode4(raw.z, c8, b4); fw = (fw << 8) | c8; bad |= b4 << 8;
    encode4(raw.w, c8, b4); fw = (fw << 8) | c8; bad |= b4 << 12;
    if (pos < lo_pos || pos + 16 > hi_pos) {  // outside the reads' span
      uint32_t okm = 0;
#pragma unroll
      for (int b = 0; b < 16; ++b) okm |= (uint32_t)(pos + b >= lo_pos && pos + b < hi_pos) << b;
      bad |= ~okm & 0xFFFFu;
    }
    S.fwd[wi] = fw;
    S.rcw[wi] = ~pairswap(__brev(fw));
    S.bad[wi] = bad;
  };
  // Iterations advance by U*16 bases, so the last NC staged words of one are
  // the first NC of the next: the range's first iteration stages all kStage
  // words here, and every iteration stages the next one's other U words at
  // its end (their bytes prefetched one iteration ahead).
  constexpr int NC = kStage - U;
  if (it0 < it1) {
    stage(p0, lane, raw_a);
    if (lane < kStage - 32) stage(p0, lane + 32, raw_b);
    if (it0 + 1 < it1 && lane < U)
      raw_a = load16(seg.seq, p0 + ADV + 16ull * (lane + NC), seq_len, aligned);
  }

  for (uint64_t it = it0; it < it1; ++it, p0 += ADV) {
    // ---------------- staged words of this iteration: into registers ------
    if (lane < 17) {
      S.kill_w[lane] = 0;
      S.own_w[lane] = 0;
    }
    __syncwarp();

    const uint32_t F0 = S.fwd[lane], F1 = S.fwd[lane + 1], F2 = S.fwd[lane + 2];
    const uint32_t R0 = S.rcw[lane + 2], R1 = S.rcw[lane + 1], R2 = S.rcw[lane];
    const uint64_t bad48 = (uint64_t)S.bad[lane] | ((uint64_t)S.bad[lane + 1] << 16) |
                           ((uint64_t)S.bad[lane + 2] << 32);

    // ---------------- read ends inside the window; cursor advance --------
    uint64_t E48 = 0;
    uint64_t adv = 0;
    const uint64_t own_hi = p0 + ADV;
    {
      // every read ending in the window marks its last base in position-space
      // words (pref_w is free until the answers); each lane then reads the
      // 48 positions from its chunk on
      const uint64_t win_hi = p0 + 16ull * kStage;
      if (lane < 17) S.pref_w[lane] = 0;
      __syncwarp();
      uint64_t q0 = r_cur;
      uint64_t e = e_batch;
      while (true) {
        unsigned bw = __ballot_sync(kFull, e < win_hi);
        adv += __popc(__ballot_sync(kFull, e <= own_hi));
        if (e < win_hi && e > p0) {
          const uint32_t d = (uint32_t)(e - 1 - p0);  // last base of that read, < 544
          atomicOr(&S.pref_w[d >> 5], 1u << (d & 31u));
        }
        if (bw != kFull) break;
        q0 += 32;
        e = read_end(q0 + lane);
      }
      __syncwarp();
      const uint64_t w = ((uint64_t)S.pref_w[(lane >> 1) + 1] << 32) | S.pref_w[lane >> 1];
      E48 = (w >> ((lane & 1) * 16)) & 0xFFFFFFFFFFFFull;
    }

    // ---------------- validity of the lane's 16 k-mers --------------------
    uint32_t valid16;
    {
      // invalid(j) <=> an invalid base in [j, j+k-1] or a read's last base in [j, j+k-2]
      uint64_t X = bad48 | (bad48 >> 1) | E48;
      int len = 1;
      while (2 * len <= k - 1) {
        X |= X >> len;
        len *= 2;
      }
      X |= X >> (k - 1 - len);
      valid16 = (uint32_t)(~X) & 0xFFFFu;
      if (lane >= U) valid16 = 0;
    }

    // ---------------- m-mer order keys --------------------------------------
    KeyT key[kLanePos];
#pragma unroll
    for (int j = 0; j < kLanePos; ++j) {
      const uint32_t hi = __funnelshift_l(F1, F0, 2 * j);
      const uint32_t rlo = __funnelshift_r(R2, R1, 2 * j);
      if constexpr (KEY64) {
        const uint32_t lo = __funnelshift_l(F2, F1, 2 * j);
        const uint32_t rhi = __funnelshift_r(R1, R0, 2 * j);
        uint64_t fm = (((uint64_t)hi << 32) | lo) >> (64 - 2 * m);
        uint64_t rm = (((uint64_t)rhi << 32) | rlo) & mmask;
        uint64_t cm = (canon && rm < fm) ? rm : fm;
        key[j] = cm * kGolden64;
      } else {
        uint32_t fm = hi >> (32 - 2 * m);
        uint32_t rm = rlo & (uint32_t)mmask;
        uint32_t cm = (canon && rm < fm) ? rm : fm;
        key[j] = cm * kGolden32;
      }
    }

    // ---------------- sliding minimum over W windows (van Herk) -----------
    constexpr int NE = 15 + W;  // positions 0 .. 15+W-1 of the extended chunk
    KeyT mk[kLanePos];
    {
      KeyT ext[NE];
#pragma unroll
      for (int i = 0; i < NE; ++i) {
        if (i < 16) {
          ext[i] = key[i];
        } else {
          const int src = i < 32 ? i - 16 : i - 32;
          const int dl = i < 32 ? 1 : 2;
          if constexpr (KEY64) {
            uint32_t h = __shfl_down_sync(kFull, (uint32_t)(key[src] >> 32), dl);
            uint32_t l = __shfl_down_sync(kFull, (uint32_t)key[src], dl);
            ext[i] = ((uint64_t)h << 32) | l;
          } else {
            ext[i] = __shfl_down_sync(kFull, key[src], dl);
          }
        }
      }
      // blocks [0, W), [W, 2W), ...: window [j, j+W-1] = suffix minimum of
      // j's block from j, and prefix minimum of the next block up to j+W-1.
      KeyT suf[NE], pre[NE];
#pragma unroll
      for (int i = NE - 1; i >= 0; --i) {
        if (i == NE - 1 || i % W == W - 1) {
          suf[i] = ext[i];
        } else {
          suf[i] = ext[i] < suf[i + 1] ? ext[i] : suf[i + 1];
        }
      }
#pragma unroll
      for (int i = 0; i < NE; ++i) {
        if (i % W == 0) {
          pre[i] = ext[i];
        } else {
          pre[i] = ext[i] < pre[i - 1] ? ext[i] : pre[i - 1];
        }
      }
#pragma unroll
      for (int j = 0; j < kLanePos; ++j) {
        if (j % W == 0) {
          mk[j] = suf[j];
        } else {
          KeyT a = suf[j], b = pre[j + W - 1];
          mk[j] = a < b ? a : b;
        }
      }
    }

    // ---------------- run heads / ends ------------------------------------
    uint32_t eq_prev = 0;  // bit j: mk[j] == mk[j-1] (bit 0: vs previous lane)
#pragma unroll
    for (int j = 1; j < kLanePos; ++j) eq_prev |= (uint32_t)(mk[j] == mk[j - 1]) << j;
    KeyT prev_mk, next_mk;
    if constexpr (KEY64) {
      prev_mk = ((uint64_t)__shfl_up_sync(kFull, (uint32_t)(mk[15] >> 32), 1) << 32) |
                __shfl_up_sync(kFull, (uint32_t)mk[15], 1);
      next_mk = ((uint64_t)__shfl_down_sync(kFull, (uint32_t)(mk[0] >> 32), 1) << 32) |
                __shfl_down_sync(kFull, (uint32_t)mk[0], 1);
    } else {
      prev_mk = __shfl_up_sync(kFull, mk[15], 1);
      next_mk = __shfl_down_sync(kFull, mk[0], 1);
    }
    uint32_t prev_valid = (__shfl_up_sync(kFull, valid16, 1) >> 15) & 1u;
    uint32_t next_valid = __shfl_down_sync(kFull, valid16, 1) & 1u;
    if (lane == 0) {
      prev_valid = carry_valid ? 1u : 0u;
      prev_mk = carry_key;
    }
    eq_prev |= (uint32_t)(prev_mk == mk[0]);
    const uint32_t vprev = ((valid16 << 1) | prev_valid) & 0xFFFFu;
    const uint32_t head16 = valid16 & ~(vprev & eq_prev);
    const uint32_t eq_next = (eq_prev >> 1) | ((uint32_t)(mk[15] == next_mk) << 15);
    const uint32_t vnext = ((valid16 >> 1) | (next_valid << 15)) & 0xFFFFu;
    uint32_t end16 = valid16 & ~(vnext & eq_next);
    if (lane == U - 1) end16 |= valid16 & 0x8000u;  // iteration end closes every run
    const uint32_t slot16 = head16 | (lane == 0 ? (valid16 & 1u) : 0u);
    // carry for the next iteration: position p0 + ADV - 1 = lane U-1, j = 15
    {
      uint32_t cv = __shfl_sync(kFull, valid16 >> 15, U - 1) & 1u;
      KeyT ck;
      if constexpr (KEY64) {
        ck = ((uint64_t)__shfl_sync(kFull, (uint32_t)(mk[15] >> 32), U - 1) << 32) |
             __shfl_sync(kFull, (uint32_t)mk[15], U - 1);
      } else {
        ck = __shfl_sync(kFull, mk[15], U - 1);
      }
      carry_valid = cv != 0;
      carry_key = ck;
    }
    if (!INSERT && P.stats) {
      st_valid += __popc(valid16);
      st_runs += __popc(head16);
    }

    // ---------------- slots: one per run piece ----------------------------
    uint32_t n_slot = __popc(slot16), n_end = __popc(end16);
    uint32_t slot_base = n_slot, end_base = n_end;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t a = __shfl_up_sync(kFull, slot_base, d);
      uint32_t b = __shfl_up_sync(kFull, end_base, d);
      if (lane >= d) {
        slot_base += a;
        end_base += b;
      }
    }
    const uint32_t total_slots = __shfl_sync(kFull, slot_base, 31);
    const uint32_t total_ends = __shfl_sync(kFull, end_base, 31);
    slot_base -= n_slot;
    end_base -= n_end;
    {
      uint32_t sl = slot_base - 1u, en = end_base;
#pragma unroll
      for (int j = 0; j < kLanePos; ++j) {
        const uint32_t t = 16u * lane + j;
        if ((slot16 >> j) & 1u) {
          ++sl;
          S.slot_x[sl] = (typename Sm::SlotT)mk[j];
        }
        if (kFastOwn || ((valid16 >> j) & 1u)) S.slot_of[j * 34 + lane] = (uint16_t)sl;
        if ((end16 >> j) & 1u) S.end_list[en++] = (uint16_t)t;
      }
    }
    reinterpret_cast<uint16_t*>(S.valid_w)[lane] = (uint16_t)valid16;
    reinterpret_cast<uint16_t*>(S.end_w)[lane] = (uint16_t)end16;
    if (lane == 0) {
      S.valid_w[16] = 0;
      S.end_w[16] = 0;
    }
    // prefetch the first batch of read ends of the next iteration
    const uint64_t r_next = (n_reads > 0 && r_cur + adv > n_reads - 1) ? n_reads - 1 : r_cur + adv;
    const uint64_t e_next = read_end(r_next + lane);
    __syncwarp();

    // ---------------- shards of the runs: index, then async copy ----------
    const uint64_t n_shards = g.n_shards;
    const bool masked = g.layout == 1;  // the paper's shard rule: key & (2^P - 1)
    // slots [kTmaFromSlot, min(total, SC)) of a large filter go to the TMA engine
    const uint32_t n_copy = total_slots < (uint32_t)SC ? total_slots : (uint32_t)SC;
    uint32_t n_bulk = 0;
    if constexpr (BULK)
      n_bulk = (n_shards * (uint64_t)(B / 8) >= kTmaMinBytes && n_copy > kTmaFromSlot)
                   ? n_copy - kTmaFromSlot : 0u;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&S.bar);
    if (BULK && n_bulk) {
      // this lane's earlier generic accesses of the slots precede the bulk writes
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      if (lane == 0)
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
                     ::"r"(bar), "r"(n_bulk * (uint32_t)(B / 8)) : "memory");
      __syncwarp();
    }
    for (uint32_t si = lane; si < total_slots; si += 32) {
      uint64_t x;
      if (masked) {
        x = (uint64_t)S.slot_x[si] & (n_shards - 1);
      } else {
        uint64_t mu;
        if constexpr (KEY64) {
          mu = S.slot_x[si] * inv64(kGolden64);
        } else {
          mu = (uint32_t)S.slot_x[si] * inv32(kGolden32);
        }
        x = __umul64hi(mix64(mu ^ kShardKey), n_shards);
      }
      S.slot_x[si] = (typename Sm::SlotT)x;
      if (si < (uint32_t)SC) {
        if constexpr (INSERT) {
#pragma unroll
          for (int w = 0; w < L::W32; w += 4)
            *reinterpret_cast<uint4*>(&S.shard[si * L::SLOT + w]) = make_uint4(0, 0, 0, 0);
        } else {
          const uint8_t* src = reinterpret_cast<const uint8_t*>(g.words) + x * (uint64_t)(B / 8);
          uint32_t dst = (uint32_t)__cvta_generic_to_shared(&S.shard[si * L::SLOT]);
          if (BULK && n_bulk && si >= kTmaFromSlot) {  // 16-byte aligned, B/8 a multiple of 16
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                ::"r"(dst), "l"(src), "n"(B / 8), "r"(bar) : "memory");
          } else {
#pragma unroll
            for (int c = 0; c < B / 128; ++c)
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16 * c),
                           "l"(src + 16 * c));
          }
        }
      }
    }
    if constexpr (!INSERT) asm volatile("cp.async.commit_group;\n" ::);

    // ---------------- s-mer bit-address packs (overlaps the copies) -------
    // s > 16 on this path, so the right shift 64 - 2s is below 32 and the
    // 64-bit extraction is two funnel shifts.  mix64(v ^ K) starts with
    // x ^= x >> 30, which is linear: (v ^ K) ^ ((v ^ K) >> 30) =
    // v ^ (v >> 30) ^ K30 with the constant K30 = K ^ (K >> 30).
    constexpr uint64_t K30 = kSmerKey ^ (kSmerKey >> 30);
    const uint32_t sh_s = 64u - 2u * (uint32_t)s;
    const uint32_t smask_hi = (uint32_t)(smask >> 32);
    // four positions per step: with 64-bit order keys a fully unrolled loop
    // made inserts 6-8% and queries 3-6% slower (code size)
    constexpr int kHashUnroll = 4;
#pragma unroll kHashUnroll
    for (int j = 0; j < kLanePos; ++j) {
      const uint32_t hi = __funnelshift_l(F1, F0, 2 * j);
      const uint32_t lo = __funnelshift_l(F2, F1, 2 * j);
      const uint32_t rlo = __funnelshift_r(R2, R1, 2 * j);
      const uint32_t rhi = __funnelshift_r(R1, R0, 2 * j) & smask_hi;
      const uint32_t flo = __funnelshift_r(lo, hi, sh_s);
      const uint32_t fhi = hi >> sh_s;
      const bool use_rc = canon && (rhi < fhi || (rhi == fhi && rlo < flo));
      const uint64_t cs = use_rc ? (((uint64_t)rhi << 32) | rlo) : (((uint64_t)fhi << 32) | flo);
      uint64_t x = cs ^ (cs >> 30) ^ K30;
      x *= kMixMul1;
      x ^= x >> 27;
      x *= kMixMul2;
      x ^= x >> 31;
      S.hs[j * HS + lane] = make_pack<H, B>(x);
    }
    if constexpr (!INSERT) asm volatile("cp.async.wait_group 0;\n" ::);
    if (BULK && n_bulk) {
      if (!__all_sync(kFull, wait_phase(bar, bar_phase))) {
        // give up: record it, let copies still in flight land (bounded), stop
        if (lane == 0 && g.status) atomicOr(g.status, 1u);
        wait_phase(bar, bar_phase);
        return false;
      }
      bar_phase ^= 1u;
    }
    __syncwarp();

    // ---------------- pair tests / sets ------------------------------------
    auto test_pair = [&](Pack pk, uint32_t slot) -> bool {
      if (slot < (uint32_t)SC) return test_slot<H, B>(&S.shard[slot * L::SLOT], pk) != 0u;
      uint32_t acc = 1u;
      const uint32_t* gp = words32 + S.slot_x[slot] * (uint64_t)L::W32;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const uint32_t p = pack_addr<H, B>(pk, i);
        const uint32_t w = __ldg(gp + (i % L::S) * L::SW32 + (p >> 5));
        acc &= __funnelshift_r(w, w, p);
      }
      return acc & 1u;
    };
    auto set_pair = [&](Pack pk, uint32_t slot) {
      if (slot < (uint32_t)SC) {
        set_slot_rot<H, B>(&S.shard[slot * L::SLOT], pk, (uint32_t)lane & (uint32_t)(H - 1));
      } else {
        uint32_t* gp = words32 + S.slot_x[slot] * (uint64_t)L::W32;
#pragma unroll
        for (int i = 0; i < H; ++i) {
          const uint32_t p = pack_addr<H, B>(pk, i);
          atomicOr(&gp[(i % L::S) * L::SW32 + (p >> 5)], 1u << (p & 31u));
        }
      }
    };

    // own pairs (t, shard(t)), position-per-lane: t = 32*pass + lane, so
    // t & 15 = lane & 15 and t >> 4 = 2*pass + (lane >> 4); lanes of one pass
    // mostly share a few run slots, so their shard reads broadcast.  Two
    // passes per step for independent work.
    if constexpr (kFastOwn) {
      // Own bits of invalid positions are never read: the AND below takes
      // position t + d only while t + d is in t's run (all valid), and the
      // answer word keeps valid positions only.  So no lane masks its test.
      const uint32_t hs_i0 = (lane & 15u) * HS + (lane >> 4);
      const uint32_t so_i0 = (lane & 15u) * 34 + (lane >> 4);
      if (total_slots <= (uint32_t)SC) {
        // every run has a shared copy; an invalid position's slot entry
        // (written, but of no run) is reduced into range
        constexpr bool kPow2 = (SC & (SC - 1)) == 0;
        constexpr uint32_t kMask = kPow2 ? (uint32_t)(SC - 1) : 0xFFFFFFFFu;
#pragma unroll 4
        for (int pass = 0; pass < 16; pass += 2) {
          uint32_t sla = S.slot_of[so_i0 + 2 * pass] & kMask;
          uint32_t slb = S.slot_of[so_i0 + 2 * pass + 2] & kMask;
          if constexpr (!kPow2) {
            sla = sla < (uint32_t)SC ? sla : 0u;
            slb = slb < (uint32_t)SC ? slb : 0u;
          }
          const unsigned own_a = __ballot_sync(
              kFull, test_slot<H, B>(&S.shard[sla * L::SLOT], S.hs[hs_i0 + 2 * pass]) != 0u);
          const unsigned own_b = __ballot_sync(
              kFull, test_slot<H, B>(&S.shard[slb * L::SLOT], S.hs[hs_i0 + 2 * pass + 2]) != 0u);
          if (lane == 0) {
            S.own_w[pass] = own_a;
            S.own_w[pass + 1] = own_b;
          }
        }
      } else {
        // some runs test against global memory: invalid positions test slot
        // 0, since their entry may index past the runs
#pragma unroll 2
        for (int pass = 0; pass < 16; pass += 2) {
          const uint32_t va = (S.valid_w[pass] >> lane) & 1u;
          const uint32_t vb = (S.valid_w[pass + 1] >> lane) & 1u;
          const uint32_t sla = va ? (uint32_t)S.slot_of[so_i0 + 2 * pass] : 0u;
          const uint32_t slb = vb ? (uint32_t)S.slot_of[so_i0 + 2 * pass + 2] : 0u;
          const unsigned own_a = __ballot_sync(kFull, test_pair(S.hs[hs_i0 + 2 * pass], sla));
          const unsigned own_b = __ballot_sync(kFull, test_pair(S.hs[hs_i0 + 2 * pass + 2], slb));
          if (lane == 0) {
            S.own_w[pass] = own_a;
            S.own_w[pass + 1] = own_b;
          }
        }
      }
    } else {
      // invalid positions test slot 0 (their slot entry may be stale) and
      // are masked out
      const uint32_t hs_i0 = (lane & 15u) * HS + (lane >> 4);
      const uint32_t so_i0 = (lane & 15u) * 34 + (lane >> 4);
#pragma unroll 2
      for (int pass = 0; pass < 16; pass += 2) {
        const uint32_t va = (S.valid_w[pass] >> lane) & 1u;
        const uint32_t vb = (S.valid_w[pass + 1] >> lane) & 1u;
        const Pack pka = S.hs[hs_i0 + 2 * pass];
        const Pack pkb = S.hs[hs_i0 + 2 * pass + 2];
        const uint32_t sla = va ? (uint32_t)S.slot_of[so_i0 + 2 * pass] : 0u;
        const uint32_t slb = vb ? (uint32_t)S.slot_of[so_i0 + 2 * pass + 2] : 0u;
        if constexpr (INSERT) {
          if (va) set_pair(pka, sla);
          if (vb) set_pair(pkb, slb);
        } else {
          const bool oka = ((uint32_t)test_pair(pka, sla) & va) != 0u;
          const bool okb = ((uint32_t)test_pair(pkb, slb) & vb) != 0u;
          const unsigned own_a = __ballot_sync(kFull, oka);
          const unsigned own_b = __ballot_sync(kFull, okb);
          if (lane == 0) {
            S.own_w[pass] = own_a;
            S.own_w[pass + 1] = own_b;
          }
        }
      }
    }

    // extra pairs after each run end e: (e+d, shard(e)), d = 1..z.  A failure
    // at d kills the run's k-mers [max(e+d-z, head), e]; the smallest failing
    // d gives the largest range, so testing stops there.  Every slot holds
    // one run piece with one end, and slots and ends are both numbered in
    // position order, so end i belongs to slot i.  Every valid position
    // between run i-1's end and run i's head would be in a run, so none is:
    // the position after end i-1 serves as the head (the positions it adds
    // to a kill range are invalid, and answers keep valid positions only).
    for (uint32_t ei = lane; ei < total_ends; ei += 32) {
      const uint32_t e = S.end_list[ei];
      const uint32_t slot = ei;
      if constexpr (INSERT) {
        for (int d = 1; d <= z; ++d) {
          const uint32_t t = e + d;
          set_pair(S.hs[(t & 15u) * HS + (t >> 4)], slot);
        }
      } else {
        int fail = 0;
        for (int d = 1; d <= z; ++d) {
          const uint32_t t = e + d;
          if (!test_pair(S.hs[(t & 15u) * HS + (t >> 4)], slot)) {
            fail = d;
            break;
          }
        }
        if (fail) {
          int lo = (int)e + fail - z;
          const int hd = ei > 0 ? (int)S.end_list[ei - 1] + 1 : 0;
          if (lo < hd) lo = hd;
          const uint32_t w1 = (uint32_t)lo >> 5, w2 = e >> 5;
          const uint32_t bl = (uint32_t)lo & 31u, bh = e & 31u;
          if (w1 == w2) {
            atomicOr(&S.kill_w[w1], (0xFFFFFFFFu >> (31u - bh)) & (0xFFFFFFFFu << bl));
          } else {
            atomicOr(&S.kill_w[w1], 0xFFFFFFFFu << bl);
            atomicOr(&S.kill_w[w2], 0xFFFFFFFFu >> (31u - bh));
          }
        }
      }
    }
    __syncwarp();

    if constexpr (INSERT) {
      // ---------------- flush run masks: coalesced 64-bit atomics ----------
      const uint32_t n_mem = total_slots < (uint32_t)SC ? total_slots : (uint32_t)SC;
      constexpr uint32_t W64 = B / 64;
      const uint32_t n_words = n_mem * W64;
      for (uint32_t i = lane; i < n_words; i += 32) {
        const uint32_t si = i / W64, wd = i % W64;
        const uint64_t v = *reinterpret_cast<const uint64_t*>(&S.shard[si * L::SLOT + 2 * wd]);
        if (v)
          atomicOr(reinterpret_cast<unsigned long long*>(g.words) + S.slot_x[si] * (uint64_t)W64 + wd,
                   (unsigned long long)v);
      }
    } else {
      // ---------------- Findere AND inside runs -> answer words -----------
      if (lane < 16) {
        const uint64_t O64 = (uint64_t)S.own_w[lane] | ((uint64_t)S.own_w[lane + 1] << 32);
        const uint64_t E64 = (uint64_t)S.end_w[lane] | ((uint64_t)S.end_w[lane + 1] << 32);
        uint64_t res = O64, c = 0;
        for (int d = 1; d <= z; ++d) {
          c |= E64 >> (d - 1);
          res &= (O64 >> d) | c;
        }
        const uint32_t K = (uint32_t)res & ~S.kill_w[lane] & S.valid_w[lane];
        S.k_w[lane] = K;
        if (P.stats) st_pos += __popc(K);
        // output: bits of positions p0 + 32*lane + b
        if (K && seg.bits) {
          const uint64_t gpos = p0 + 32ull * lane;
          const uint32_t sh = (uint32_t)(gpos & 31u);
          const uint64_t gword = gpos >> 5;
          if (sh == 0) {
            atomicOr(&seg.bits[gword], K);
          } else {
            const uint32_t a = K << sh, b = K >> (32u - sh);
            if (a) atomicOr(&seg.bits[gword], a);
            if (b) atomicOr(&seg.bits[gword + 1], b);
          }
        }
      }
      // per-read hit counts from prefix popcounts of the answer words.
      // Batch 0 reuses the prefetched read ends: read q = r_cur + lane spans
      // [end of q-1, end of q).  Reads of at most P.hits_above positions are
      // left to the short-read pass; an iteration that holds no other read
      // (and no second batch) skips the counting.
      uint64_t q0 = r_cur;
      uint64_t re = e_batch;
      uint64_t rs = __shfl_up_sync(kFull, re, 1);
      if (lane == 0) rs = r_cur_start;
      const uint64_t ha = P.hits_above;
      bool count_here = seg.hits != nullptr;
      if (count_here && ha != 0) {
        const bool mine = q0 + lane < n_reads && rs < own_hi && re > p0 && re - rs > ha;
        count_here = __any_sync(kFull, mine) || __all_sync(kFull, re < own_hi);
      }
      if (count_here) {
        __syncwarp();
        const uint32_t pc = lane < 16 ? __popc(S.k_w[lane]) : 0u;
        uint32_t incl = pc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          uint32_t a = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += a;
        }
        if (lane < 16) S.pref_w[lane] = incl - pc;
        if (lane == 16) {
          S.pref_w[16] = incl;  // lane 16 holds the total (pc = 0 there)
          S.k_w[16] = 0;
        }
        __syncwarp();
        auto bits_before = [&](uint32_t x) -> uint32_t {  // x in [0, 512]
          const uint32_t w = x >> 5, b = x & 31u;
          return S.pref_w[w] + (b ? __popc(S.k_w[w] & (0xFFFFFFFFu >> (32u - b))) : 0u);
        };
        while (true) {
          const uint64_t q = q0 + lane;
          if (q < n_reads && rs < own_hi && re > p0 && (ha == 0 || re - rs > ha)) {
            const uint64_t a = rs > p0 ? rs - p0 : 0;
            const uint64_t b = (re < own_hi ? re : own_hi) - p0;
            if (b > a) {
              const uint32_t cnt = bits_before((uint32_t)b) - bits_before((uint32_t)a);
              if (cnt) atomicAdd(&seg.hits[q], cnt);
            }
          }
          const unsigned more = __ballot_sync(kFull, re < own_hi);
          if (more != kFull) break;
          const uint64_t last_end = __shfl_sync(kFull, re, 31);
          q0 += 32;
          re = read_end(q0 + lane);
          rs = __shfl_up_sync(kFull, re, 1);
          if (lane == 0) rs = last_end;
        }
      }
    }
    // advance the read cursor (adv is warp-uniform): the new current read
    // starts where read r_next - 1 ends
    if (adv > 0) {
      if (r_cur + adv > r_next || adv > 32) {
        const uint64_t st = off[r_next];
        r_cur_start = st < seq_len ? st : seq_len;
      } else {
        r_cur_start = __shfl_sync(kFull, e_batch, (int)(adv - 1));
      }
    }
    r_cur = r_next;
    e_batch = e_next;
    // ---------------- the next iteration's words ---------------------------
    if (it + 1 < it1) {
      uint32_t cf = 0, cr = 0, cb = 0;
      if (lane < NC) {
        cf = S.fwd[U + lane];
        cr = S.rcw[U + lane];
        cb = S.bad[U + lane];
      }
      __syncwarp();
      if (lane < NC) {
        S.fwd[lane] = cf;
        S.rcw[lane] = cr;
        S.bad[lane] = cb;
      }
      if (lane < U) stage(p0 + ADV, lane + NC, raw_a);
      if (it + 2 < it1 && lane < U)
        raw_a = load16(seg.seq, p0 + 2 * ADV + 16ull * (lane + NC), seq_len, aligned);
    }
    __syncwarp();
  }
  return true;
}

// Blocks per SM the register budget is sized for: four (128 registers) in
// general; three (up to 168, no spills) for 64-bit order keys where that
// measured faster -- inserts, and queries on 512-bit shards.
template <bool KEY64, bool INSERT, int B>
constexpr int min_blocks() {
  return (KEY64 && (INSERT || B == 512)) ? 3 : 4;
}

template <int W, int H, int B, bool KEY64, bool INSERT, bool BULK>
__global__ void __launch_bounds__(kThreads, min_blocks<KEY64, INSERT, B>()) fused_kernel(Params P) {
  static_assert(!(INSERT && BULK), "bulk shard copies are a query variant");
  using Sm = WarpSmem<slot_cap<W, INSERT, B>(), H, B, KEY64>;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Sm& S = reinterpret_cast<Sm*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  unsigned long long st_valid = 0, st_runs = 0, st_pos = 0;
  uint32_t bar_phase = 0;  // phase of the warp's shard-copy barrier
  bool alive = true;       // false once a wait ran out
  if constexpr (BULK) {
    if (lane == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&S.bar)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncwarp();
  }

  // Walk global iterations [a, b): split them at segment boundaries.
  auto walk = [&](uint64_t a, uint64_t b) {
    uint32_t si = 0;
    if (P.segs) {  // last segment with iter_begin <= a (warp-uniform)
      uint32_t lo = 0, hi = P.n_segs;
      while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (P.segs[mid].iter_begin <= a) lo = mid; else hi = mid;
      }
      si = lo;
    }
    while (a < b) {
      const Segment seg = P.segs ? P.segs[si] : P.seg0;
      const uint64_t s_end = seg.iter_begin + seg.iters;
      const uint64_t e = b < s_end ? b : s_end;
      if (a < e && !run_range<W, H, B, KEY64, INSERT, BULK>(S, P, seg, a - seg.iter_begin,
                                                      e - seg.iter_begin, lane, st_valid, st_runs,
                                                      st_pos, bar_phase)) {
        alive = false;
        return;
      }
      a = e > a ? e : a;
      if (a >= s_end) ++si;
      if (P.segs == nullptr || si >= P.n_segs) break;
    }
  };

  const uint64_t tw = (uint64_t)gridDim.x * kWarps;
  const uint64_t gw = (uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (P.work == nullptr) {
    // static split: each warp a contiguous share of the iterations
    const uint64_t per = P.iters / tw, rem = P.iters % tw;
    const uint64_t a = gw * per + (gw < rem ? gw : rem);
    const uint64_t b = a + per + (gw < rem ? 1 : 0);
    if (a < b) walk(a, b);
  } else {
    // dynamic: claim chunks of iterations from a global counter
    while (alive) {
      uint64_t start = 0;
      if (lane == 0) start = (uint64_t)atomicAdd(P.work, (unsigned long long)P.chunk);
      start = __shfl_sync(kFull, start, 0);
      if (start >= P.iters) break;
      const uint64_t end = start + P.chunk < P.iters ? start + P.chunk : P.iters;
      walk(start, end);
    }
  }

  if constexpr (BULK) {
    __syncwarp();
    if (alive && lane == 0)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&S.bar)) : "memory");
  }
  if (!INSERT && P.stats) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      st_valid += __shfl_down_sync(kFull, st_valid, d);
      st_runs += __shfl_down_sync(kFull, st_runs, d);
      st_pos += __shfl_down_sync(kFull, st_pos, d);
    }
    if (lane == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats[0]), st_valid);
      atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats[1]), st_runs);
      atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats[2]), st_pos);
    }
  }
}

template <int W, int H, int B, bool KEY64, bool INSERT, bool BULK = false>
cudaError_t launch(const Params& P, cudaStream_t st) {
  auto kern = fused_kernel<W, H, B, KEY64, INSERT, BULK>;
  constexpr size_t smem = sizeof(WarpSmem<slot_cap<W, INSERT, B>(), H, B, KEY64>) * kWarps;
  static int blocks_per_sm = 0;  // per instantiation; same on every GB300
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    blocks_per_sm = nb > 0 ? nb : 1;
  }
  if (P.iters == 0) return cudaSuccess;
  uint64_t want_blocks = (P.iters + kWarps - 1) / kWarps;
  uint64_t cap = (uint64_t)sm_count() * blocks_per_sm;
  if (P.grid_blocks > 0 && P.grid_blocks < cap) cap = P.grid_blocks;
  int grid = (int)(want_blocks < cap ? want_blocks : cap);
  if (grid < 1) grid = 1;
  kern<<<grid, kThreads, smem, st>>>(P);
  return cudaGetLastError();
}

// True if a filter has kTmaMinBytes or more (its queries take the BULK kernels).
inline bool is_big(const Geom& g) {
  return g.n_shards * (uint64_t)(g.shard_bits / 8) >= kTmaMinBytes;
}

// Launch a prepared parameter block (dispatch over the compiled grid).
cudaError_t launch_params(const Params& P, bool insert, cudaStream_t st);
// Reads of at most this many positions have their hits counted from the
// answer words by short_read_hits when a query writes both outputs.
constexpr uint32_t kShortReadMax = 2048;
// Below this many start positions per launch the query kernel counts every
// read itself: the second launch's fixed cost (about 10-20 us) exceeds what
// it saves (about 0.3 ns per position).
constexpr uint64_t kHitsPassMinPositions = 1ull << 26;
// hits_above for a query launch over `positions` start positions that writes
// both outputs (0 otherwise).  SBF_HITS_PASS_MIN_POSITIONS overrides the
// minimum (the tests set 0 to run the pass on small inputs).
uint32_t hits_above_for(uint64_t positions, bool both_outputs);
// The short-read pass of a query launched with hits_above = `above`: hits of
// the reads of at most `above` positions, from the answer words `bits`
// (indexed by position; one thread per read).  Launch it after the query
// kernel on the same stream; it does nothing when above is 0.
cudaError_t short_read_hits(const uint32_t* bits, const uint64_t* off, uint64_t n_reads,
                            uint64_t seq_len, uint32_t above, uint32_t* hits, cudaStream_t st);
// Start positions covered by one iteration for these parameters.
int advance_of(const Geom& g);

}  // namespace fused
}  // namespace sbf
