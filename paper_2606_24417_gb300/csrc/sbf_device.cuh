// sbf_device.cuh -- device-side definition of the Super Bloom filter's hashes
// and layout, shared by all kernels of the library.
//
// cuSBF paper references: 2-bit packing with the first base most significant
// (Sec. IV-C), minimizer by one multiplicative mix and s-mer hash by a
// stronger xorshift-multiply mix (Sec. IV-G "role-specialised hashing"),
// sectorised shards with hash i in sector i mod S (Sec. IV-B), bit-slicing
// and the salted-multiply fallback (Sec. IV-G), Findere AND (Eq. 2, Alg. 2).
//
// Constants: Knuth's golden-ratio multiplier floor(2^64/phi) (and its top 32
// bits), the SplitMix64 finaliser (Steele, Lea & Flood 2014), and Knuth's
// MMIX LCG multiplier / increment as the s-mer and shard keys.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace sbf {

constexpr uint64_t kGolden64 = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kGolden32 = 0x9E3779B9u;
constexpr uint64_t kMixMul1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMixMul2 = 0x94D049BB133111EBull;
constexpr uint64_t kSmerKey = 0x5851F42D4C957F2Dull;   // 6364136223846793005
constexpr uint64_t kShardKey = 0x14057B7EF767814Full;  // 1442695040888963407

// Runtime description of one filter, passed by value to kernels.
struct Geom {
  uint64_t* words;     // N * W uint64 words
  uint64_t n_shards;   // N
  int k, m, s, H;
  int shard_bits;      // B
  int canonical;
  int layout;          // 0: this library's layout; 1: the paper's literal one
  int alphabet;        // 0: DNA; 1: protein; 2: DNA triplets (Sec. IV-A)
  int sym_bits;        // bits per symbol: 2, 5, 6
  int sym_bytes;       // bytes per symbol: 1, 1, 3
  int sectors;         // S = largest power of two <= min(H, B/64); B/64 for layout 1
  int sector_bits;     // B / S
  int sector_log2;     // b = log2(B / S)
  int slice;           // q = floor(64 / H)
  uint32_t* status;    // device word: nonzero after a kernel stopped on a timed-out wait, or NULL
};

// Layout 1 is Sec. IV-B and Alg. 1/2 taken literally: 2^P shards (the caller
// rounds N up), shard = minimizer order key & (N - 1), and every 64-bit word
// is a sector (hash i in word i mod W; with H < W some words stay unused).
// Alphabets (Sec. IV-A): DNA (A/C/G/T -> 0..3, 2 bits), protein (A..Z either
// case -> 0..25, 5 bits), DNA triplets (three DNA bytes -> 16 c0 + 4 c1 + c2,
// 6 bits).  Packing, sub-windows and the order key's width follow the symbol
// width; a read's k-mers start at its first byte and every symbol after.
__host__ __device__ inline Geom make_geom(uint64_t* words, uint64_t n_shards, int k, int m, int s,
                                          int H, int shard_bits, int canonical, int layout = 0,
                                          int alphabet = 0) {
  Geom g;
  g.words = words;
  g.n_shards = n_shards;
  g.k = k; g.m = m; g.s = s; g.H = H;
  g.shard_bits = shard_bits;
  g.canonical = canonical;
  g.layout = layout;
  g.alphabet = alphabet;
  g.sym_bits = alphabet == 1 ? 5 : alphabet == 2 ? 6 : 2;
  g.sym_bytes = alphabet == 2 ? 3 : 1;
  int W = shard_bits / 64;
  int lim = H < W ? H : W;  // sectors: the largest power of two not above min(H, W)
  g.sectors = 1;
  while (2 * g.sectors <= lim) g.sectors *= 2;
  if (layout == 1) g.sectors = W;
  g.sector_bits = shard_bits / g.sectors;
  int b = 0;
  while ((1 << b) < g.sector_bits) ++b;
  g.sector_log2 = b;
  g.slice = 64 / H;
  g.status = nullptr;
  return g;
}

// SplitMix64 finaliser.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= kMixMul1;
  x ^= x >> 27;
  x *= kMixMul2;
  x ^= x >> 31;
  return x;
}

// 2-bit code of an ASCII base: ((c >> 1) ^ (c >> 2)) & 3 maps A/a->0, C/c->1,
// G/g->2, T/t->3.  Validity is checked separately.
__device__ __forceinline__ uint32_t base_code(uint32_t ch) { return ((ch >> 1) ^ (ch >> 2)) & 3u; }

__device__ __forceinline__ bool base_valid(uint32_t ch) {
  uint32_t lc = ch | 0x20u;
  return lc == 'a' || lc == 'c' || lc == 'g' || lc == 't';
}

// Minimizer order key of a canonical m-mer of m_bits bits: bijective
// multiplicative hash in the narrowest machine word holding them.
__device__ __forceinline__ uint64_t order_key(uint64_t v, int m_bits) {
  return (m_bits <= 32) ? (uint64_t)((uint32_t)v * kGolden32) : v * kGolden64;
}

__device__ __forceinline__ uint64_t shard_of(uint64_t mu, uint64_t n_shards) {
  return __umul64hi(mix64(mu ^ kShardKey), n_shards);
}

// Shard of minimizer mu under either layout (layout 1: n_shards is 2^P).
__device__ __forceinline__ uint64_t shard_of(const Geom& g, uint64_t mu) {
  if (g.layout == 1) return order_key(mu, g.m * g.sym_bits) & (g.n_shards - 1);
  return shard_of(mu, g.n_shards);
}

__device__ __forceinline__ uint64_t smer_hash(uint64_t v) { return mix64(v ^ kSmerKey); }

// Bit index inside a shard for hash function i (runtime geometry).
__device__ __forceinline__ uint32_t bit_in_shard(const Geom& g, uint64_t h, int i) {
  uint32_t p;
  if (g.slice >= g.sector_log2) {
    p = (uint32_t)(h >> (i * g.slice)) & (uint32_t)(g.sector_bits - 1);
  } else {
    uint64_t salt = kGolden64 * (uint64_t)(2 * i + 1);
    p = (uint32_t)((h * salt) >> (64 - g.sector_log2));
  }
  return (uint32_t)(i % g.sectors) * (uint32_t)g.sector_bits + p;
}

__device__ __forceinline__ uint64_t len_mask(int len) {
  return len >= 32 ? ~0ull : ((1ull << (2 * len)) - 1ull);
}

__device__ __forceinline__ uint64_t bit_mask(int nbits) {
  return nbits >= 64 ? ~0ull : ((1ull << nbits) - 1ull);
}

// Code of the symbol at x, or -1 if it is not in the alphabet.
__device__ __forceinline__ int symbol_code(const Geom& g, const uint8_t* x) {
  if (g.alphabet == 1) {
    const uint32_t u = (uint32_t)(x[0] | 0x20u) - (uint32_t)'a';  // either case
    const uint32_t c = x[0];
    return (u < 26u && ((c >= 'A' && c <= 'Z') || (c >= 'a' && c <= 'z'))) ? (int)u : -1;
  }
  if (g.alphabet == 2) {
    if (!base_valid(x[0]) || !base_valid(x[1]) || !base_valid(x[2])) return -1;
    return (int)(16u * base_code(x[0]) + 4u * base_code(x[1]) + base_code(x[2]));
  }
  return base_valid(x[0]) ? (int)base_code(x[0]) : -1;
}

}  // namespace sbf
