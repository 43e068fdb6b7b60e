// sbf_rolling.cu -- insert / query kernels for every parameter set outside
// the fused grid (protein and DNA-triplet alphabets, H in {3, 5..7, 12, 16},
// windows w = k - m + 1 other than 12, 16, 18, 20), with the bits of Alg. 1
// and Alg. 2.
//
// One thread owns a chunk of 32 consecutive start positions (one answer
// word).  It finds the read of its first position once, then walks the
// chunk's reads with a rolling k-mer: each symbol is decoded once and
// shifted in (Sec. IV-C packing, first symbol most significant), instead of
// re-packing k symbols and re-searching the read table per k-mer.  The
// minimizer slides too: a full scan of the k - m + 1 windows only when the
// window holding the smallest key leaves the k-mer (about every (w+1)/2
// positions on random sequence), one new window otherwise.
//
// Consecutive valid k-mers of one read with the same shard share their
// s-mers' tests: k-mer j needs s-mers j..j+z (z = k - s) in shard(j), so
// within such a run every s-mer is hashed and tested (or set) once.  The
// query keeps the next untested s-mer and the last failing one: k-mer j is
// positive iff no s-mer of [j, j + z] failed; testing stops at a failure and
// resumes after it for the next k-mer past it; the run's shard is copied to
// shared memory with 16-byte loads when the run starts and tested there.  The
// insert sets each s-mer's H bits once per run instead of once per k-mer.
//
// The answer word of a chunk has exactly one owner, so it is stored without
// an atomic (and covers positions where no k-mer starts with zeros); read hit
// counts are added once per read segment of the chunk.
#include "sbf_internal.h"

namespace sbf {
namespace {

constexpr int kChunk = 32;    // start positions per thread (one answer word)
constexpr int kThreads = 256; // threads per block

// Symbols are 1 byte (DNA, protein) or 3 bytes (DNA triplets): divisions by
// the symbol width as a multiply by a constant, not a general division.
__device__ __forceinline__ int div_sb(uint64_t x, uint64_t sb) {
  return (int)(sb == 1 ? x : x / 3);
}
__device__ __forceinline__ uint64_t mod_sb(uint64_t x, uint64_t sb) { return sb == 1 ? 0 : x % 3; }

__device__ __forceinline__ uint64_t first_read(const uint64_t* off, uint64_t n_reads, uint64_t p) {
  uint64_t lo = 0, hi = n_reads;  // last r with off[r] <= p, or 0
  while (hi - lo > 1) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t sub_value(const Geom& g, uint64_t fwd, uint64_t rc, int i,
                                              int len) {
  const uint64_t f = (fwd >> (g.sym_bits * (g.k - len - i))) & bit_mask(g.sym_bits * len);
  if (!g.canonical) return f;
  const uint64_t r = (rc >> (2 * i)) & len_mask(len);
  return f < r ? f : r;
}

__device__ __forceinline__ uint64_t min_of(const Geom& g, uint64_t fwd, uint64_t rc) {
  uint64_t best = 0, mu = 0;
  for (int i = 0; i <= g.k - g.m; ++i) {
    const uint64_t v = sub_value(g, fwd, rc, i, g.m);
    const uint64_t key = order_key(v, g.m * g.sym_bits);
    if (i == 0 || key < best) {
      best = key;
      mu = v;
    }
  }
  return mu;
}

// All H bits of hash h set in the shard whose words this thread copied to
// shared memory (word w at sw[w * kThreads])?
__device__ __forceinline__ bool test_bits_shared(const Geom& g, const uint64_t* sw, uint64_t h) {
  for (int i = 0; i < g.H; ++i) {
    const uint32_t b = bit_in_shard(g, h, i);
    if (!((sw[(b >> 6) * kThreads] >> (b & 63)) & 1ull)) return false;
  }
  return true;
}

// Insert: the H bits of hash h in shard `base` (bit index of its first bit).
// (Accumulating a run's bits in shared memory and OR-ing each word once per
// run measured 3% slower than these atomics, which the memory system merges.)
__device__ __forceinline__ void set_bits(const Geom& g, uint64_t base, uint64_t h) {
  for (int i = 0; i < g.H; ++i) {
    const uint64_t bit = base + bit_in_shard(g, h, i);
    atomicOr(reinterpret_cast<unsigned long long*>(g.words + (bit >> 6)), 1ull << (bit & 63));
  }
}

// Minimizer of the k-mer at byte p straight from memory (previous chunk's
// last k-mer, for the run statistics only); false if no valid k-mer starts there.
__device__ bool kmer_min_at(const Geom& g, const uint8_t* seq, uint64_t rs, uint64_t re, uint64_t p,
                            uint64_t& mu) {
  const uint64_t sb = (uint64_t)g.sym_bytes;
  if (p < rs || mod_sb(p - rs, sb) != 0 || p + (uint64_t)g.k * sb > re) return false;
  uint64_t fwd = 0, rc = 0;
  for (int i = 0; i < g.k; ++i) {
    const int c = symbol_code(g, seq + p + (uint64_t)i * sb);
    if (c < 0) return false;
    fwd = (fwd << g.sym_bits) | (uint64_t)c;
    if (g.alphabet == 0) rc |= (uint64_t)(3 - c) << (2 * i);
  }
  mu = min_of(g, fwd, rc);
  return true;
}

template <bool INSERT>
__global__ void __launch_bounds__(kThreads) rolling_kernel(Geom g, const uint8_t* __restrict__ seq,
                                                      uint64_t seq_len,
                                                      const uint64_t* __restrict__ off,
                                                      uint64_t n_reads, uint32_t* __restrict__ bits,
                                                      uint32_t* __restrict__ hits,
                                                      uint64_t* __restrict__ stats) {
  const uint64_t n_chunks = (seq_len + kChunk - 1) / kChunk;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t sb = (uint64_t)g.sym_bytes;
  const int z = g.k - g.s;
  const uint64_t kmask = bit_mask(g.k * g.sym_bits);
  const uint64_t span = (uint64_t)g.k * sb;  // bytes of one k-mer
  const int n_win = g.k - g.m + 1;           // m-mer windows of a k-mer
  unsigned long long n_valid = 0, n_runs = 0, n_pos = 0;
  // query: each thread's copy of its current run's shard (up to 8 words),
  // word-major so that a warp's accesses to one word index are conflict-free;
  // a run loads its shard once with 16-byte loads instead of testing bits in
  // global memory one s-mer at a time
  __shared__ uint64_t shard_copy[INSERT ? 1 : 8 * kThreads];
  uint64_t* const sw = shard_copy + (INSERT ? 0 : threadIdx.x);
  const int shard_words = g.shard_bits / 64;
  for (uint64_t ch = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks; ch += stride) {
    const uint64_t c0 = ch * kChunk;
    const uint64_t c1 = c0 + kChunk < seq_len ? c0 + kChunk : seq_len;
    uint32_t word = 0;
    uint64_t r = n_reads ? first_read(off, n_reads, c0) : 0;
    while (n_reads && r < n_reads) {
      const uint64_t rs = off[r] < seq_len ? off[r] : seq_len;
      const uint64_t re0 = off[r + 1] < seq_len ? off[r + 1] : seq_len;
      const uint64_t re = re0 > rs ? re0 : rs;
      if (rs >= c1) break;
      uint64_t p = c0 > rs ? c0 : rs;
      if (sb > 1) p += (sb - mod_sb(p - rs, sb)) % sb;  // the read's symbol frame
      const uint64_t p_end = c1 < re ? c1 : re;
      uint32_t cnt = 0;
      if (p < p_end && p + span <= re) {
        // rolling k-mer: symbols [p, p + (k-1) sb) first, then one per step
        uint64_t fwd = 0, rc = 0;
        int good = 0;
        uint64_t q = p;
        for (int i = 0; i < g.k - 1; ++i, q += sb) {
          const int c = symbol_code(g, seq + q);
          if (c < 0) {
            good = 0;
          } else {
            fwd = ((fwd << g.sym_bits) | (uint64_t)c) & kmask;
            if (g.alphabet == 0) rc = (rc >> 2) | ((uint64_t)(3 - c) << (2 * (g.k - 1)));
            ++good;
          }
        }
        bool in_run = false;     // a run of one shard is open at the previous position
        uint64_t run_x = 0, next_t = 0, last_fail = 0, prev_mu = 0;
        bool has_fail = false;
        bool prev_valid = false; // the previous position's k-mer was valid (same read)
        // sliding minimum of the previous position's k-mer: smallest order key,
        // its m-mer and its window index (keys are a bijection of m-mers, so
        // equal keys are equal m-mers)
        bool have_min = false;
        uint64_t min_key = 0, min_val = 0;
        int min_pos = 0;
        if (!INSERT && stats && p >= rs + sb)     // run heads across the chunk edge
          prev_valid = kmer_min_at(g, seq, rs, re, p - sb, prev_mu);
        for (; p < p_end && p + span <= re; p += sb, q += sb) {
          const int c = symbol_code(g, seq + q);
          if (c < 0) {
            good = 0;
          } else {
            fwd = ((fwd << g.sym_bits) | (uint64_t)c) & kmask;
            if (g.alphabet == 0) rc = (rc >> 2) | ((uint64_t)(3 - c) << (2 * (g.k - 1)));
            ++good;
          }
          if (good < g.k) {
            prev_valid = false;
            in_run = false;
            have_min = false;
            continue;
          }
          // the minimizer slides with the k-mer: while the window holding the
          // smallest key stays inside, only the new last window is compared;
          // when it leaves, all k - m + 1 windows are scanned again
          if (have_min && min_pos > 0) {
            const uint64_t v = sub_value(g, fwd, rc, n_win - 1, g.m);
            const uint64_t key = order_key(v, g.m * g.sym_bits);
            --min_pos;
            if (key < min_key) {
              min_key = key;
              min_val = v;
              min_pos = n_win - 1;
            }
          } else {
            for (int i = 0; i < n_win; ++i) {
              const uint64_t v = sub_value(g, fwd, rc, i, g.m);
              const uint64_t key = order_key(v, g.m * g.sym_bits);
              if (i == 0 || key < min_key) {
                min_key = key;
                min_val = v;
                min_pos = i;
              }
            }
            have_min = true;
          }
          const uint64_t mu = min_val;
          const uint64_t x = shard_of(g, mu);
          if (!INSERT && stats) {
            ++n_valid;
            if (!prev_valid || mu != prev_mu) ++n_runs;
          }
          prev_valid = true;
          prev_mu = mu;
          if (!in_run || x != run_x) {   // a new run of one shard: nothing tested yet
            in_run = true;
            run_x = x;
            next_t = p;
            has_fail = false;
            if (!INSERT) {
              const ulonglong2* src = reinterpret_cast<const ulonglong2*>(g.words + x * shard_words);
              for (int w = 0; w < shard_words; w += 2) {
                const ulonglong2 v = __ldg(src + w / 2);
                sw[w * kThreads] = v.x;
                sw[(w + 1) * kThreads] = v.y;
              }
            }
          }
          const uint64_t last = p + (uint64_t)z * sb;   // the k-mer's last s-mer
          uint64_t t = next_t > p ? next_t : p;
          if (INSERT) {
            for (; t <= last; t += sb)
              set_bits(g, x * (uint64_t)g.shard_bits,
                       smer_hash(sub_value(g, fwd, rc, div_sb(t - p, sb), g.s)));
          } else {
            if (!(has_fail && last_fail >= p)) {
              for (; t <= last; t += sb) {
                if (!test_bits_shared(g, sw, smer_hash(sub_value(g, fwd, rc, div_sb(t - p, sb), g.s)))) {
                  has_fail = true;
                  last_fail = t;
                  t += sb;
                  break;
                }
              }
            }
            if (!(has_fail && last_fail >= p)) {
              word |= 1u << (uint32_t)(p - c0);
              ++cnt;
            }
          }
          next_t = t > next_t ? t : next_t;
        }
      }
      if (!INSERT) {
        if (hits && cnt) atomicAdd(&hits[r], cnt);
        n_pos += cnt;
      }
      if (re >= c1) break;
      ++r;
    }
    if (!INSERT && bits) bits[ch] = word;
  }
  if (!INSERT && stats) {
    if (n_valid) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[0]), n_valid);
    if (n_runs) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[1]), n_runs);
    if (n_pos) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[2]), n_pos);
  }
}

int rolling_grid(uint64_t seq_len) {
  const uint64_t chunks = (seq_len + kChunk - 1) / kChunk;
  uint64_t blocks = (chunks + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

cudaError_t rolling_insert(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                           uint64_t n_reads, cudaStream_t st) {
  if (seq_len == 0 || n_reads == 0) return cudaSuccess;
  rolling_kernel<true><<<rolling_grid(seq_len), kThreads, 0, st>>>(g, seq, seq_len, off, n_reads,
                                                               nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t rolling_query(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                          uint64_t n_reads, uint32_t* bits, uint32_t* hits, uint64_t* stats,
                          cudaStream_t st) {
  cudaError_t e;
  // every answer word has one owner thread that stores it; only the hit
  // counts, added per read segment, need zeroing
  if (hits && n_reads) {
    e = cudaMemsetAsync(hits, 0, n_reads * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
  }
  if (seq_len == 0) return cudaSuccess;
  rolling_kernel<false><<<rolling_grid(seq_len), kThreads, 0, st>>>(g, seq, seq_len, off, n_reads, bits,
                                                                hits, stats);
  return cudaGetLastError();
}

}  // namespace sbf
