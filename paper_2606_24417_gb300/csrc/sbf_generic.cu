// sbf_generic.cu -- generic insert/query kernels: one k-mer start position per
// thread, every step recomputed from the bases (Alg. 1 / Alg. 2 without the
// shared-memory tiling or warp cooperation).  They serve every valid
// parameter set; the fused kernels (sbf_fused.cu) take over for the compiled
// grid and give identical bits.
#include "sbf_internal.h"

namespace sbf {
namespace {

// Read holding position p: the last r in [0, n_reads) with off[r] <= p.
__device__ __forceinline__ uint64_t read_of(const uint64_t* off, uint64_t n_reads, uint64_t p) {
  uint64_t lo = 0, hi = n_reads;
  while (hi - lo > 1) {
    uint64_t mid = lo + ((hi - lo) >> 1);
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

struct KmerView {
  bool valid;
  uint64_t read;
  uint64_t fwd, rc;  // packed k-mer and its reverse complement
};

// The k-mer starting at byte p: valid iff p is a symbol start of its read
// (read start + a multiple of the symbol bytes), it ends inside the read and
// all k symbols are in the alphabet.
__device__ __forceinline__ KmerView load_kmer(const Geom& g, const uint8_t* seq, uint64_t seq_len,
                                              const uint64_t* off, uint64_t n_reads, uint64_t p) {
  KmerView v{false, 0, 0, 0};
  if (n_reads == 0) return v;
  v.read = read_of(off, n_reads, p);
  uint64_t end = off[v.read + 1];
  if (end > seq_len) end = seq_len;
  const uint64_t sb = (uint64_t)g.sym_bytes;
  if (off[v.read] > p || p + (uint64_t)g.k * sb > end) return v;
  if (sb > 1 && (p - off[v.read]) % sb != 0) return v;
  uint64_t fwd = 0, rc = 0;
  for (int i = 0; i < g.k; ++i) {
    const int c = symbol_code(g, seq + p + (uint64_t)i * sb);
    if (c < 0) return v;
    fwd = (fwd << g.sym_bits) | (uint64_t)c;
    if (g.alphabet == 0) rc |= (uint64_t)(3 - c) << (2 * i);
  }
  v.valid = true;
  v.fwd = fwd;
  v.rc = rc;
  return v;
}

__device__ __forceinline__ uint64_t canon(const Geom& g, uint64_t fwd_packed, uint64_t rc_packed,
                                          int i, int len) {
  uint64_t f = (fwd_packed >> (g.sym_bits * (g.k - len - i))) & bit_mask(g.sym_bits * len);
  if (!g.canonical) return f;
  uint64_t r = (rc_packed >> (2 * i)) & len_mask(len);
  return f < r ? f : r;
}

__device__ __forceinline__ uint64_t minimizer(const Geom& g, uint64_t fwd, uint64_t rc) {
  uint64_t best = 0, mu = 0;
  for (int i = 0; i <= g.k - g.m; ++i) {
    uint64_t v = canon(g, fwd, rc, i, g.m);
    uint64_t key = order_key(v, g.m * g.sym_bits);
    if (i == 0 || key < best) {
      best = key;
      mu = v;
    }
  }
  return mu;
}

__global__ void generic_insert_kernel(Geom g, const uint8_t* __restrict__ seq, uint64_t seq_len,
                                      const uint64_t* __restrict__ off, uint64_t n_reads) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < seq_len; p += stride) {
    KmerView v = load_kmer(g, seq, seq_len, off, n_reads, p);
    if (!v.valid) continue;
    uint64_t x = shard_of(g, minimizer(g, v.fwd, v.rc));
    uint64_t base = x * (uint64_t)g.shard_bits;
    for (int t = 0; t <= g.k - g.s; ++t) {
      uint64_t h = smer_hash(canon(g, v.fwd, v.rc, t, g.s));
      for (int i = 0; i < g.H; ++i) {
        uint64_t bit = base + bit_in_shard(g, h, i);
        atomicOr((unsigned long long*)&g.words[bit >> 6], 1ull << (bit & 63));
      }
    }
  }
}

__global__ void generic_query_kernel(Geom g, const uint8_t* __restrict__ seq, uint64_t seq_len,
                                     const uint64_t* __restrict__ off, uint64_t n_reads,
                                     uint32_t* __restrict__ bits, uint32_t* __restrict__ hits,
                                     uint64_t* __restrict__ stats) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long n_valid = 0, n_runs = 0, n_pos = 0;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < seq_len; p += stride) {
    KmerView v = load_kmer(g, seq, seq_len, off, n_reads, p);
    if (!v.valid) continue;
    uint64_t mu = minimizer(g, v.fwd, v.rc);
    uint64_t x = shard_of(g, mu);
    uint64_t base = x * (uint64_t)g.shard_bits;
    bool present = true;
    for (int t = 0; t <= g.k - g.s && present; ++t) {
      uint64_t h = smer_hash(canon(g, v.fwd, v.rc, t, g.s));
      for (int i = 0; i < g.H; ++i) {
        uint64_t bit = base + bit_in_shard(g, h, i);
        if (!((g.words[bit >> 6] >> (bit & 63)) & 1ull)) {
          present = false;
          break;
        }
      }
    }
    if (present) {
      if (bits) atomicOr(&bits[p >> 5], 1u << (p & 31));
      if (hits) atomicAdd(&hits[v.read], 1u);
    }
    if (stats) {
      ++n_valid;
      n_pos += present ? 1 : 0;
      bool head = true;
      if (p >= (uint64_t)g.sym_bytes) {
        KmerView u = load_kmer(g, seq, seq_len, off, n_reads, p - (uint64_t)g.sym_bytes);
        if (u.valid && u.read == v.read && minimizer(g, u.fwd, u.rc) == mu) head = false;
      }
      n_runs += head ? 1 : 0;
    }
  }
  if (stats) {
    if (n_valid) atomicAdd((unsigned long long*)&stats[0], n_valid);
    if (n_runs) atomicAdd((unsigned long long*)&stats[1], n_runs);
    if (n_pos) atomicAdd((unsigned long long*)&stats[2], n_pos);
  }
}

int grid_for(uint64_t work, int threads) {
  uint64_t blocks = (work + threads - 1) / threads;
  uint64_t cap = (uint64_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

cudaError_t generic_insert(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                           uint64_t n_reads, cudaStream_t st) {
  if (seq_len == 0 || n_reads == 0) return cudaSuccess;
  generic_insert_kernel<<<grid_for(seq_len, 256), 256, 0, st>>>(g, seq, seq_len, off, n_reads);
  return cudaGetLastError();
}

cudaError_t generic_query(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                          uint64_t n_reads, uint32_t* bits, uint32_t* hits, uint64_t* stats,
                          cudaStream_t st) {
  cudaError_t e;
  if (bits && seq_len) {
    e = cudaMemsetAsync(bits, 0, ((seq_len + 31) / 32) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
  }
  if (hits && n_reads) {
    e = cudaMemsetAsync(hits, 0, n_reads * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
  }
  if (seq_len == 0 || n_reads == 0) return cudaSuccess;
  generic_query_kernel<<<grid_for(seq_len, 256), 256, 0, st>>>(g, seq, seq_len, off, n_reads, bits,
                                                              hits, stats);
  return cudaGetLastError();
}

}  // namespace sbf
