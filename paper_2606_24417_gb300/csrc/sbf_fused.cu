// sbf_fused.cu -- dispatch of the fused kernels (sbf_fused.cuh) over the
// compiled grid: w = k-m+1 in {12 (64-bit order key), 16, 18, 20},
// H in {1, 2, 4, 8}, shard bits in {256, 512}.  Any other valid parameter
// set runs the generic kernels with identical results.
#include "sbf_fused.cuh"

#include <cstdlib>

namespace sbf {
namespace fused {
cudaError_t run_w12(const Params&, int, int, bool, cudaStream_t);
cudaError_t run_w16(const Params&, int, int, bool, cudaStream_t);
cudaError_t run_w18(const Params&, int, int, bool, cudaStream_t);
cudaError_t run_w20(const Params&, int, int, bool, cudaStream_t);

static int window_of(const Geom& g) { return g.k - g.m + 1; }

static bool key64_for(int w) { return w == 12; }

static cudaError_t run(const Params& P, bool insert, cudaStream_t st) {
  switch (window_of(P.g)) {
    case 12: return run_w12(P, P.g.H, P.g.shard_bits, insert, st);
    case 16: return run_w16(P, P.g.H, P.g.shard_bits, insert, st);
    case 18: return run_w18(P, P.g.H, P.g.shard_bits, insert, st);
    case 20: return run_w20(P, P.g.H, P.g.shard_bits, insert, st);
    default: return cudaErrorNotSupported;
  }
}

int advance_of(const Geom& g) {
  int w = window_of(g);
  return (15 + w - 1 >= 32 ? 30 : 31) * kLanePos;
}

// The single-segment launch of one call: positions [0, seq_len).
static Params single(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                     uint64_t n_reads, uint32_t* bits, uint32_t* hits, uint64_t* stats) {
  Params P{};
  P.g = g;
  P.stats = stats;
  P.segs = nullptr;
  P.n_segs = 1;
  const uint64_t adv = (uint64_t)advance_of(g);
  P.seg0 = Segment{g.words, g.n_shards, seq,  seq_len, off, n_reads, bits, hits,
                   0,       0,          (seq_len + adv - 1) / adv};
  P.iters = P.seg0.iters;
  P.work = nullptr;
  P.chunk = 1;
  P.grid_blocks = 0;
  P.big = is_big(g) ? 1u : 0u;
  return P;
}

cudaError_t launch_params(const Params& P, bool insert, cudaStream_t st) { return run(P, insert, st); }

// Hits of the reads of at most `above` positions, one thread per read: the
// set answer bits at the read's start positions [min(off[r], seq_len),
// min(off[r+1], seq_len)) -- the k-mers of read r that Alg. 2 reports present.
// The query kernel counted the longer reads itself and left these; hits were
// zeroed before it ran.  A thread reads at most above / 32 + 2 words, and the
// threads of a warp read neighbouring reads' words.
__global__ void __launch_bounds__(256) short_read_hits_kernel(const uint32_t* __restrict__ bits,
                                                              const uint64_t* __restrict__ off,
                                                              uint64_t n_reads, uint64_t seq_len,
                                                              uint32_t above,
                                                              uint32_t* __restrict__ hits) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_reads) return;
  uint64_t a = __ldg(off + r), b = __ldg(off + r + 1);
  a = a < seq_len ? a : seq_len;
  b = b < seq_len ? b : seq_len;
  if (b <= a || b - a > above) return;
  const uint64_t w0 = a >> 5, w1 = (b - 1) >> 5;
  uint32_t cnt = 0;
  for (uint64_t w = w0; w <= w1; ++w) {
    uint32_t x = __ldg(bits + w);
    if (w == w0) x &= 0xFFFFFFFFu << (uint32_t)(a & 31u);
    if (w == w1) x &= 0xFFFFFFFFu >> (31u - (uint32_t)((b - 1) & 31u));
    cnt += __popc(x);
  }
  hits[r] = cnt;
}

// The pass's blocks wait for free SMs, so paths that overlap query kernels
// on several streams (the host-input path) count every read in the kernel.
uint32_t hits_above_for(uint64_t positions, bool both_outputs) {
  if (!both_outputs) return 0u;
  uint64_t min_positions = kHitsPassMinPositions;
  const char* env = getenv("SBF_HITS_PASS_MIN_POSITIONS");
  if (env && *env) min_positions = strtoull(env, nullptr, 10);
  return positions >= min_positions ? kShortReadMax : 0u;
}

cudaError_t short_read_hits(const uint32_t* bits, const uint64_t* off, uint64_t n_reads,
                            uint64_t seq_len, uint32_t above, uint32_t* hits, cudaStream_t st) {
  if (above == 0 || n_reads == 0 || !bits || !hits) return cudaSuccess;
  const uint64_t blocks = (n_reads + 255) / 256;
  short_read_hits_kernel<<<(unsigned)blocks, 256, 0, st>>>(bits, off, n_reads, seq_len, above, hits);
  return cudaGetLastError();
}

}  // namespace fused

bool fused_supported(const Geom& g) {
  if (getenv("SBF_FORCE_GENERIC")) return false;
  if (g.alphabet != 0) return false;  // the fused staging encodes 2-bit DNA
  if (g.k < 2 || g.k > 32) return false;
  if (g.s <= 16) return false;  // the s-mer extraction shifts by 64 - 2s < 32
  int w = fused::window_of(g);
  if (w != 12 && w != 16 && w != 18 && w != 20) return false;
  if ((2 * g.m > 32) != fused::key64_for(w)) return false;
  if (g.H != 1 && g.H != 2 && g.H != 4 && g.H != 8) return false;
  // the fused address packs use min(H, W) sectors; layout 1 always has W
  if (g.layout == 1 && g.H < g.shard_bits / 64) return false;
  // 32-bit slot entries hold the shard index unless the order key is 64-bit
  if (!fused::key64_for(w) && g.n_shards > (1ull << 32)) return false;
#ifdef SBF_MINIMAL_GRID
  if (w != 16 || g.H != 4) return false;
#endif
  return g.shard_bits == 256 || g.shard_bits == 512;
}

cudaError_t fused_insert(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                         uint64_t n_reads, cudaStream_t st) {
  if (seq_len == 0 || n_reads == 0) return cudaSuccess;
  fused::Params P = fused::single(g, seq, seq_len, off, n_reads, nullptr, nullptr, nullptr);
  return fused::run(P, true, st);
}

cudaError_t fused_query(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
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
  fused::Params P = fused::single(g, seq, seq_len, off, n_reads, bits, hits, stats);
  // with both outputs, short reads' hits come from the answer words afterwards
  P.hits_above = fused::hits_above_for(seq_len, bits && hits);
  if ((e = fused::run(P, false, st)) != cudaSuccess) return e;
  return fused::short_read_hits(bits, off, n_reads, seq_len, P.hits_above, hits, st);
}

}  // namespace sbf
