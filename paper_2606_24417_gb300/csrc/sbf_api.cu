// sbf_api.cu -- the C ABI of libsbf (declared in include/sbf.h): parameter
// validation, filter lifetime, dispatch to the fused or generic kernels, and
// the host-input path (chunked copies overlapped with kernels on two streams,
// the paper's host-facing entry points, Sec. IV-A and Sec. V-F).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "sbf_fused.cuh"
#include "sbf_internal.h"

namespace sbf {

static thread_local char g_err[512] = {0};

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SBF_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_err[0] = 0; }

int sm_count() {
  static thread_local int dev_cached = -1;
  static thread_local int count = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != dev_cached) {
    cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    if (count <= 0) count = 1;
    dev_cached = dev;
  }
  return count;
}

}  // namespace sbf

using namespace sbf;

namespace {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int check_params(int k, int m, int s, int H, uint64_t bits, int shard_bits) {
  if (k < 1 || k > 32) return fail(SBF_EINVAL, "k=%d outside [1, 32]", k);
  if (m < 1 || m > k) return fail(SBF_EINVAL, "m=%d outside [1, k=%d]", m, k);
  if (s < 1 || s > k) return fail(SBF_EINVAL, "s=%d outside [1, k=%d]", s, k);
  if (k - m + 1 > 32) return fail(SBF_EINVAL, "window k-m+1=%d exceeds 32", k - m + 1);
  if (k - s > 15) return fail(SBF_EINVAL, "k-s=%d exceeds 15", k - s);
  if (H < 1 || H > 16) return fail(SBF_EINVAL, "H=%d outside [1, 16]", H);
  if (shard_bits != 256 && shard_bits != 512)
    return fail(SBF_EINVAL, "shard_bits=%d not 256 or 512", shard_bits);
  if (bits < (uint64_t)shard_bits)
    return fail(SBF_EINVAL, "bits=%llu below one shard", (unsigned long long)bits);
  if (bits > (1ull << 46)) return fail(SBF_EINVAL, "bits=%llu above 2^46", (unsigned long long)bits);
  return SBF_OK;
}

int launch_insert(sbf_filter* f, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                  uint64_t n_reads, cudaStream_t st) {
  cudaError_t e = f->variant == 1 ? fused_insert(f->geom, seq, seq_len, off, n_reads, st)
                 : f->variant == 2 ? rolling_insert(f->geom, seq, seq_len, off, n_reads, st)
                                   : generic_insert(f->geom, seq, seq_len, off, n_reads, st);
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "insert launch");
}

int launch_query(const sbf_filter* f, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                 uint64_t n_reads, uint32_t* bits, uint32_t* hits, uint64_t* stats,
                 cudaStream_t st) {
  cudaError_t e =
      f->variant == 1 ? fused_query(f->geom, seq, seq_len, off, n_reads, bits, hits, stats, st)
      : f->variant == 2 ? rolling_query(f->geom, seq, seq_len, off, n_reads, bits, hits, stats, st)
                        : generic_query(f->geom, seq, seq_len, off, n_reads, bits, hits, stats, st);
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "query launch");
}

int check_seq_args(const void* seq, uint64_t seq_len, const void* off, uint64_t n_reads) {
  if (n_reads > 0 && !off) return fail(SBF_EINVAL, "offsets pointer is NULL");
  if (seq_len > 0 && !seq) return fail(SBF_EINVAL, "sequence pointer is NULL");
  if (seq_len >= (1ull << 62)) return fail(SBF_EINVAL, "seq_len too large");
  return SBF_OK;
}

}  // namespace

extern "C" {

const char* sbf_last_error(void) { return g_err; }

int sbf_create_full(int k, int m, int s, int H, uint64_t bits, int shard_bits, int canonical,
                    int layout, int alphabet, sbf_filter** out) {
  clear_error();
  if (!out) return fail(SBF_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_params(k, m, s, H, bits, shard_bits);
  if (rc != SBF_OK) return rc;
  if (alphabet != SBF_ALPHABET_DNA && alphabet != SBF_ALPHABET_PROTEIN &&
      alphabet != SBF_ALPHABET_DNA_TRIPLET)
    return fail(SBF_EINVAL, "alphabet must be 0, 1 or 2 (got %d)", alphabet);
  if (alphabet != SBF_ALPHABET_DNA) {
    const int sym_bits = alphabet == SBF_ALPHABET_PROTEIN ? 5 : 6;
    if (canonical) return fail(SBF_EINVAL, "canonical k-mers need the DNA alphabet");
    if (k * sym_bits > 64)
      return fail(SBF_EINVAL, "k=%d symbols of %d bits exceed 64 bits", k, sym_bits);
  }
  if (layout != SBF_LAYOUT_DEFAULT && layout != SBF_LAYOUT_PAPER)
    return fail(SBF_EINVAL, "layout must be 0 or 1 (got %d)", layout);
  if (layout == SBF_LAYOUT_PAPER && shard_bits != 256)
    return fail(SBF_EINVAL, "the paper's layout has 256-bit shards (got %d)", shard_bits);
  uint64_t n_shards = (bits + (uint64_t)shard_bits - 1) / (uint64_t)shard_bits;
  if (layout == SBF_LAYOUT_PAPER) {  // 2^P shards
    if (n_shards > (1ull << 56)) return fail(SBF_EINVAL, "filter too large");
    uint64_t p2 = 1;
    while (p2 < n_shards) p2 <<= 1;
    n_shards = p2;
  }
  uint64_t n_words = n_shards * (uint64_t)(shard_bits / 64);
  sbf_filter* f = new (std::nothrow) sbf_filter();
  if (!f) return fail(SBF_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&f->device);
  if (e != cudaSuccess) {
    delete f;
    return cuda_fail(e, "cudaGetDevice");
  }
  uint64_t* words = nullptr;
  e = cudaMalloc(&words, n_words * sizeof(uint64_t));
  if (e != cudaSuccess) {
    delete f;
    cudaGetLastError();
    return fail(SBF_ENOMEM, "cudaMalloc of %llu bytes failed: %s",
                (unsigned long long)(n_words * 8), cudaGetErrorString(e));
  }
  e = cudaMemset(words, 0, n_words * sizeof(uint64_t));
  uint32_t* status = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(uint32_t));
  if (e != cudaSuccess) {
    cudaFree(status);
    cudaFree(words);
    delete f;
    return cuda_fail(e, "filter allocation");
  }
  f->geom = make_geom(words, n_shards, k, m, s, H, shard_bits, canonical ? 1 : 0, layout, alphabet);
  f->geom.status = status;
  f->n_words = n_words;
  f->fused = fused_supported(f->geom);
  f->variant = f->fused ? 1 : getenv("SBF_FORCE_GENERIC") ? 0 : 2;
  *out = f;
  return SBF_OK;
}

int sbf_create_layout(int k, int m, int s, int H, uint64_t bits, int shard_bits, int canonical,
                      int layout, sbf_filter** out) {
  return sbf_create_full(k, m, s, H, bits, shard_bits, canonical, layout, SBF_ALPHABET_DNA, out);
}

int sbf_create_ex(int k, int m, int s, int H, uint64_t bits, int shard_bits, int canonical,
                  sbf_filter** out) {
  return sbf_create_layout(k, m, s, H, bits, shard_bits, canonical, SBF_LAYOUT_DEFAULT, out);
}

int sbf_create(int k, int m, int s, int H, uint64_t bits, sbf_filter** out) {
  return sbf_create_layout(k, m, s, H, bits, 512, 1, SBF_LAYOUT_DEFAULT, out);
}

int sbf_layout(const sbf_filter* f) { return f ? f->geom.layout : SBF_EINVAL; }

int sbf_alphabet(const sbf_filter* f) { return f ? f->geom.alphabet : SBF_EINVAL; }

void sbf_destroy(sbf_filter* f) {
  if (!f) return;
  DeviceGuard dg(f->device);
  for (int i = 0; i < 2; ++i) {
    if (f->host_streams[i]) cudaStreamDestroy(f->host_streams[i]);
    cudaFree(f->host_dev_seq[i]);
    cudaFree(f->host_dev_off[i]);
    cudaFree(f->host_dev_bits[i]);
    cudaFree(f->host_dev_hits[i]);
  }
  cudaFree(f->geom.words);
  cudaFree(f->geom.status);
  cudaFreeHost(f->host_first);
  for (int i = 0; i < 2; ++i) {
    cudaFreeHost(f->host_stage_bits[i]);
    cudaFreeHost(f->host_stage_hits[i]);
  }
  delete f;
}

int sbf_info(const sbf_filter* f, int* k, int* m, int* s, int* H, int* shard_bits, int* canonical,
             uint64_t* n_shards) {
  clear_error();
  if (!f) return fail(SBF_EINVAL, "filter is NULL");
  if (k) *k = f->geom.k;
  if (m) *m = f->geom.m;
  if (s) *s = f->geom.s;
  if (H) *H = f->geom.H;
  if (shard_bits) *shard_bits = f->geom.shard_bits;
  if (canonical) *canonical = f->geom.canonical;
  if (n_shards) *n_shards = f->geom.n_shards;
  return SBF_OK;
}

uint64_t sbf_num_words(const sbf_filter* f) { return f ? f->n_words : 0; }

int sbf_device_status(const sbf_filter* f, uint32_t* status, int clear) {
  clear_error();
  if (!f || !status) return fail(SBF_EINVAL, "NULL argument");
  DeviceGuard dg(f->device);
  cudaError_t e = cudaMemcpy(status, f->geom.status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear && *status) e = cudaMemset(f->geom.status, 0, sizeof(uint32_t));
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "device_status");
}

int sbf_kernel_variant(const sbf_filter* f) { return f ? f->variant : 0; }

const uint64_t* sbf_device_words(const sbf_filter* f) { return f ? f->geom.words : nullptr; }

int sbf_clear(sbf_filter* f, sbf_stream_t stream) {
  clear_error();
  if (!f) return fail(SBF_EINVAL, "filter is NULL");
  DeviceGuard dg(f->device);
  cudaError_t e = cudaMemsetAsync(f->geom.words, 0, f->n_words * 8, (cudaStream_t)stream);
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "clear");
}

int sbf_get_bits(const sbf_filter* f, uint64_t* h_words) {
  clear_error();
  if (!f || !h_words) return fail(SBF_EINVAL, "NULL argument");
  DeviceGuard dg(f->device);
  cudaError_t e = cudaMemcpy(h_words, f->geom.words, f->n_words * 8, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "get_bits");
}

int sbf_set_bits(sbf_filter* f, const uint64_t* h_words) {
  clear_error();
  if (!f || !h_words) return fail(SBF_EINVAL, "NULL argument");
  DeviceGuard dg(f->device);
  cudaError_t e = cudaMemcpy(f->geom.words, h_words, f->n_words * 8, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "set_bits");
}

int sbf_copy_bits_device(sbf_filter* f, uint64_t* d_words, uint64_t word_begin, uint64_t n_words,
                         int to_filter, sbf_stream_t stream) {
  clear_error();
  if (!f || (n_words && !d_words)) return fail(SBF_EINVAL, "NULL argument");
  if (word_begin > f->n_words || n_words > f->n_words - word_begin)
    return fail(SBF_EINVAL, "words [%llu, %llu) outside the filter's %llu",
                (unsigned long long)word_begin, (unsigned long long)(word_begin + n_words),
                (unsigned long long)f->n_words);
  if (n_words == 0) return SBF_OK;
  DeviceGuard dg(f->device);
  uint64_t* fw = f->geom.words + word_begin;
  cudaError_t e = to_filter
      ? cudaMemcpyAsync(fw, d_words, n_words * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream)
      : cudaMemcpyAsync(d_words, fw, n_words * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "copy_bits_device");
}

int sbf_insert_seqs(sbf_filter* f, const uint8_t* d_seq, uint64_t seq_len, const uint64_t* d_off,
                    uint64_t n_reads, sbf_stream_t stream) {
  clear_error();
  if (!f) return fail(SBF_EINVAL, "filter is NULL");
  int rc = check_seq_args(d_seq, seq_len, d_off, n_reads);
  if (rc != SBF_OK) return rc;
  DeviceGuard dg(f->device);
  return launch_insert(f, d_seq, seq_len, d_off, n_reads, (cudaStream_t)stream);
}

int sbf_query_seqs_ex(const sbf_filter* f, const uint8_t* d_seq, uint64_t seq_len,
                      const uint64_t* d_off, uint64_t n_reads, uint32_t* d_kmer_bits,
                      uint32_t* d_read_hits, uint64_t* d_stats, sbf_stream_t stream) {
  clear_error();
  if (!f) return fail(SBF_EINVAL, "filter is NULL");
  int rc = check_seq_args(d_seq, seq_len, d_off, n_reads);
  if (rc != SBF_OK) return rc;
  DeviceGuard dg(f->device);
  return launch_query(f, d_seq, seq_len, d_off, n_reads, d_kmer_bits, d_read_hits, d_stats,
                      (cudaStream_t)stream);
}

int sbf_query_seqs(const sbf_filter* f, const uint8_t* d_seq, uint64_t seq_len,
                   const uint64_t* d_off, uint64_t n_reads, uint32_t* d_kmer_bits,
                   uint32_t* d_read_hits, sbf_stream_t stream) {
  return sbf_query_seqs_ex(f, d_seq, seq_len, d_off, n_reads, d_kmer_bits, d_read_hits, nullptr,
                           stream);
}

int sbf_num_kmers(const uint64_t* h_off, uint64_t n_reads, int k, uint64_t* out) {
  clear_error();
  if (!out || (n_reads && !h_off) || k < 1) return fail(SBF_EINVAL, "bad argument");
  uint64_t total = 0;
  for (uint64_t r = 0; r < n_reads; ++r) {
    uint64_t len = h_off[r + 1] > h_off[r] ? h_off[r + 1] - h_off[r] : 0;
    if (len >= (uint64_t)k) total += len - (uint64_t)k + 1;
  }
  *out = total;
  return SBF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Host-input path.  The reads are cut into chunks at read boundaries (about
// kChunkBytes each; a read longer than that is a chunk of its own).  Chunk c
// uses buffer set c & 1 and stream c & 1, so the copy of one chunk overlaps
// the kernel of the other.
//
// Insert chunks start exactly at their first read.  Query chunks start at the
// 32-aligned position A <= off[r0] so that their output words line up with
// the caller's; the bytes [A, off[r0]) (which may hold pieces of several
// earlier reads) form a leading dummy read whose answers are masked out and
// whose hit count is dropped.  The first output word of a query chunk is
// shared with the previous chunk and is merged on the host after both finish.
// ---------------------------------------------------------------------------
namespace {

// 128 MB: smaller chunks shorten the pipeline's fill (the first upload) and
// drain (the last download), larger ones save per-chunk launches.  Measured on
// GB300 with pinned buffers (100 Mbp insert + 20M reads queried): 256 MB
// 24.6 ms, 128 MB 23.8 ms, 64 MB 24.1 ms, 32 MB 24.9 ms per step.
constexpr uint64_t kDefaultChunkBytes = 128ull << 20;

// SBF_HOST_CHUNK_BYTES overrides the chunk size (tests use small chunks to
// exercise the chunk seams).
uint64_t chunk_bytes() {
  const char* env = getenv("SBF_HOST_CHUNK_BYTES");
  if (env && *env) {
    unsigned long long v = strtoull(env, nullptr, 10);
    if (v >= 64) return v;
  }
  return kDefaultChunkBytes;
}

struct Chunk {
  uint64_t r0, r1;   // reads [r0, r1)
  uint64_t a;        // device position 0 of the chunk
  uint64_t end;      // off[r1]
};

// Chunks found by binary search over the offsets (no pass over all reads).
std::vector<Chunk> plan_chunks(const uint64_t* off, uint64_t n_reads, bool align32) {
  std::vector<Chunk> out;
  const uint64_t kChunkBytes = chunk_bytes();
  uint64_t r = 0;
  while (r < n_reads) {
    uint64_t a = align32 ? (off[r] & ~31ull) : off[r];
    // reads r .. r1-1 with off[r1] - a <= kChunkBytes, at least one read
    const uint64_t* hi = std::upper_bound(off + r + 1, off + n_reads + 1, a + kChunkBytes);
    uint64_t r1 = (uint64_t)(hi - off) - 1;
    if (r1 < r + 1) r1 = r + 1;
    out.push_back(Chunk{r, r1, a, off[r1]});
    r = r1;
  }
  return out;
}

uint32_t* ensure_first_words(sbf_filter* f, uint64_t n) {
  if (n > f->host_first_cap) {
    cudaFreeHost(f->host_first);
    f->host_first = nullptr;
    f->host_first_cap = 0;
    uint64_t cap = n < 64 ? 64 : n;
    if (cudaMallocHost(&f->host_first, cap * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    f->host_first_cap = cap;
  }
  return f->host_first;
}

int ensure_host_buffers(sbf_filter* f, uint64_t seq_cap, uint64_t reads_cap) {
  for (int i = 0; i < 2; ++i) {
    if (!f->host_streams[i]) {
      cudaError_t e = cudaStreamCreateWithFlags(&f->host_streams[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "stream create");
    }
  }
  if (seq_cap > f->host_cap_seq) {
    for (int i = 0; i < 2; ++i) {
      cudaFree(f->host_dev_seq[i]);
      cudaFree(f->host_dev_bits[i]);
      f->host_dev_seq[i] = nullptr;
      f->host_dev_bits[i] = nullptr;
      if (cudaMalloc(&f->host_dev_seq[i], seq_cap) != cudaSuccess ||
          cudaMalloc(&f->host_dev_bits[i], ((seq_cap + 31) / 32) * 4) != cudaSuccess) {
        cudaGetLastError();
        f->host_cap_seq = 0;
        return fail(SBF_ENOMEM, "device staging allocation failed");
      }
    }
    f->host_cap_seq = seq_cap;
  }
  if (reads_cap > f->host_cap_reads) {
    for (int i = 0; i < 2; ++i) {
      cudaFree(f->host_dev_off[i]);
      cudaFree(f->host_dev_hits[i]);
      f->host_dev_off[i] = nullptr;
      f->host_dev_hits[i] = nullptr;
      if (cudaMalloc(&f->host_dev_off[i], (reads_cap + 1) * 8) != cudaSuccess ||
          cudaMalloc(&f->host_dev_hits[i], reads_cap * 4) != cudaSuccess) {
        cudaGetLastError();
        f->host_cap_reads = 0;
        return fail(SBF_ENOMEM, "device staging allocation failed");
      }
    }
    f->host_cap_reads = reads_cap;
  }
  return SBF_OK;
}

// True if p is host memory the device can copy to without staging (pinned
// or registered); false for pageable memory (and NULL).
bool is_pinned(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

int ensure_stage(sbf_filter* f, uint64_t words, uint64_t reads) {
  if (words > f->host_stage_words) {
    for (int i = 0; i < 2; ++i) {
      cudaFreeHost(f->host_stage_bits[i]);
      f->host_stage_bits[i] = nullptr;
      if (cudaMallocHost(&f->host_stage_bits[i], words * 4) != cudaSuccess) {
        cudaGetLastError();
        f->host_stage_words = 0;
        return fail(SBF_ENOMEM, "pinned staging allocation failed");
      }
    }
    f->host_stage_words = words;
  }
  if (reads > f->host_stage_reads) {
    for (int i = 0; i < 2; ++i) {
      cudaFreeHost(f->host_stage_hits[i]);
      f->host_stage_hits[i] = nullptr;
      if (cudaMallocHost(&f->host_stage_hits[i], reads * 4) != cudaSuccess) {
        cudaGetLastError();
        f->host_stage_reads = 0;
        return fail(SBF_ENOMEM, "pinned staging allocation failed");
      }
    }
    f->host_stage_reads = reads;
  }
  return SBF_OK;
}

// Host path of filters with fused kernels.  A chunk's bytes are copied from
// the 32-aligned position A <= off[r0], and the kernel takes the caller's
// offsets unchanged: its sequence and answer pointers are shifted back by A
// so that absolute positions index the chunk buffers (the kernel only reads
// positions >= A).  No offset is rewritten on the host.
int host_run_fused(sbf_filter* f, bool is_query, const uint8_t* h_seq, const uint64_t* h_off,
                   uint64_t n_reads, uint32_t* h_bits, uint32_t* h_hits) {
  std::vector<Chunk> chunks = plan_chunks(h_off, n_reads, true);
  uint64_t seq_cap = 0, reads_cap = 0;
  for (const Chunk& c : chunks) {
    seq_cap = std::max(seq_cap, c.end - c.a);
    reads_cap = std::max(reads_cap, c.r1 - c.r0);
  }
  std::lock_guard<std::mutex> lock(f->host_mu);
  DeviceGuard dg(f->device);
  int rc = ensure_host_buffers(f, seq_cap, reads_cap);
  if (rc != SBF_OK) return rc;
  const uint64_t adv = (uint64_t)fused::advance_of(f->geom);
  uint32_t* first_words = ensure_first_words(f, chunks.size());
  if (!first_words) return fail(SBF_ENOMEM, "pinned host allocation failed");
  // pageable output buffers: answers go through pinned staging, copied out
  // when their buffer set is next needed (or at the end)
  const bool stage_bits = is_query && h_bits && !is_pinned(h_bits);
  const bool stage_hits = is_query && h_hits && !is_pinned(h_hits);
  if ((stage_bits || stage_hits) &&
      (rc = ensure_stage(f, stage_bits ? (seq_cap + 31) / 32 + 1 : 0, stage_hits ? reads_cap : 0)) != SBF_OK)
    return rc;
  int64_t pending[2] = {-1, -1};  // chunk whose staged answers buffer set b still holds
  auto copy_out = [&](int b) {
    if (pending[b] < 0) return;
    const Chunk& c = chunks[(size_t)pending[b]];
    const uint64_t nr = c.r1 - c.r0, nwords = (c.end - c.a + 31) / 32;
    if (stage_hits) std::memcpy(h_hits + c.r0, f->host_stage_hits[b], nr * 4);
    if (stage_bits && nwords > 1)
      std::memcpy(h_bits + c.a / 32 + 1, f->host_stage_bits[b] + 1, (nwords - 1) * 4);
    pending[b] = -1;
  };
  for (size_t ci = 0; ci < chunks.size(); ++ci) {
    const Chunk& c = chunks[ci];
    const int b = (int)(ci & 1);
    cudaStream_t st = f->host_streams[b];
    cudaError_t e = cudaStreamSynchronize(st);  // buffer set b is free again
    if (e != cudaSuccess) return cuda_fail(e, "host path sync");
    copy_out(b);
    const uint64_t len = c.end - c.a, nr = c.r1 - c.r0, nwords = (len + 31) / 32;
    if ((e = cudaMemcpyAsync(f->host_dev_seq[b], h_seq + c.a, len, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(f->host_dev_off[b], h_off + c.r0, (nr + 1) * 8, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
      return cuda_fail(e, "host path H2D");
    const bool want_bits = is_query && h_bits;
    const bool want_hits = is_query && h_hits;
    if (want_bits && (e = cudaMemsetAsync(f->host_dev_bits[b], 0, nwords * 4, st)) != cudaSuccess)
      return cuda_fail(e, "memset");
    if (want_hits && (e = cudaMemsetAsync(f->host_dev_hits[b], 0, nr * 4, st)) != cudaSuccess)
      return cuda_fail(e, "memset");
    fused::Params P{};
    P.g = f->geom;
    P.stats = nullptr;
    P.segs = nullptr;
    P.n_segs = 1;
    fused::Segment& sg = P.seg0;
    sg.words = f->geom.words;
    sg.n_shards = f->geom.n_shards;
    sg.seq = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(f->host_dev_seq[b]) - c.a);
    sg.seq_len = c.end;
    sg.off = f->host_dev_off[b];
    sg.n_reads = nr;
    sg.bits = want_bits ? reinterpret_cast<uint32_t*>(reinterpret_cast<uintptr_t>(f->host_dev_bits[b]) -
                                                       (c.a / 32) * 4)
                        : nullptr;
    sg.hits = want_hits ? f->host_dev_hits[b] : nullptr;
    sg.p_begin = c.a;
    sg.iter_begin = 0;
    sg.iters = (len + adv - 1) / adv;
    P.iters = P.seg0.iters;
    P.work = nullptr;
    P.chunk = 1;
    P.grid_blocks = 0;
    P.big = fused::is_big(f->geom) ? 1u : 0u;
    // hits of every read are counted in the kernel: a short-read pass after
    // it could not start before the other stream's query kernel (which holds
    // every SM) ended, and the chunk's copies queued behind it would stop
    // overlapping the kernels (measured: 20.6 -> 25.1 ms for 20M reads)
    P.hits_above = 0;
    if ((e = fused::launch_params(P, !is_query, st)) != cudaSuccess) return cuda_fail(e, "host path launch");
    uint32_t* hits_dst = stage_hits ? f->host_stage_hits[b] : h_hits + c.r0;
    uint32_t* bits_dst = stage_bits ? f->host_stage_bits[b] + 1 : h_bits + c.a / 32 + 1;
    if (stage_bits || stage_hits) pending[b] = (int64_t)ci;
    if (want_hits &&
        (e = cudaMemcpyAsync(hits_dst, f->host_dev_hits[b], nr * 4, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
      return cuda_fail(e, "host path D2H");
    if (want_bits) {
      if (nwords > 1 && (e = cudaMemcpyAsync(bits_dst, f->host_dev_bits[b] + 1,
                                             (nwords - 1) * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "host path D2H");
      if ((e = cudaMemcpyAsync(&first_words[ci], f->host_dev_bits[b], 4, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
        return cuda_fail(e, "host path D2H");
    }
  }
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = cudaStreamSynchronize(f->host_streams[b]);
    if (e != cudaSuccess) return cuda_fail(e, "host path sync");
    copy_out(b);
  }
  if (is_query && fused::is_big(f->geom)) {  // the bulk-copy kernels' bounded waits
    uint32_t status = 0;
    cudaError_t e = cudaMemcpy(&status, f->geom.status, sizeof(status), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (status)
      return fail(SBF_ETIMEOUT, "a shard-copy wait ran out; answers are incomplete "
                                "(sbf_device_status reports it until cleared)");
  }
  if (is_query && h_bits) {
    // word A/32 of a chunk: its bits below off[r0] belong to the previous chunk
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
      const Chunk& c = chunks[ci];
      const uint64_t lead = h_off[c.r0] - c.a;
      const uint32_t mine = first_words[ci] & (lead >= 32 ? 0u : (~0u << lead));
      const uint64_t w0 = c.a / 32;
      const uint32_t prev = (ci > 0 && chunks[ci - 1].end > c.a) ? h_bits[w0] : 0u;
      h_bits[w0] = prev | mine;
    }
  }
  return SBF_OK;
}

int host_run(sbf_filter* f, bool is_query, const uint8_t* h_seq, uint64_t seq_len,
             const uint64_t* h_off, uint64_t n_reads, uint32_t* h_bits, uint32_t* h_hits) {
  if (n_reads == 0) {
    if (h_bits && seq_len) memset(h_bits, 0, ((seq_len + 31) / 32) * 4);
    return SBF_OK;
  }
  // Offsets are not checked one by one (that would cost a pass over all reads);
  // the kernels stay in bounds for any offsets, and malformed ones only give
  // wrong answers, as on the device path.
  if (h_off[0] != 0 || h_off[n_reads] != seq_len)
    return fail(SBF_EINVAL, "offsets must start at 0 and end at seq_len");
  if (f->fused) return host_run_fused(f, is_query, h_seq, h_off, n_reads, h_bits, h_hits);
  const uint64_t dummy = is_query ? 1 : 0;  // leading dummy read of query chunks
  std::vector<Chunk> chunks = plan_chunks(h_off, n_reads, is_query);
  uint64_t seq_cap = 0, reads_cap = 0;
  for (const Chunk& c : chunks) {
    seq_cap = std::max(seq_cap, c.end - c.a);
    reads_cap = std::max(reads_cap, c.r1 - c.r0 + dummy);
  }
  std::lock_guard<std::mutex> lock(f->host_mu);
  DeviceGuard dg(f->device);
  int rc = ensure_host_buffers(f, seq_cap, reads_cap);
  if (rc != SBF_OK) return rc;
  std::vector<uint64_t> offs[2];
  uint32_t* first_words = ensure_first_words(f, chunks.size());
  if (!first_words) return fail(SBF_ENOMEM, "pinned host allocation failed");
  for (size_t ci = 0; ci < chunks.size(); ++ci) {
    const Chunk& c = chunks[ci];
    int b = (int)(ci & 1);
    cudaStream_t st = f->host_streams[b];
    // buffer set b (and offs[b]) is free once its previous chunk is done
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "host path sync");
    std::vector<uint64_t>& o = offs[b];
    uint64_t nr = c.r1 - c.r0 + dummy;
    o.resize(nr + 1);
    o[0] = 0;
    for (uint64_t r = c.r0; r <= c.r1; ++r) o[r - c.r0 + dummy] = h_off[r] - c.a;
    uint64_t len = c.end - c.a;
    if ((e = cudaMemcpyAsync(f->host_dev_seq[b], h_seq + c.a, len, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(f->host_dev_off[b], o.data(), (nr + 1) * 8, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
      return cuda_fail(e, "host path H2D");
    if (!is_query) {
      rc = launch_insert(f, f->host_dev_seq[b], len, f->host_dev_off[b], nr, st);
      if (rc != SBF_OK) return rc;
      continue;
    }
    rc = launch_query(f, f->host_dev_seq[b], len, f->host_dev_off[b], nr,
                      h_bits ? f->host_dev_bits[b] : nullptr,
                      h_hits ? f->host_dev_hits[b] : nullptr, nullptr, st);
    if (rc != SBF_OK) return rc;
    uint64_t nwords = (len + 31) / 32;
    if (h_bits) {
      uint64_t w0 = c.a / 32;
      if (nwords > 1 &&
          (e = cudaMemcpyAsync(h_bits + w0 + 1, f->host_dev_bits[b] + 1, (nwords - 1) * 4,
                               cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "host path D2H");
      if ((e = cudaMemcpyAsync(&first_words[ci], f->host_dev_bits[b], 4, cudaMemcpyDeviceToHost,
                               st)) != cudaSuccess)
        return cuda_fail(e, "host path D2H");
    }
    if (h_hits && (e = cudaMemcpyAsync(h_hits + c.r0, f->host_dev_hits[b] + 1, (nr - 1) * 4,
                                       cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "host path D2H");
  }
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = cudaStreamSynchronize(f->host_streams[b]);
    if (e != cudaSuccess) return cuda_fail(e, "host path sync");
  }
  if (is_query && h_bits) {
    // Every output word is written: words [A/32 + 1, ceil(end/32)) by the
    // chunk's copy, word A/32 here.  Its bits below off[r0] belong to the
    // previous chunk, which wrote them (and zeros above) when it ended there.
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
      const Chunk& c = chunks[ci];
      uint64_t lead = h_off[c.r0] - c.a;
      uint32_t mine = first_words[ci] & (lead >= 32 ? 0u : (~0u << lead));
      uint64_t w0 = c.a / 32;
      uint32_t prev = (ci > 0 && chunks[ci - 1].end > c.a) ? h_bits[w0] : 0u;
      h_bits[w0] = prev | mine;
    }
  }
  return SBF_OK;
}

}  // namespace

extern "C" {

int sbf_insert_seqs_host(sbf_filter* f, const uint8_t* h_seq, uint64_t seq_len,
                         const uint64_t* h_off, uint64_t n_reads) {
  clear_error();
  if (!f) return fail(SBF_EINVAL, "filter is NULL");
  int rc = check_seq_args(h_seq, seq_len, h_off, n_reads);
  if (rc != SBF_OK) return rc;
  return host_run(f, false, h_seq, seq_len, h_off, n_reads, nullptr, nullptr);
}

int sbf_query_seqs_host(const sbf_filter* f, const uint8_t* h_seq, uint64_t seq_len,
                        const uint64_t* h_off, uint64_t n_reads, uint32_t* h_kmer_bits,
                        uint32_t* h_read_hits) {
  clear_error();
  if (!f) return fail(SBF_EINVAL, "filter is NULL");
  int rc = check_seq_args(h_seq, seq_len, h_off, n_reads);
  if (rc != SBF_OK) return rc;
  // the host staging state is mutable; queries stay logically const
  return host_run(const_cast<sbf_filter*>(f), true, h_seq, seq_len, h_off, n_reads, h_kmer_bits,
                  h_read_hits);
}

}  // extern "C"
