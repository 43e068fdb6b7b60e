// sbf_noalloc.cu -- a batched query that allocates nothing.
//
// sbf_batch_query (sbf_batch.cu) keeps its segment table and work counter in
// device memory that sbf_batch_create obtains with cudaMalloc.  Some callers
// cannot do that: a process whose framework's caching allocator already
// reserved nearly all of the GPU's memory (a fresh cudaMalloc would fail or
// push the framework out of memory), or a latency-critical serving path where
// cudaMalloc's implicit device-wide synchronisation is not acceptable.  This
// entry point runs the same persistent launch with its scratch in a fixed
// array compiled into the library instead: every GPU that loads the library
// holds that array (kScratchBytes) until the process exits, and no call here
// allocates device or pinned memory.
#include <mutex>

#include "sbf_fused.cuh"

namespace {

using sbf::cuda_fail;
using sbf::fail;
using sbf::fused::Params;
using sbf::fused::Segment;

constexpr int kMaxFilters = 512;       // largest batch this entry point takes
constexpr size_t kHeaderBytes = 256;   // work counter, padded to the table's alignment
static_assert(sizeof(Segment) == 88, "documented scratch size assumes 88-byte segments");
constexpr size_t kScratchBytes = kHeaderBytes + kMaxFilters * sizeof(Segment);  // 45,312
static_assert(kScratchBytes == 45312, "documented scratch size");
// Segments per table-writing launch: they travel by value in the kernel's
// parameters (32 * 88 = 2,816 bytes, inside the classic 4 KB parameter limit).
constexpr int kParamSegments = 32;

struct SegmentChunk {
  Segment seg[kParamSegments];
};

// Copies `cnt` segments from the kernel parameters to dst[0, cnt), and zeroes
// the work counter when `work` is not NULL.  The table thus reaches the
// scratch without a host-to-device copy from pageable memory, which would
// make the host wait for earlier work on the stream.
__global__ void write_table_kernel(Segment* dst, SegmentChunk chunk, int cnt,
                                   unsigned long long* work) {
  const int words = cnt * (int)(sizeof(Segment) / 8);
  const uint64_t* src = reinterpret_cast<const uint64_t*>(chunk.seg);
  uint64_t* out = reinterpret_cast<uint64_t*>(dst);
  for (int i = threadIdx.x; i < words; i += blockDim.x) out[i] = src[i];
  if (work && threadIdx.x == 0) *work = 0ull;
}

// The scratch: a 64-bit work counter at offset 0 and the segment table at
// kHeaderBytes.  Shared by all calls on a device; each call overwrites it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol is
// only a host-side stand-in, so its address must come from
// cudaGetSymbolAddress, taken once per device with that device current.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int scratch_for_device(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SBF_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return SBF_OK;
}

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

}  // namespace

extern "C" int sbf_batch_query_noalloc(sbf_filter* const* filters, int n_filters,
                                       const uint8_t* d_seq, uint64_t seq_len,
                                       const uint64_t* d_off, const uint64_t* h_off,
                                       uint64_t n_reads, const uint64_t* h_group,
                                       uint32_t* d_kmer_bits, uint32_t* d_read_hits,
                                       sbf_stream_t stream) {
  sbf::clear_error();
  if (!filters || n_filters < 1) return fail(SBF_EINVAL, "no filters");
  if (n_filters > kMaxFilters)
    return fail(SBF_EINVAL, "%d filters: this entry point takes at most %d (its scratch is fixed)",
                n_filters, kMaxFilters);
  if (!h_off || !h_group || (n_reads && !d_off) || (seq_len && !d_seq))
    return fail(SBF_EINVAL, "NULL argument");
  const sbf_filter* f0 = filters[0];
  if (!f0) return fail(SBF_EINVAL, "filter 0 is NULL");
  for (int i = 0; i < n_filters; ++i) {
    const sbf_filter* f = filters[i];
    if (!f) return fail(SBF_EINVAL, "filter %d is NULL", i);
    if (f->geom.k != f0->geom.k || f->geom.m != f0->geom.m || f->geom.s != f0->geom.s ||
        f->geom.H != f0->geom.H || f->geom.shard_bits != f0->geom.shard_bits ||
        f->geom.canonical != f0->geom.canonical ||
        f->geom.layout != f0->geom.layout || f->device != f0->device)
      return fail(SBF_EINVAL, "filter %d differs in parameters or device", i);
    if (!f->fused) return fail(SBF_EUNSUPPORTED, "filter %d has no fused kernel", i);
  }
  if (h_off[0] != 0 || h_off[n_reads] != seq_len)
    return fail(SBF_EINVAL, "offsets must start at 0 and end at seq_len");
  if (h_group[0] != 0 || h_group[n_filters] != n_reads)
    return fail(SBF_EINVAL, "groups must start at read 0 and end at n_reads");
  for (int i = 0; i < n_filters; ++i)
    if (h_group[i + 1] < h_group[i] || h_off[h_group[i + 1]] < h_off[h_group[i]])
      return fail(SBF_EINVAL, "groups or offsets decrease at filter %d", i);

  DeviceGuard dg(f0->device);
  unsigned char* scratch = nullptr;
  int rc = scratch_for_device(f0->device, &scratch);
  if (rc != SBF_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* d_work = reinterpret_cast<unsigned long long*>(scratch);
  Segment* d_table = reinterpret_cast<Segment*>(scratch + kHeaderBytes);
  cudaError_t e;

  // Segment table, written by small kernels that carry it in their parameters
  // (kParamSegments per launch); the first launch also zeroes the work
  // counter, which keeps the last call's value otherwise.
  const uint64_t adv = (uint64_t)sbf::fused::advance_of(f0->geom);
  SegmentChunk chunk;
  uint64_t iters = 0;
  for (int c0 = 0; c0 < n_filters; c0 += kParamSegments) {
    const int cnt = n_filters - c0 < kParamSegments ? n_filters - c0 : kParamSegments;
    for (int j = 0; j < cnt; ++j) {
      const int fi = c0 + j;
      const uint64_t g0 = h_group[fi], g1 = h_group[fi + 1];
      Segment sg{};
      sg.words = filters[fi]->geom.words;
      sg.n_shards = filters[fi]->geom.n_shards;
      sg.seq = d_seq;
      sg.seq_len = seq_len;
      sg.off = d_off + g0;
      sg.n_reads = g1 - g0;
      sg.bits = d_kmer_bits;
      sg.hits = d_read_hits ? d_read_hits + g0 : nullptr;
      sg.iter_begin = iters;
      if (g1 > g0) {
        sg.p_begin = h_off[g0] & ~15ull;
        const uint64_t p_end = h_off[g1];
        sg.iters = p_end > sg.p_begin ? (p_end - sg.p_begin + adv - 1) / adv : 0;
      }
      iters += sg.iters;
      chunk.seg[j] = sg;
    }
    write_table_kernel<<<1, 128, 0, st>>>(d_table + c0, chunk, cnt, c0 == 0 ? d_work : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "segment table write");
  }
  if (d_kmer_bits && seq_len &&
      (e = cudaMemsetAsync(d_kmer_bits, 0, ((seq_len + 31) / 32) * 4, st)) != cudaSuccess)
    return cuda_fail(e, "memset");
  if (d_read_hits && n_reads && (e = cudaMemsetAsync(d_read_hits, 0, n_reads * 4, st)) != cudaSuccess)
    return cuda_fail(e, "memset");
  Params P{};
  P.g = f0->geom;
  P.stats = nullptr;
  P.segs = d_table;
  P.n_segs = (uint32_t)n_filters;
  P.iters = iters;
  P.work = d_work;
  P.chunk = 64;
  P.grid_blocks = 0;
  P.big = 0;
  for (int i = 0; i < n_filters; ++i)
    if (sbf::fused::is_big(filters[i]->geom)) P.big = 1;
  e = sbf::fused::launch_params(P, false, st);
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "batched launch");
}
