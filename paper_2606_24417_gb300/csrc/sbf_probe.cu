// sbf_probe.cu -- random-sector bandwidth probe (measurement, not a step of
// the method).
//
// A query loads one shard of B/8 bytes per super-k-mer run and an insert
// read-modify-writes one (Alg. 1/2); which shard is decided by a hash, so the
// accesses are random B/8-byte sectors.  The ceiling such accesses can reach is
// lower than a streaming copy's, so the shard part of the roofline is taken
// against this probe: random, sector-aligned loads of whole sectors (gather),
// or one 64-bit atomicOr per word of a random sector (the insert flush), over
// a caller buffer.  Sector indices come from a counter-based hash (SplitMix64
// finaliser of seed + i), so every run touches the same sectors.
#include "sbf_internal.h"

namespace {

using sbf::cuda_fail;
using sbf::fail;

__device__ __forceinline__ uint64_t probe_mix(uint64_t x) {
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return x;
}

__device__ __forceinline__ uint4 ld_nc_v4(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// LPS lanes read one sector (16 bytes each); each thread group keeps UNROLL
// sectors in flight before it consumes them.
template <int LPS>
__global__ void __launch_bounds__(256) gather_kernel(const uint4* __restrict__ buf, uint64_t n_sectors,
                                                     uint64_t n, uint64_t seed,
                                                     unsigned long long* sink) {
  constexpr int UNROLL = 4;
  const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / LPS;
  const uint64_t grp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS;
  const int part = threadIdx.x % LPS;
  uint32_t acc = 0;
  for (uint64_t i0 = grp; i0 < n; i0 += groups * UNROLL) {
    uint4 v[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const uint64_t i = i0 + (uint64_t)u * groups;
      if (i < n) {
        const uint64_t x = __umul64hi(probe_mix(seed + i), n_sectors);
        v[u] = ld_nc_v4(buf + x * LPS + part);
      } else {
        v[u] = make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
  }
  // keeps the loads live; the condition is practically never true
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

// W lanes OR one random nonzero bit into each word of a random sector.
template <int W>
__global__ void __launch_bounds__(256) rmw_kernel(unsigned long long* __restrict__ buf,
                                                  uint64_t n_sectors, uint64_t n, uint64_t seed) {
  const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / W;
  const uint64_t grp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
  const int part = threadIdx.x % W;
  for (uint64_t i = grp; i < n; i += groups) {
    const uint64_t h = probe_mix(seed + i);
    const uint64_t x = __umul64hi(h, n_sectors);
    atomicOr(buf + x * W + part, 1ull << ((h >> (6 * part)) & 63));
  }
}

}  // namespace

extern "C" int sbf_probe_sectors(void* d_buf, uint64_t buf_bytes, int sector_bytes, uint64_t n,
                                 uint64_t seed, int rmw, uint64_t* d_sink, sbf_stream_t stream) {
  sbf::clear_error();
  if (sector_bytes != 32 && sector_bytes != 64)
    return fail(SBF_EINVAL, "sector_bytes must be 32 or 64 (got %d)", sector_bytes);
  if (!d_buf || !d_sink) return fail(SBF_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(d_buf) % 64 != 0)
    return fail(SBF_EINVAL, "the buffer must be 64-byte aligned");
  const uint64_t n_sectors = buf_bytes / (uint64_t)sector_bytes;
  if (n_sectors == 0) return fail(SBF_EINVAL, "the buffer holds no sector");
  if (n == 0) return SBF_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = sbf::sm_count() * 8;  // 8 blocks of 256 threads: full occupancy
  unsigned long long* sink = reinterpret_cast<unsigned long long*>(d_sink);
  if (rmw) {
    unsigned long long* b = static_cast<unsigned long long*>(d_buf);
    if (sector_bytes == 64)
      rmw_kernel<8><<<grid, 256, 0, st>>>(b, n_sectors, n, seed);
    else
      rmw_kernel<4><<<grid, 256, 0, st>>>(b, n_sectors, n, seed);
  } else {
    const uint4* b = static_cast<const uint4*>(d_buf);
    if (sector_bytes == 64)
      gather_kernel<4><<<grid, 256, 0, st>>>(b, n_sectors, n, seed, sink);
    else
      gather_kernel<2><<<grid, 256, 0, st>>>(b, n_sectors, n, seed, sink);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SBF_OK : cuda_fail(e, "probe launch");
}
