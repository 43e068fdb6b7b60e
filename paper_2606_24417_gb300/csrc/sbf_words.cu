// sbf_words.cu -- bitwise OR of several word arrays on the device.
//
// A filter after inserting a set of reads is the OR of the bits each read
// sets (Alg. 1), so filters that inserted disjoint read shares combine by a
// word-wise OR.  With several processes, each owning one slice of the words
// after an all-to-all exchange, every slice is the OR of world equally long
// pieces: out[i] = in[0 * n + i] | in[1 * n + i] | ... | in[(parts-1) * n + i].
//
// The kernel is bound by HBM bandwidth: it reads parts * n words once and
// writes n words once.  Each thread handles 16-byte vectors (two words) in a
// grid-stride loop over a grid of a few blocks per SM; a ragged last word is
// handled by thread 0 of block 0.
#include "sbf_internal.h"

namespace {

__global__ void __launch_bounds__(256) or_reduce_kernel(uint64_t* __restrict__ out,
                                                        const uint64_t* __restrict__ in,
                                                        uint64_t n_words, int parts) {
  const uint64_t n_vec = n_words / 2;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_vec; v += stride) {
    ulonglong2 acc = __ldg(reinterpret_cast<const ulonglong2*>(in) + v);
    for (int j = 1; j < parts; ++j) {
      const ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2*>(in + (uint64_t)j * n_words) + v);
      acc.x |= x.x;
      acc.y |= x.y;
    }
    reinterpret_cast<ulonglong2*>(out)[v] = acc;
  }
  if ((n_words & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    uint64_t acc = 0;
    for (int j = 0; j < parts; ++j) acc |= in[(uint64_t)j * n_words + n_words - 1];
    out[n_words - 1] = acc;
  }
}

}  // namespace

extern "C" int sbf_or_reduce_device(uint64_t* d_out, const uint64_t* d_in, uint64_t n_words,
                                    int n_parts, sbf_stream_t stream) {
  sbf::clear_error();
  if (n_parts < 1) return sbf::fail(SBF_EINVAL, "n_parts must be at least 1");
  if (n_words == 0) return SBF_OK;
  if (!d_out || !d_in) return sbf::fail(SBF_EINVAL, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(d_out) | reinterpret_cast<uintptr_t>(d_in)) & 15u)
    return sbf::fail(SBF_EINVAL, "word arrays must be 16-byte aligned");
  if ((n_words & 1) && n_parts > 1)
    return sbf::fail(SBF_EINVAL, "pieces of an odd word count are not 16-byte aligned");
  const uint64_t n_vec = n_words / 2;
  uint64_t blocks = (n_vec + 255) / 256;
  const uint64_t cap = (uint64_t)sbf::sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  or_reduce_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_out, d_in, n_words,
                                                                        n_parts);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SBF_OK : sbf::cuda_fail(e, "or_reduce");
}
