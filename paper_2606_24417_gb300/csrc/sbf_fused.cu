// sbf_fused.cu -- placeholder until the fused kernels land.
#include "sbf_internal.h"

namespace sbf {
bool fused_supported(const Geom&) { return false; }
cudaError_t fused_insert(const Geom&, const uint8_t*, uint64_t, const uint64_t*, uint64_t,
                         cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t fused_query(const Geom&, const uint8_t*, uint64_t, const uint64_t*, uint64_t, uint32_t*,
                        uint32_t*, uint64_t*, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace sbf
