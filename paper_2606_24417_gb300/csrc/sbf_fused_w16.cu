// sbf_fused_w16.cu -- fused kernels for minimizer window w = k - m + 1 = 16.
#include "sbf_fused.cuh"

namespace sbf {
namespace fused {

template <bool INSERT, bool BULK>
static cudaError_t run(const Params& P, int H, int B, cudaStream_t st) {
#ifdef SBF_MINIMAL_GRID
  if (H == 4 && B == 512) return launch<16, 4, 512, false, INSERT, BULK>(P, st);
  if (H == 4 && B == 256) return launch<16, 4, 256, false, INSERT, BULK>(P, st);
#else
  switch (H * 1000 + B) {
    case 1256: return launch<16, 1, 256, false, INSERT, BULK>(P, st);
    case 1512: return launch<16, 1, 512, false, INSERT, BULK>(P, st);
    case 2256: return launch<16, 2, 256, false, INSERT, BULK>(P, st);
    case 2512: return launch<16, 2, 512, false, INSERT, BULK>(P, st);
    case 4256: return launch<16, 4, 256, false, INSERT, BULK>(P, st);
    case 4512: return launch<16, 4, 512, false, INSERT, BULK>(P, st);
    case 8256: return launch<16, 8, 256, false, INSERT, BULK>(P, st);
    case 8512: return launch<16, 8, 512, false, INSERT, BULK>(P, st);
    default: break;
  }
#endif
  return cudaErrorNotSupported;
}

cudaError_t run_w16(const Params& P, int H, int B, bool insert, cudaStream_t st) {
  if (insert) return run<true, false>(P, H, B, st);
  return P.big ? run<false, true>(P, H, B, st) : run<false, false>(P, H, B, st);
}

}  // namespace fused
}  // namespace sbf
