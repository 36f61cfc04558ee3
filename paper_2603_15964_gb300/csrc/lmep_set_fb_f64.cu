// lmep_set_fb_f64.cu -- the fallback kernel of the frozen-velocity sets in
// the FP64 path (finite series, then Pade scaling and squaring, for the
// points the factorised-row kernel rejected).
#include "lmep_frozen_set.cuh"

namespace lmep {
cudaError_t launch_set_fallback_f64(const FbArgs& a, unsigned grid, cudaStream_t s) {
  const size_t smem = WARPS * Ws<double>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_frozen_set_fallback<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return e;
  return launch_pdl(k_frozen_set_fallback<double>, grid, 32 * WARPS, smem, s, a);
}
}  // namespace lmep
