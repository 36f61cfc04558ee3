// lmep_expm_f32.cu -- FP32-form instantiation of the warp kernel: Pade
// products in FP32 with FP32 accumulation, denominator solve and squaring
// phase in FP64, state and weights stored as float.
// Widths d <= 9 here, d >= 10 in lmep_expm_f32_hi.cu.
#include "lmep_warp_kernel.cuh"

namespace lmep {
cudaError_t warp_job_f32(int d, const WarpJob& job, cudaStream_t s) {
  return d <= 9 ? dispatch_warp_lo<float>(d, job, s) : warp_job_f32_hi(d, job, s);
}
}  // namespace lmep
