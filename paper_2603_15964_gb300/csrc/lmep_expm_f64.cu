// lmep_expm_f64.cu -- FP64 instantiation of the warp kernel (all products in FP64).
// Widths d <= 9 here, d >= 10 in lmep_expm_f64_hi.cu.
#include "lmep_warp_kernel.cuh"

namespace lmep {
cudaError_t warp_job_f64(int d, const WarpJob& job, cudaStream_t s) {
  return d <= 9 ? dispatch_warp_lo<double>(d, job, s) : warp_job_f64_hi(d, job, s);
}
}  // namespace lmep
