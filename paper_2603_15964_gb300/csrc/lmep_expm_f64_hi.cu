// lmep_expm_f64_hi.cu -- the FP64 warp kernel for widths d >= 10 (see lmep_expm_f64.cu).
#include "lmep_warp_kernel.cuh"

namespace lmep {
cudaError_t warp_job_f64_hi(int d, const WarpJob& job, cudaStream_t s) { return dispatch_warp_hi<double>(d, job, s); }
}  // namespace lmep
