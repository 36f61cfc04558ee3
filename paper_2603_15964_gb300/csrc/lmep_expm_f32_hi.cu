// lmep_expm_f32_hi.cu -- the FP32-form warp kernel for widths d >= 10 (see lmep_expm_f32.cu).
#include "lmep_warp_kernel.cuh"

namespace lmep {
cudaError_t warp_job_f32_hi(int d, const WarpJob& job, cudaStream_t s) { return dispatch_warp_hi<float>(d, job, s); }
}  // namespace lmep
