// lmep_expm_f64.cu -- FP64 instantiation of the warp kernel (all products in FP64).
#include "lmep_warp_kernel.cuh"

namespace lmep {
cudaError_t warp_job_f64(int d, const WarpJob& job, cudaStream_t s) { return dispatch_warp<double>(d, job, s); }
}  // namespace lmep
