// lmep_apply_rk4_f64.cu -- the FP64 instantiations of the ETDRK4 step kernels
// (lmep_apply_rk4.cuh), in a unit of their own so that they compile in parallel
// with the FP32 ones.
#include "lmep_apply_rk4.cuh"

namespace lmep {
const void* rk4_kernel_f64(int nonlin, int n) { return rk4_pick<double>(nonlin, n); }
}  // namespace lmep
