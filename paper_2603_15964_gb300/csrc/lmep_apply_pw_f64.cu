// lmep_apply_pw_f64.cu -- the FP64 instantiations of the stored-weight apply
// (lmep_apply_pw.cuh), in a unit of their own so that they compile in parallel
// with the FP32 ones.
#include "lmep_apply_pw.cuh"

namespace lmep {
const void* pw_kernel_f64(int scheme, int nonlin, int n) { return pw_pick<double>(scheme, nonlin, n); }
}  // namespace lmep
