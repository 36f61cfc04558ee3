// lmep_apply_f64.cu -- the FP64 instantiations of the CTA-tiled apply
// (lmep_apply_tile.cuh), in a unit of their own so that they compile in
// parallel with the FP32 ones.
#include "lmep_apply_tile.cuh"

namespace lmep {
const void* apply_kernel_f64(int scheme, int nonlin, int n) { return apply_pick<double>(scheme, nonlin, n); }
}  // namespace lmep
