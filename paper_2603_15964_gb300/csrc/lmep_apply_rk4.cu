// lmep_apply_rk4.cu -- launch of the ETDRK4 step (kernels in
// lmep_apply_rk4.cuh; this unit instantiates the FP32 form, lmep_apply_rk4_f64.cu
// the FP64 one).
#include <cstdio>

#include "lmep_apply_rk4.cuh"

namespace lmep {

const void* rk4_kernel_f32(int nonlin, int n) { return rk4_pick<float>(nonlin, n); }

int rk4_halo(int n, int nonlin, int bc) {
  const int hs = (n - 1) / 2;
  const int rs = bc == BC_DIRICHLET ? 2 * hs : hs;  // one-sided windows reach n - 1 next to a wall
  const int rN = nonlin >= 2 ? rs : 0;
  return 4 * rs + 4 * rN;
}

cudaError_t launch_apply_rk4(int64_t N, double h, int bc, int n, int nonlin, double dt, double bc_lo, double bc_hi,
                             const void* u, void* out, const void* W, bool mixed, unsigned* flags, cudaStream_t s) {
  Rk4Params a{};
  a.N = N;
  a.h = h;
  a.inv_h = 1.0 / h;
  a.dt = dt;
  a.bc_lo = bc_lo;
  a.bc_hi = bc_hi;
  a.n = n;
  a.bc = bc;
  a.halo = rk4_halo(n, nonlin, bc);
  const int hs = (n - 1) / 2;
  a.rs = bc == BC_DIRICHLET ? 2 * hs : hs;
  a.rN = nonlin >= 2 ? a.rs : 0;
  const size_t cap = size_t(device_info().smem_optin);
  int tile = mixed ? 2048 : 1024;
  while (tile > 64 && rk4_smem(tile, a.halo, mixed) > cap) tile /= 2;
  a.tile = tile;
  a.ntiles = (N + tile - 1) / tile;
  const size_t smem = rk4_smem(tile, a.halo, mixed);
  const void* k = mixed ? rk4_kernel_f32(nonlin, n) : rk4_kernel_f64(nonlin, n);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t cap_ctas = int64_t(device_info().sms) * per_sm;
  const int grid = int(a.ntiles < cap_ctas ? a.ntiles : cap_ctas);
  const double* dh;
  const float* dhf;
  if ((e = fornberg_of(n, &dh, &dhf)) != cudaSuccess) return e;
  void* args[] = {&a, (void*)&u, &out, (void*)&W, (void*)&dh, &flags};
  return cudaLaunchKernel(k, dim3(grid), dim3(256), args, smem, s);
}

}  // namespace lmep
