// lmep_apply_pw.cu -- step (a6) with weights stored per point (non-uniform
// grids, Sec. 4.3.3).
//
// On a non-uniform grid every node has its own harvested rows, computed once
// (lmep_harvest_nodes) and stored as W[N][R][n]; a step is then a banded
// product with those rows (Sec. 3.1 step 3).  Windows are those of the
// harvest: start_i = clamp(i - (n-1)/2, 0, N - n), the walls keep their
// values.  One CTA owns a tile of consecutive points; the state and the
// intermediate fields of the scheme live in shared memory (tile plus a halo of
// one window reach, n - 1, per stencil stage); each point reads its own weight
// rows from HBM once per stage that needs them, so a step moves R n values of
// weights and two of state per point: the apply is bound by the weights'
// bandwidth.  Schemes: linear, ETD1, ETDRK2 and ETDRK4 with N(u) = u - u^3 or
// none (pointwise).  The kernel is compiled per stencil width, so a point's n
// weight loads of a row are issued together before its FMAs (many loads in
// flight per thread, which the weight bandwidth needs).  This unit holds the
// launch and the FP32 kernels; lmep_apply_pw_f64.cu the FP64 ones.
#include <cstdio>

#include "lmep_apply_pw.cuh"

namespace lmep {

const void* pw_kernel_f32(int scheme, int nonlin, int n) { return pw_pick<float>(scheme, nonlin, n); }

int pw_rows(int scheme) { return scheme == 3 ? 6 : scheme + 1; }

int pw_halo(int n, int scheme) {
  const int reach = n - 1;  // one-sided windows next to a wall
  return scheme == 3 ? 4 * reach : (scheme == 2 ? 2 * reach : reach);
}

cudaError_t launch_apply_pw(int64_t N, int n, int scheme, int nonlin, double dt, double bc_lo, double bc_hi,
                            const void* u, void* out, const void* W, bool mixed, unsigned* flags, cudaStream_t s) {
  PwParams a{};
  a.N = N;
  a.dt = dt;
  a.inv_dt = 1.0 / dt;
  a.bc_lo = bc_lo;
  a.bc_hi = bc_hi;
  a.n = n;
  a.R = pw_rows(scheme);
  a.halo = pw_halo(n, scheme);
  const size_t es = mixed ? 4 : 8;
  const int arrays = scheme == 0 ? 1 : (scheme == 1 ? 2 : (scheme == 2 ? 4 : 8));
  a.tile = 1024;
  a.ntiles = (N + a.tile - 1) / a.tile;
  const size_t smem = size_t(arrays) * size_t(a.tile + 2 * a.halo) * es;
  const void* k = mixed ? pw_kernel_f32(scheme, nonlin, n) : pw_kernel_f64(scheme, nonlin, n);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  const int grid = int(a.ntiles < cap ? a.ntiles : cap);
  void* args[] = {&a, (void*)&u, &out, (void*)&W, &flags};
  return cudaLaunchKernel(k, dim3(grid), dim3(256), args, smem, s);
}

}  // namespace lmep
