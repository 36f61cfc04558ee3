// lmep_apply.cu -- step (a6): launch of the banded application of stored
// weights: the CTA-tiled kernel (lmep_apply_tile.cuh; FP32 forms instantiated
// here, FP64 in lmep_apply_f64.cu) and the warp-streaming kernel
// (lmep_apply_stream.cu), its halo, tile and grid sizes, and the weight-pair
// tables of the streaming kernel.
#include <cstdio>
#include <type_traits>

#include "lmep_apply_tile.cuh"
#include "lmep_device.cuh"
#include "lmep_internal.h"
#include "lmep_stream.cuh"

namespace lmep {


// Halo staged on each side of a tile: the stages shrink the valid range by
// hs (a stencil) or hN (the KdV derivative).  Dirichlet adds hs so that the
// one-sided windows of points next to a wall stay inside the staged range
// even when the last tile is shorter than a stencil.
int apply_halo(int n, int scheme, int nonlin, int bc) {
  const int hs = (n - 1) / 2;
  const int hN = nonlin >= 2 ? hs : 0;
  int H = scheme == 0 ? hs : (scheme == 1 ? hs + hN : 2 * hs + 2 * hN);
  if (bc == BC_DIRICHLET) H += hs;
  return H;
}

size_t apply_smem_bytes(int tile, int halo, int scheme, bool mixed) {
  const size_t es = mixed ? 4 : 8;
  const size_t F = size_t(tile) + 2 * size_t(halo) + RUN_PAD;
  const size_t arrays = scheme == 0 ? 2 : (scheme == 1 ? 3 : 4);  // the linear scheme's result field
  return (MAXW + DMAX) * es + arrays * F * es;
}

const void* apply_kernel_f32(int scheme, int nonlin, int n) { return apply_pick<float>(scheme, nonlin, n); }

// ------------------------------------------------------------------ streaming fast path
// Geometry of the warp-streaming kernel (lmep_apply_stream.cu): a warp takes
// 128 staged points per round; for ETDRK2 the first stage runs on all 128 and
// the second updates the inner 128 - 2 hr of them.  A tile of `tile` staged
// points per round-set (tile / 128 rounds) updates fast_tile_out points.
int fast_tile_out(int tile, int n, int scheme) {
  const int hr = ((n - 1) / 2 + 3) / 4 * 4;
  const int rounds = tile / 128 > 0 ? tile / 128 : 1;
  return rounds * (scheme == 2 ? 128 - 2 * hr : 128);
}

int apply_fast_halo(int n, int scheme) {
  const int hs = (n - 1) / 2;
  const int hr = (hs + 3) / 4 * 4;
  return scheme == 2 ? 2 * hr : hr;
}

template <typename ST>
__global__ void k_pair_tables(const ST* __restrict__ W, int64_t w_stride, int wq, int n, int scheme, int64_t B,
                              int stride, ST* __restrict__ tab) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= B * stride) return;
  const int64_t b = i / stride;
  const int e = int(i % stride);
  tab[i] = pair_table_entry(W, w_stride, wq, n, scheme, b, e);
}

int pair_table_stride(int n) { return (3 * 2 * ((n + 1) / 2) * 2 + 3) / 4 * 4; }

cudaError_t launch_pair_tables(const void* W, int64_t w_stride, int wq, int n, int scheme, int64_t B, void* tab,
                               bool mixed, cudaStream_t s) {
  const int stride = pair_table_stride(n);
  const int64_t total = B * stride;
  if (total == 0) return cudaSuccess;
  const int block = 256;
  const unsigned grid = unsigned((total + block - 1) / block);
  if (mixed)
    k_pair_tables<float><<<grid, block, 0, s>>>(static_cast<const float*>(W), w_stride, wq, n, scheme, B, stride,
                                                static_cast<float*>(tab));
  else
    k_pair_tables<double><<<grid, block, 0, s>>>(static_cast<const double*>(W), w_stride, wq, n, scheme, B, stride,
                                                 static_cast<double*>(tab));
  return cudaGetLastError();
}


// The fast kernels hard-wire the Allen-Cahn nonlinearity for ETD schemes; with
// no nonlinearity every ETD step reduces to u+ = W0 u, the linear kernel (the
// weight stride wq is passed separately and keeps the stored layout).
static int fast_scheme(const ApplyParams& a) { return a.nonlin == 0 ? 0 : a.scheme; }

static const void* kernel_of(const ApplyParams& a, bool mixed) {
  if (a.fast) return stream_kernel(fast_scheme(a), a.n, mixed);
  return mixed ? apply_kernel_f32(a.scheme, a.nonlin, a.n) : apply_kernel_f64(a.scheme, a.nonlin, a.n);
}

static size_t smem_of(const ApplyParams& a, bool mixed, int block) {
  if (a.fast) return size_t(a.warp_smem) * size_t(block / 32);
  return apply_smem_bytes(a.tile, a.halo, a.scheme, mixed);
}

// Pipeline depth of the streaming kernel: 4 slots per warp, or 3 when 4 do
// not fit `block` threads' worth of warps in shared memory.
bool apply_configure(ApplyParams& a, bool mixed, int block) {
  a.stages = 0;
  a.warp_smem = 0;
  const size_t cap = size_t(device_info().smem_optin);
  if (!a.fast) return apply_smem_bytes(a.tile, a.halo, a.scheme, mixed) <= cap;
  for (int st = STREAM_MAX_STAGES; st >= 3; --st) {
    const size_t w = stream_warp_smem(a, mixed, st, fast_scheme(a));
    if (w * size_t(block / 32) <= cap) {
      a.stages = st;
      a.warp_smem = int(w);
      return true;
    }
  }
  return false;
}

int apply_grid(const ApplyParams& a, int block, int ctas_per_sm, bool mixed) {
  const void* k = kernel_of(a, mixed);
  const size_t smem = smem_of(a, mixed, block);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
  if (per_sm < 1) per_sm = 1;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  // the streaming kernel gives every warp its own tiles
  const int64_t units = a.fast ? (a.ntiles + block / 32 - 1) / (block / 32) : a.ntiles;
  return int(units < cap ? (units > 0 ? units : 1) : cap);
}

cudaError_t launch_apply(const ApplyParams& a, const void* u, void* out, const void* W, bool mixed,
                         int block, int grid, unsigned* flags, cudaStream_t s) {
  const size_t smem = smem_of(a, mixed, block);
  int wq = a.wq;
  const void* k = kernel_of(a, mixed);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  ApplyParams ap = a;
  // constants formed once here instead of in every thread (FP64 divisions are slow on this GPU)
  ap.inv_dt = 1.0 / a.dt;
  ap.inv_h = 1.0 / a.h;
  ap.dh = nullptr;
  if (!a.fast && a.nonlin >= 2) {
    const float* dhf;
    if ((e = fornberg_of(a.n, &ap.dh, &dhf)) != cudaSuccess) return e;
  }
  void* args[] = {&ap, (void*)&u, &out, (void*)&W, (void*)&wq, &flags};
  return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace lmep
