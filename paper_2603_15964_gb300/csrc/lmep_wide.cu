// lmep_wide.cu -- wide stencils (n = 17 .. 25, odd) of the constant-coefficient
// linear scheme: the harvest of their rows and their banded apply on periodic
// grids, with any fixed window shift (the one-sided stencils of Sec. 4.1).
//
// One warp holds at most a 16 x 16 local matrix (lmep_device.cuh), so these
// widths do not go through the Pade kernels.  Their rows come instead from the
// factorised form of the local exponential (Thm. 1 with the General Exactness
// theorem): on the window's polynomial space the derivative matrices are
// powers of one nilpotent matrix, Dh2 = Dh1^2 and Dh3 = Dh1^3, so with
// X = c0 dt I + a Dh1 + E (a = c1 dt / h, E = c2h Dh2 + c3h Dh3)
//
//   row r of exp(X) = e^{c0 dt} l(r + a)^T exp(E),
//
// l(z) the Lagrange weights of the window's nodes at the departure point z,
// and exp(E) the finite Taylor sum of the nilpotent E (E^n = 0).  For pure
// advection E = 0 and the row is the semi-Lagrangian interpolant itself.
// Everything is formed in FP64 and the rows are stored in the state type.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "lmep_internal.h"
#include "lmep_runs.cuh"

namespace lmep {

namespace {

constexpr int WMAX = 25;  // widest stencil of this path

// Dh1 on the nodes 0 .. n-1, from the barycentric form of the interpolant's
// derivative: for i != j, Dh1[i][j] = (b_j / b_i) / (i - j) with b_j =
// (-1)^j C(n-1, j) (equispaced barycentric weights, common factor dropped);
// the diagonal makes every row sum to zero (derivatives of constants vanish).
__device__ void wide_d1(int n, double* D1, int lane) {
  for (int i = lane; i < n; i += 32) {
    double bi = 1.0;  // C(n-1, i), exact for n <= 25
    for (int k = 1; k <= i; ++k) bi = bi * double(n - k) / double(k);
    if (i & 1) bi = -bi;
    double diag = 0.0;
    double bj = 1.0;
    for (int j = 0; j < n; ++j) {
      if (j > 0) bj = bj * double(n - j) / double(j);
      const double b = (j & 1) ? -bj : bj;
      double d = 0.0;
      if (j != i) {
        d = (b / bi) / double(i - j);
        diag -= d;
      }
      D1[i * WMAX + j] = d;
    }
    D1[i * WMAX + i] = diag;
  }
}

// C = A B for n x n matrices of stride WMAX in shared memory.
__device__ void wide_matmul(int n, const double* A, const double* B, double* C, int lane) {
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = fma(A[i * WMAX + k], B[k * WMAX + j], s);
    C[i * WMAX + j] = s;
  }
}

// Rows of every row class r (blockIdx.x) of a constant-coefficient problem:
// W[r][0][j], the layout of the harvest of n_phi = 0.
template <typename OT>
__global__ void __launch_bounds__(32) k_harvest_wide(int n, double a, double c2h, double c3h, double c0dt,
                                                     OT* __restrict__ W) {
  __shared__ double D1[WMAX * WMAX], D2[WMAX * WMAX], E[WMAX * WMAX];
  __shared__ double v[WMAX], s[WMAX], t[WMAX];
  const int lane = threadIdx.x, r = blockIdx.x;
  const bool has_e = c2h != 0.0 || c3h != 0.0;
  if (has_e) {
    wide_d1(n, D1, lane);
    __syncwarp();
    wide_matmul(n, D1, D1, D2, lane);  // Dh2 = Dh1^2
    __syncwarp();
    wide_matmul(n, D2, D1, E, lane);   // Dh3 = Dh1^3, held in E for a moment
    __syncwarp();
    for (int e = lane; e < n * n; e += 32) {
      const int i = e / n, j = e % n;
      E[i * WMAX + j] = fma(c2h, D2[i * WMAX + j], c3h * E[i * WMAX + j]);
    }
    __syncwarp();
  }
  // Lagrange weights at the departure point z = r + a
  const double z = double(r) + a;
  for (int j = lane; j < n; j += 32) {
    double num = 1.0, den = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) {
        num *= z - double(k);
        den *= double(j - k);
      }
    v[j] = num / den;
    s[j] = v[j];
  }
  __syncwarp();
  // l^T exp(E): the finite Taylor sum, term_{k} = term_{k-1} E / k
  if (has_e)
    for (int k = 1; k < n; ++k) {
      for (int j = lane; j < n; j += 32) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc = fma(v[i], E[i * WMAX + j], acc);
        t[j] = acc / double(k);
      }
      __syncwarp();
      for (int j = lane; j < n; j += 32) {
        v[j] = t[j];
        s[j] += t[j];
      }
      __syncwarp();
    }
  const double g = exp(c0dt);
  for (int j = lane; j < n; j += 32) W[int64_t(r) * n + j] = OT(g * s[j]);
}

// One step of the linear scheme on a periodic grid: u+_i = sum_j w_j u_{i - WS + j},
// WS = (NW - 1) / 2 + shift.  A CTA stages a tile and its halo of H = (NW - 1) / 2
// + |shift| points; each thread updates runs of RUN_RP consecutive points from a
// register window, the row held in registers; results leave through a shared
// field in coalesced stores.
template <typename ST, int NW>
__global__ void __launch_bounds__(256) k_apply_wide(int64_t N, int shift, int tile, const ST* __restrict__ w,
                                                    const ST* __restrict__ u, ST* __restrict__ out,
                                                    unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int HS = (NW - 1) / 2;
  const int WS = HS + shift;
  const int H = HS + (shift < 0 ? -shift : shift);
  const int F = tile + 2 * H + RUN_RP + NW;  // staged field with the runs' slack
  ST* su = reinterpret_cast<ST*>(smem);
  ST* res = su + F;
  ST row[NW];
  run_row<ST, NW>(w, row);
  unsigned bad = 0;
  const int64_t ntiles = (N + tile - 1) / tile;
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t t0 = tl * tile;
    const int len = int(N - t0 < tile ? N - t0 : tile);
    __syncthreads();  // the previous tile is done with both fields
    for (int q = threadIdx.x; q < len + 2 * H; q += blockDim.x) {
      int64_t i = (t0 - H + q) % N;
      if (i < 0) i += N;
      su[q] = u[i];
    }
    __syncthreads();
    for (int q0 = int(threadIdx.x) * RUN_RP; q0 < len; q0 += int(blockDim.x) * RUN_RP) {
      ST x[RUN_RP + NW - 1], acc[RUN_RP];
      run_window<ST, NW>(su, q0 + H - WS, x);
#pragma unroll
      for (int p = 0; p < RUN_RP; ++p) acc[p] = ST(0);
      run_dot<ST, NW>(row, x, acc);
#pragma unroll
      for (int p = 0; p < RUN_RP; ++p)
        if (q0 + p < len) res[q0 + p] = acc[p];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < len; q += blockDim.x) {
      const ST y = res[q];
      out[t0 + q] = y;
      bad |= !isfinite(y);
    }
  }
  if (bad) atomicOr(flags, 1u);
}

template <typename ST>
const void* wide_kernel(int n) {
  switch (n) {
    case 17: return (const void*)k_apply_wide<ST, 17>;
    case 19: return (const void*)k_apply_wide<ST, 19>;
    case 21: return (const void*)k_apply_wide<ST, 21>;
    case 23: return (const void*)k_apply_wide<ST, 23>;
    default: return (const void*)k_apply_wide<ST, 25>;
  }
}

}  // namespace

bool wide_width(int n) { return n >= 17 && n <= WMAX && (n & 1); }

cudaError_t launch_harvest_wide(const KParams& p, void* W, bool mixed, cudaStream_t s) {
  const double a = p.c1 * p.dt_h;
  if (mixed)
    k_harvest_wide<float><<<unsigned(p.n), 32, 0, s>>>(p.n, a, p.c2h, p.c3h, p.c0dt, static_cast<float*>(W));
  else
    k_harvest_wide<double><<<unsigned(p.n), 32, 0, s>>>(p.n, a, p.c2h, p.c3h, p.c0dt, static_cast<double*>(W));
  return cudaGetLastError();
}

cudaError_t launch_apply_wide(int64_t N, int n, int shift, const void* W, const void* u, void* out, bool mixed,
                              unsigned* flags, cudaStream_t s) {
  const int es = mixed ? 4 : 8;
  const int tile = mixed ? 2048 : 1024;
  const int H = (n - 1) / 2 + (shift < 0 ? -shift : shift);
  const size_t smem = size_t(2 * tile + 2 * H + RUN_RP + n) * es;
  const void* k = mixed ? wide_kernel<float>(n) : wide_kernel<double>(n);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (N + tile - 1) / tile;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  const unsigned grid = unsigned(ntiles < cap ? ntiles : cap);
  // the row of the class every point of a periodic grid takes: WS = (n - 1) / 2 + shift
  const int WS = (n - 1) / 2 + shift;
  if (mixed) {
    const float* w = static_cast<const float*>(W) + int64_t(WS) * n;
    void* args[] = {&N, &shift, const_cast<int*>(&tile), &w, const_cast<void**>(&u), &out, &flags};
    return cudaLaunchKernel(k, dim3(grid), dim3(256), args, smem, s);
  }
  const double* w = static_cast<const double*>(W) + int64_t(WS) * n;
  void* args[] = {&N, &shift, const_cast<int*>(&tile), &w, const_cast<void**>(&u), &out, &flags};
  return cudaLaunchKernel(k, dim3(grid), dim3(256), args, smem, s);
}

}  // namespace lmep
