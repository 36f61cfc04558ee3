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
// none (pointwise).
#include <cstdio>

#include "lmep_device.cuh"
#include "lmep_internal.h"

namespace lmep {

namespace {

struct PwParams {
  int64_t N;
  double dt, bc_lo, bc_hi;
  int n, R, tile, halo;
  int64_t ntiles;
};

template <typename ST, int NONLIN>
__device__ __forceinline__ ST nl(ST x) {
  if constexpr (NONLIN == 1) return x - x * x * x;
  else return ST(0);
}

template <typename ST, int SCHEME, int NONLIN>
__global__ void __launch_bounds__(256) k_apply_pw(PwParams a, const ST* __restrict__ u, ST* __restrict__ out,
                                                  const ST* __restrict__ W, unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  ST* su = reinterpret_cast<ST*>(smem);
  const int n = a.n, hs = (n - 1) >> 1, R = a.R;
  const int H = a.halo;
  const int Lmax = a.tile + 2 * H;
  ST* s1 = su + Lmax;   // N(u)
  ST* s2 = s1 + Lmax;   // a
  ST* s3 = s2 + Lmax;   // N(a) (ETDRK2: N(a) - N(u); ETDRK4: N(a) + N(b) later)
  ST* s4 = s3 + Lmax;   // b, then 2 N(b) - N(u)
  ST* s5 = s4 + Lmax;   // N(b)
  ST* s6 = s5 + Lmax;   // c
  ST* s7 = s6 + Lmax;   // N(c)
  const int64_t N = a.N;
  const int R4 = 2 * hs;  // reach of a one-sided window
  const ST lo_v = ST(a.bc_lo), hi_v = ST(a.bc_hi);
  const ST inv_dt = ST(1.0 / a.dt);
  unsigned bad = 0;
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t t0 = tile * int64_t(a.tile);
    const int64_t t1 = t0 + a.tile < N ? t0 + a.tile : N;
    const int L = int(t1 - t0) + 2 * H;
    const int64_t base = t0 - H;
    __syncthreads();
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
      const int64_t i = base + q;
      su[q] = (i >= 0 && i < N) ? u[i] : ST(0);
    }
    __syncthreads();
    auto inside = [&](int q) { const int64_t i = base + q; return i >= 0 && i < N; };
    auto wall = [&](int q, ST& v) {
      const int64_t i = base + q;
      if (i == 0) { v = lo_v; return true; }
      if (i == N - 1) { v = hi_v; return true; }
      return false;
    };
    // row k of point q applied to v on the point's window
    auto dot = [&](int q, int k, const ST* v) {
      const int64_t i = base + q;
      int64_t st = i - hs;
      st = st < 0 ? 0 : (st > N - n ? N - n : st);
      const int ls = int(st - base);
      const ST* w = W + (i * R + k) * n;
      ST acc = ST(0);
      for (int j = 0; j < n; ++j) acc = fma(__ldg(w + j), v[ls + j], acc);
      return acc;
    };
    auto pointwise = [&](const ST* v, ST* dst, int lo) {
      for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) dst[q] = nl<ST, NONLIN>(v[q]);
    };
    // dst = row k0 (x) + row k1 (y) on [lo, L - lo) (walls keep their values)
    auto stage = [&](int k0, const ST* x, int k1, const ST* y, ST* dst, int lo) {
      for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) {
        ST v = ST(0);
        if (inside(q) && !wall(q, v)) v = dot(q, k0, x) + dot(q, k1, y);
        dst[q] = v;
      }
    };
    auto emit = [&](int q, ST y) {
      ST wv;
      if (wall(q, wv)) y = wv;
      out[base + q] = y;
      bad |= !isfinite(y);
    };
    if (SCHEME == 0) {
      for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) emit(q, dot(q, 0, su));
      continue;
    }
    pointwise(su, s1, 0);
    __syncthreads();
    if (SCHEME == 1) {
      for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) emit(q, dot(q, 0, su) + dot(q, 1, s1));
      continue;
    }
    if (SCHEME == 2) {
      stage(0, su, 1, s1, s2, R4);                                   // a
      __syncthreads();
      for (int q = R4 + threadIdx.x; q < L - R4; q += blockDim.x) s3[q] = nl<ST, NONLIN>(s2[q]) - s1[q];
      __syncthreads();
      for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) emit(q, fma(dot(q, 2, s3), inv_dt, s2[q]));
      continue;
    }
    // ETDRK4: rows 0..3 exp(dt L), dt alpha, dt beta, dt gamma; rows 4, 5 exp(dt L/2), (dt/2) phi_1(dt L/2)
    stage(4, su, 5, s1, s2, R4);                                     // a = E2 u + P2 N(u)
    __syncthreads();
    pointwise(s2, s3, R4);                                           // N(a)
    __syncthreads();
    stage(4, su, 5, s3, s4, 2 * R4);                                 // b = E2 u + P2 N(a)
    __syncthreads();
    pointwise(s4, s5, 2 * R4);                                       // N(b)
    __syncthreads();
    for (int q = 2 * R4 + threadIdx.x; q < L - 2 * R4; q += blockDim.x) {
      s4[q] = ST(2) * s5[q] - s1[q];                                 // 2 N(b) - N(u)
      s3[q] = s3[q] + s5[q];                                         // N(a) + N(b)
    }
    __syncthreads();
    stage(4, s2, 5, s4, s6, 3 * R4);                                 // c = E2 a + P2 (2 N(b) - N(u))
    __syncthreads();
    pointwise(s6, s7, 3 * R4);                                       // N(c)
    __syncthreads();
    for (int q = H + threadIdx.x; q < L - H; q += blockDim.x)
      emit(q, dot(q, 0, su) + dot(q, 1, s1) + dot(q, 2, s3) + dot(q, 3, s7));
  }
  if (bad) atomicOr(flags, 1u);
}

template <typename ST>
const void* pw_kernel(int scheme, int nonlin) {
  if (scheme == 0) return (const void*)k_apply_pw<ST, 0, 0>;
  if (nonlin == 0) {
    if (scheme == 1) return (const void*)k_apply_pw<ST, 1, 0>;
    if (scheme == 2) return (const void*)k_apply_pw<ST, 2, 0>;
    return (const void*)k_apply_pw<ST, 3, 0>;
  }
  if (scheme == 1) return (const void*)k_apply_pw<ST, 1, 1>;
  if (scheme == 2) return (const void*)k_apply_pw<ST, 2, 1>;
  return (const void*)k_apply_pw<ST, 3, 1>;
}

}  // namespace

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
  const void* k = mixed ? pw_kernel<float>(scheme, nonlin) : pw_kernel<double>(scheme, nonlin);
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
