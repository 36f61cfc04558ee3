// lmep_apply_pw.cuh -- the kernel of step (a6) with weights stored per point
// (non-uniform grids, Sec. 4.3.3); see lmep_apply_pw.cu.
#pragma once

#include "lmep_device.cuh"
#include "lmep_internal.h"

namespace lmep {

struct PwParams {
  int64_t N;
  double dt, bc_lo, bc_hi;
  double inv_dt;  // 1 / dt, formed on the host
  int n, R, tile, halo;
  int64_t ntiles;
};

template <typename ST, int NONLIN>
__device__ __forceinline__ ST pw_nl(ST x) {
  if constexpr (NONLIN == 1) return x - x * x * x;
  else return ST(0);
}

template <typename ST, int SCHEME, int NONLIN, int NW>
__global__ void __launch_bounds__(256) k_apply_pw(PwParams a, const ST* __restrict__ u, ST* __restrict__ out,
                                                  const ST* __restrict__ W, unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  ST* su = reinterpret_cast<ST*>(smem);
  constexpr int n = NW, hs = (NW - 1) >> 1;
  const int R = a.R;
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
  const ST inv_dt = ST(a.inv_dt);
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
    // row k of point q applied to v on the point's window: the n weight loads
    // are issued together, then the FMAs
    auto dot = [&](int q, int k, const ST* v) {
      const int64_t i = base + q;
      int64_t st = i - hs;
      st = st < 0 ? 0 : (st > N - n ? N - n : st);
      const int ls = int(st - base);
      const ST* w = W + (i * R + k) * n;
      ST wr[NW];
#pragma unroll
      for (int j = 0; j < NW; ++j) wr[j] = __ldg(w + j);
      ST acc = ST(0);
#pragma unroll
      for (int j = 0; j < NW; ++j) acc = fma(wr[j], v[ls + j], acc);
      return acc;
    };
    auto pointwise = [&](const ST* v, ST* dst, int lo) {
      for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) dst[q] = pw_nl<ST, NONLIN>(v[q]);
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
      for (int q = R4 + threadIdx.x; q < L - R4; q += blockDim.x) s3[q] = pw_nl<ST, NONLIN>(s2[q]) - s1[q];
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

template <typename ST, int NW>
const void* pw_kernel_n(int scheme, int nonlin) {
  if (scheme == 0) return (const void*)k_apply_pw<ST, 0, 0, NW>;
  if (nonlin == 0) {
    if (scheme == 1) return (const void*)k_apply_pw<ST, 1, 0, NW>;
    if (scheme == 2) return (const void*)k_apply_pw<ST, 2, 0, NW>;
    return (const void*)k_apply_pw<ST, 3, 0, NW>;
  }
  if (scheme == 1) return (const void*)k_apply_pw<ST, 1, 1, NW>;
  if (scheme == 2) return (const void*)k_apply_pw<ST, 2, 1, NW>;
  return (const void*)k_apply_pw<ST, 3, 1, NW>;
}

template <typename ST>
const void* pw_pick(int scheme, int nonlin, int n) {
  switch (n) {
    case 3: return pw_kernel_n<ST, 3>(scheme, nonlin);
    case 5: return pw_kernel_n<ST, 5>(scheme, nonlin);
    case 7: return pw_kernel_n<ST, 7>(scheme, nonlin);
    case 9: return pw_kernel_n<ST, 9>(scheme, nonlin);
    case 11: return pw_kernel_n<ST, 11>(scheme, nonlin);
    case 13: return pw_kernel_n<ST, 13>(scheme, nonlin);
    default: return pw_kernel_n<ST, 15>(scheme, nonlin);
  }
}

// Kernel of a launch (lmep_apply_pw.cu: FP32; lmep_apply_pw_f64.cu: FP64).
const void* pw_kernel_f32(int scheme, int nonlin, int n);
const void* pw_kernel_f64(int scheme, int nonlin, int n);


}  // namespace lmep
