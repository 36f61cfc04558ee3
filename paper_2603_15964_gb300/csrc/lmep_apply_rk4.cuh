// lmep_apply_rk4.cuh -- step (a6) for the ETDRK4 scheme (Sec. 3).
//
// The paper's fourth-order exponential Runge-Kutta step with localized
// weights (Sec. 3.1 step 3: every term a dot product on the point's stencil):
//   a  = E2 u + P2 N(u)                 E2, P2: rows of exp(dt L / 2) and (dt/2) phi_1(dt L / 2)
//   b  = E2 u + P2 N(a)
//   c  = E2 a + P2 (2 N(b) - N(u))
//   u+ = E u + A N(u) + B (N(a) + N(b)) + G N(c)
// with E the row of exp(dt L) and A, B, G the rows of dt alpha, dt beta,
// dt gamma (alpha = phi_1 - 3 phi_2 + 4 phi_3, beta = 2 phi_2 - 4 phi_3,
// gamma = 4 phi_3 - phi_2), all harvested once (lmep_harvest_scheme_weights).
// One CTA owns a tile of consecutive points; it stages the tile and a halo in
// shared memory with coalesced loads and evaluates the seven intermediate
// fields there on shrinking ranges, so the step reads u and writes u+ from
// HBM once (plus halo).  N: Allen-Cahn u - u^3 (pointwise), KdV -6 u u_x and
// Burgers -u u_x (u_x from the row of D^(1) of the point's window, as the
// weights).  Dirichlet walls keep their values in every stage; near a wall
// the windows are one-sided (Example 1's edge rows).
//
// Two tile bodies with the same arithmetic (every dot product summed over its
// taps in the same order, so both give the same bits):
// * interior tiles (periodic and Neumann grids; Dirichlet tiles whose halo
//   stays clear of the walls): every point takes the centre row class; the
//   rows live in registers for a stage, and each thread updates runs of RP
//   consecutive points from a window of RP + n - 1 values held in registers;
// * tiles next to a Dirichlet wall: per-point windows and row classes.
#pragma once

#include <type_traits>

#include "lmep_device.cuh"
#include "lmep_internal.h"
#include "lmep_runs.cuh"

namespace lmep {

constexpr int RK4_ROWS = 6;                       // E, A, B, G, E2, P2 per row class
constexpr int RK4_MAXW = DMAX * RK4_ROWS * DMAX;  // every row class (Dirichlet), width <= 16
constexpr int RK4_RP = RUN_RP;    // consecutive points per thread and run (interior tiles)
constexpr int RK4_PAD = RUN_PAD;  // slack after each staged field: a run's window may pass its end

struct Rk4Params {
  int64_t N;
  double h, dt, bc_lo, bc_hi;
  double inv_h;     // 1 / h, formed on the host
  int n, bc, tile, halo;
  int rs, rN;       // reach of one stencil stage and of one N(.) evaluation
  int64_t ntiles;
};

template <typename ST, int NONLIN>
__device__ __forceinline__ ST nonlin_point(ST x, ST ux, ST inv_h) {
  if constexpr (NONLIN == 1) return x - x * x * x;
  else if constexpr (NONLIN == 2) return ST(-6) * x * ux * inv_h;
  else return -x * ux * inv_h;
}

// Shared-memory fields of one tile (each Lmax + RK4_PAD elements).
template <typename ST>
struct Rk4Fields {
  ST *u, *Nu, *a, *Na, *b, *Nb, *c, *Nc;
};

// ---- tiles next to a Dirichlet wall: per-point windows and row classes.
template <typename ST, int NONLIN>
__device__ void rk4_tile_generic(const Rk4Params& a, const Rk4Fields<ST>& f, const ST* sW, const ST* sD1,
                                 int64_t base, int L, ST* __restrict__ out, unsigned& bad) {
  constexpr bool DER = NONLIN >= 2;
  const int n = a.n, hs = (n - 1) >> 1, H = a.halo;
  const bool dir = a.bc == BC_DIRICHLET;
  const int64_t N = a.N;
  const ST inv_h = ST(a.inv_h);
  const ST lo_v = ST(a.bc_lo), hi_v = ST(a.bc_hi);
  // window of local point q: local start and harvest row
  auto window = [&](int q, int& ls, int& r) {
    if (dir) {
      const int64_t i = base + q;
      int64_t st = i - hs;
      st = st < 0 ? 0 : (st > N - n ? N - n : st);
      ls = int(st - base);
      r = int(i - st);
    } else {
      ls = q - hs;
      r = hs;
    }
  };
  auto inside = [&](int q) { const int64_t i = base + q; return !dir || (i >= 0 && i < N); };
  auto wall = [&](int q, ST& v) {
    const int64_t i = base + q;
    if (!dir) return false;
    if (i == 0) { v = lo_v; return true; }
    if (i == N - 1) { v = hi_v; return true; }
    return false;
  };
  // N(v) on [lo, L - lo)
  auto eval_n = [&](const ST* v, ST* dst, int lo) {
    for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) {
      ST ux = ST(0);
      if (DER && inside(q)) {
        int ls, r;
        window(q, ls, r);
        const ST* d = sD1 + r * DMAX;
        for (int j = 0; j < n; ++j) ux = fma(d[j], v[ls + j], ux);
      }
      dst[q] = inside(q) ? nonlin_point<ST, NONLIN>(v[q], ux, inv_h) : ST(0);
    }
  };
  // dst = E2 x + P2 y on [lo, L - lo) (walls keep their values)
  auto half_stage = [&](const ST* x, const ST* y, ST* dst, int lo) {
    for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) {
      ST val = ST(0);
      if (inside(q) && !wall(q, val)) {
        int ls, r;
        window(q, ls, r);
        const ST* e2 = sW + (r * RK4_ROWS + 4) * DMAX;
        const ST* p2 = e2 + DMAX;
        ST acc = ST(0);
        for (int j = 0; j < n; ++j) acc = fma(e2[j], x[ls + j], acc);
        for (int j = 0; j < n; ++j) acc = fma(p2[j], y[ls + j], acc);
        val = acc;
      }
      dst[q] = val;
    }
  };
  const int rs = a.rs, rN = a.rN;
  int lo = rN;
  eval_n(f.u, f.Nu, lo);                   // N(u)
  __syncthreads();
  lo += rs;
  half_stage(f.u, f.Nu, f.a, lo);          // a = E2 u + P2 N(u)
  __syncthreads();
  lo += rN;
  eval_n(f.a, f.Na, lo);                   // N(a)
  __syncthreads();
  lo += rs;
  half_stage(f.u, f.Na, f.b, lo);          // b = E2 u + P2 N(a)
  __syncthreads();
  lo += rN;
  eval_n(f.b, f.Nb, lo);                   // N(b)
  __syncthreads();
  for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) {
    f.b[q] = ST(2) * f.Nb[q] - f.Nu[q];    // 2 N(b) - N(u)   (b is no longer needed)
    f.Na[q] = f.Na[q] + f.Nb[q];           // N(a) + N(b)
  }
  __syncthreads();
  lo += rs;
  half_stage(f.a, f.b, f.c, lo);           // c = E2 a + P2 (2 N(b) - N(u))
  __syncthreads();
  lo += rN;
  eval_n(f.c, f.Nc, lo);                   // N(c)
  __syncthreads();
  // u+ = E u + A N(u) + B (N(a) + N(b)) + G N(c) on [H, L - H)
  for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) {
    const int64_t i = base + q;
    ST y = ST(0);
    if (!wall(q, y)) {
      int ls, r;
      window(q, ls, r);
      const ST* e = sW + (r * RK4_ROWS) * DMAX;
      ST acc = ST(0);
      for (int j = 0; j < n; ++j) acc = fma(e[j], f.u[ls + j], acc);
      for (int j = 0; j < n; ++j) acc = fma(e[DMAX + j], f.Nu[ls + j], acc);
      for (int j = 0; j < n; ++j) acc = fma(e[2 * DMAX + j], f.Na[ls + j], acc);
      for (int j = 0; j < n; ++j) acc = fma(e[3 * DMAX + j], f.Nc[ls + j], acc);
      y = acc;
    }
    out[i] = y;
    bad |= !isfinite(y);
  }
}

// ---- interior tiles: centre rows in registers, runs of RK4_RP points.
// Thread t takes the runs starting at lo + RK4_RP (t + k blockDim.x); a run's
// points at or past `end` are computed from the field slack and not stored.
template <typename ST, int NONLIN, int NW>
__device__ __forceinline__ void rk4_eval_fast(const ST* v, ST* dst, int lo, int end, const ST* d1row, ST inv_h) {
  constexpr int HS = (NW - 1) / 2;
  if constexpr (NONLIN == 1) {
    for (int q = lo + threadIdx.x; q < end; q += blockDim.x) dst[q] = nonlin_point<ST, 1>(v[q], ST(0), inv_h);
  } else {
    ST d[NW];
    run_row<ST, NW>(d1row, d);
    for (int q0 = lo + int(threadIdx.x) * RK4_RP; q0 < end; q0 += int(blockDim.x) * RK4_RP) {
      ST x[RK4_RP + NW - 1];
      run_window<ST, NW>(v, q0 - HS, x);
      ST ux[RK4_RP];
#pragma unroll
      for (int p = 0; p < RK4_RP; ++p) ux[p] = ST(0);
      run_dot<ST, NW>(d, x, ux);
#pragma unroll
      for (int p = 0; p < RK4_RP; ++p)
        if (q0 + p < end) dst[q0 + p] = nonlin_point<ST, NONLIN>(x[p + HS], ux[p], inv_h);
    }
  }
}

// dst = E2 x + P2 y on [lo, end).
template <typename ST, int NW>
__device__ __forceinline__ void rk4_half_fast(const ST* x, const ST* y, ST* dst, int lo, int end, const ST* e2row,
                                              const ST* p2row) {
  constexpr int HS = (NW - 1) / 2;
  ST e2[NW], p2[NW];
  run_row<ST, NW>(e2row, e2);
  run_row<ST, NW>(p2row, p2);
  for (int q0 = lo + int(threadIdx.x) * RK4_RP; q0 < end; q0 += int(blockDim.x) * RK4_RP) {
    ST acc[RK4_RP];
#pragma unroll
    for (int p = 0; p < RK4_RP; ++p) acc[p] = ST(0);
    {
      ST w[RK4_RP + NW - 1];
      run_window<ST, NW>(x, q0 - HS, w);
      run_dot<ST, NW>(e2, w, acc);
    }
    {
      ST w[RK4_RP + NW - 1];
      run_window<ST, NW>(y, q0 - HS, w);
      run_dot<ST, NW>(p2, w, acc);
    }
#pragma unroll
    for (int p = 0; p < RK4_RP; ++p)
      if (q0 + p < end) dst[q0 + p] = acc[p];
  }
}

template <typename ST, int NONLIN, int NW>
__device__ void rk4_tile_fast(const Rk4Params& a, const Rk4Fields<ST>& f, const ST* sW, const ST* sD1, int64_t base,
                              int L, ST* __restrict__ out, unsigned& bad) {
  constexpr int HS = (NW - 1) / 2;
  const int H = a.halo, rs = a.rs, rN = a.rN;
  const ST inv_h = ST(a.inv_h);
  const ST* rows = sW + HS * RK4_ROWS * DMAX;  // centre class: E, A, B, G, E2, P2
  const ST* d1 = sD1 + HS * DMAX;
  int lo = rN;
  rk4_eval_fast<ST, NONLIN, NW>(f.u, f.Nu, lo, L - lo, d1, inv_h);              // N(u)
  __syncthreads();
  lo += rs;
  rk4_half_fast<ST, NW>(f.u, f.Nu, f.a, lo, L - lo, rows + 4 * DMAX, rows + 5 * DMAX);  // a
  __syncthreads();
  lo += rN;
  rk4_eval_fast<ST, NONLIN, NW>(f.a, f.Na, lo, L - lo, d1, inv_h);              // N(a)
  __syncthreads();
  lo += rs;
  rk4_half_fast<ST, NW>(f.u, f.Na, f.b, lo, L - lo, rows + 4 * DMAX, rows + 5 * DMAX);  // b
  __syncthreads();
  lo += rN;
  rk4_eval_fast<ST, NONLIN, NW>(f.b, f.Nb, lo, L - lo, d1, inv_h);              // N(b)
  __syncthreads();
  for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) {
    f.b[q] = ST(2) * f.Nb[q] - f.Nu[q];    // 2 N(b) - N(u)
    f.Na[q] = f.Na[q] + f.Nb[q];           // N(a) + N(b)
  }
  __syncthreads();
  lo += rs;
  rk4_half_fast<ST, NW>(f.a, f.b, f.c, lo, L - lo, rows + 4 * DMAX, rows + 5 * DMAX);  // c
  __syncthreads();
  lo += rN;
  rk4_eval_fast<ST, NONLIN, NW>(f.c, f.Nc, lo, L - lo, d1, inv_h);              // N(c)
  __syncthreads();
  // u+ = E u + A N(u) + B (N(a) + N(b)) + G N(c) on [H, L - H), into the free
  // field b, then copied out with coalesced stores
  {
    ST* res = f.b;
    const int end = L - H;
    for (int q0 = H + int(threadIdx.x) * RK4_RP; q0 < end; q0 += int(blockDim.x) * RK4_RP) {
      ST acc[RK4_RP];
#pragma unroll
      for (int p = 0; p < RK4_RP; ++p) acc[p] = ST(0);
      const ST* src[4] = {f.u, f.Nu, f.Na, f.Nc};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ST w[NW];
        run_row<ST, NW>(rows + k * DMAX, w);
        ST x[RK4_RP + NW - 1];
        run_window<ST, NW>(src[k], q0 - HS, x);
        run_dot<ST, NW>(w, x, acc);
      }
#pragma unroll
      for (int p = 0; p < RK4_RP; ++p)
        if (q0 + p < end) res[q0 + p] = acc[p];
    }
    __syncthreads();
    for (int q = H + threadIdx.x; q < end; q += blockDim.x) {
      const ST y = res[q];
      out[base + q] = y;
      bad |= !isfinite(y);
    }
  }
}

// NW: the stencil width n of the instance (3 .. 13).
template <typename ST, int NONLIN, int NW>
__global__ void __launch_bounds__(256) k_apply_rk4(Rk4Params a, const ST* __restrict__ u, ST* __restrict__ out,
                                                   const ST* __restrict__ W, const double* __restrict__ dh,
                                                   unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool DER = NONLIN >= 2;
  ST* sW = reinterpret_cast<ST*>(smem);
  ST* sD1 = sW + RK4_MAXW;
  const int n = NW, hs = (NW - 1) >> 1;
  const int H = a.halo;
  const int F = a.tile + 2 * H + RK4_PAD;  // elements per field
  Rk4Fields<ST> f;
  f.u = sD1 + DMAX * DMAX;
  f.Nu = f.u + F;
  f.a = f.Nu + F;
  f.Na = f.a + F;  // N(a), then N(a) + N(b)
  f.b = f.Na + F;
  f.Nb = f.b + F;
  f.c = f.Nb + F;
  f.Nc = f.c + F;
  const bool dir = a.bc == BC_DIRICHLET;
  const int64_t N = a.N;
  // the weight rows of every row class the windows use, and the rows of h D^(1)
  {
    const int r0 = dir ? 0 : hs, r1 = dir ? n : hs + 1;
    for (int e = threadIdx.x; e < (r1 - r0) * RK4_ROWS * n; e += blockDim.x) {
      const int r = r0 + e / (RK4_ROWS * n), rem = e % (RK4_ROWS * n);
      sW[(r * RK4_ROWS + rem / n) * DMAX + rem % n] = W[(r * RK4_ROWS + rem / n) * n + rem % n];
    }
    if (DER)
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) sD1[(e / n) * DMAX + e % n] = ST(dh[(e / n) * LD + e % n]);
  }
  unsigned bad = 0;
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t t0 = tile * int64_t(a.tile);
    const int64_t t1 = t0 + a.tile < N ? t0 + a.tile : N;
    const int L = int(t1 - t0) + 2 * H;
    const int64_t base = t0 - H;
    __syncthreads();  // the previous tile is done with shared memory
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
      const int64_t i = base + q;
      ST v = ST(0);
      if (!dir || (i >= 0 && i < N)) v = u[grid_index(i, N, a.bc)];
      f.u[q] = v;
    }
    __syncthreads();
    // every staged point of an interior tile has a centred window inside the
    // grid and is no wall
    const bool interior = !dir || (base - hs >= 1 && base + L + hs <= N - 2);
    if (interior) rk4_tile_fast<ST, NONLIN, NW>(a, f, sW, sD1, base, L, out, bad);
    else rk4_tile_generic<ST, NONLIN>(a, f, sW, sD1, base, L, out, bad);
  }
  if (bad) atomicOr(flags, 1u);
}

inline size_t rk4_smem(int tile, int halo, bool mixed) {
  const size_t es = mixed ? 4 : 8;
  return (size_t(RK4_MAXW) + DMAX * DMAX + 8 * (size_t(tile) + 2 * size_t(halo) + RK4_PAD)) * es;
}

// Kernel of an instance (the f64 translation unit instantiates the FP64 ones).
const void* rk4_kernel_f32(int nonlin, int n);
const void* rk4_kernel_f64(int nonlin, int n);

template <typename ST>
const void* rk4_pick(int nonlin, int n) {
  auto by_n = [&](auto tag) -> const void* {
    constexpr int NL = decltype(tag)::value;
    switch (n) {
      case 3: return (const void*)k_apply_rk4<ST, NL, 3>;
      case 5: return (const void*)k_apply_rk4<ST, NL, 5>;
      case 7: return (const void*)k_apply_rk4<ST, NL, 7>;
      case 9: return (const void*)k_apply_rk4<ST, NL, 9>;
      case 11: return (const void*)k_apply_rk4<ST, NL, 11>;
      default: return (const void*)k_apply_rk4<ST, NL, 13>;
    }
  };
  if (nonlin == 1) return by_n(std::integral_constant<int, 1>{});
  if (nonlin == 2) return by_n(std::integral_constant<int, 2>{});
  return by_n(std::integral_constant<int, 3>{});
}

}  // namespace lmep
