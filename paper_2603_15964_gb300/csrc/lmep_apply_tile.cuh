// lmep_apply_tile.cuh -- the CTA-tiled kernel of step (a6): banded application
// of stored weights (lmep_apply.cu launches it; lmep_apply_f64.cu instantiates
// the FP64 forms).
//
// Sec. 3.1 step 3: every ETD term is a dot product of a harvested row with
// the state (or the nonlinear term) on the point's stencil.  One CTA owns a
// tile of consecutive points of one instance.  It stages the tile plus a halo
// in shared memory with coalesced loads, evaluates N(u), the first stage a
// and, for ETDRK2, N(a) on the shrinking halo ranges, and writes u+ once:
// the whole step reads u and writes u+ from HBM exactly once (plus halo).
//
// Stencil handling: periodic windows wrap, Neumann windows reflect about the
// wall node, Dirichlet windows slide inside the domain (edge rows) and the
// wall values are never updated.  Two tile bodies with the same arithmetic
// (every dot product summed over its taps in the same order):
// * interior tiles (periodic and Neumann grids; Dirichlet tiles whose halo
//   stays clear of the walls): one row class, its rows in registers, runs of
//   RUN_RP consecutive points per thread (lmep_runs.cuh), results through a
//   free field and out in coalesced stores;
// * tiles next to a Dirichlet wall: per-point windows and row classes.
#pragma once

#include "lmep_device.cuh"
#include "lmep_internal.h"
#include "lmep_runs.cuh"

namespace lmep {

constexpr int MAXW = DMAX * 3 * DMAX;  // n * (1 + n_phi) * n, n <= 15, n_phi <= 2

template <typename ST>
struct TileFields {
  ST *u, *N, *a, *Na;  // state, N(u), first stage, N(a) - N(u); each Lmax + RUN_PAD elements
};

// N(v) of the state's points on [lo, end) (v staged, window of point q at q - hs).
template <typename ST, int NONLIN, int NW>
__device__ __forceinline__ void tile_nonlin_runs(const ST* v, ST* dst, const ST* sub, int lo, int end,
                                                 const ST* d1, ST ncoef, ST inv_h) {
  constexpr int HS = (NW - 1) / 2;
  if constexpr (NONLIN >= 2) {
    ST d[NW];
    run_row<ST, NW>(d1, d);
    for (int q0 = lo + int(threadIdx.x) * RUN_RP; q0 < end; q0 += int(blockDim.x) * RUN_RP) {
      ST x[RUN_RP + NW - 1];
      run_window<ST, NW>(v, q0 - HS, x);
      ST ux[RUN_RP];
#pragma unroll
      for (int p = 0; p < RUN_RP; ++p) ux[p] = ST(0);
      run_dot<ST, NW>(d, x, ux);
#pragma unroll
      for (int p = 0; p < RUN_RP; ++p)
        if (q0 + p < end) {
          const ST f = ncoef * x[p + HS] * ux[p] * inv_h;
          dst[q0 + p] = sub ? f - sub[q0 + p] : f;
        }
    }
  } else {
    for (int q = lo + threadIdx.x; q < end; q += blockDim.x) {
      const ST x = v[q];
      const ST f = x - x * x * x;
      dst[q] = sub ? f - sub[q] : f;
    }
  }
}

// Interior tile: the same stages and ranges as the per-point body below.
template <typename ST, int SCHEME, int NONLIN, int NW>
__device__ void tile_interior(const ApplyParams& a, const TileFields<ST>& f, const ST* sW, const ST* sd1, int L,
                              int64_t gbase, ST ncoef, ST inv_h, ST inv_dt, ST* __restrict__ out, unsigned& bad) {
  constexpr bool KDV = NONLIN >= 2;
  constexpr int HS = (NW - 1) / 2;
  const int hN = KDV ? HS : 0;
  const int H = a.halo;
  const int WS = HS + a.shift;           // window start of point q: q - WS (shift only with the linear scheme)
  const ST* rows = sW + (WS * 3) * DMAX; // the row class of every point: W0, W1, W2
  ST* res = f.N;                         // free when the result is formed
  if constexpr (SCHEME == 0) {
    ST w0[NW];
    run_row<ST, NW>(rows, w0);
    for (int q0 = H + int(threadIdx.x) * RUN_RP; q0 < L - H; q0 += int(blockDim.x) * RUN_RP) {
      ST x[RUN_RP + NW - 1], acc[RUN_RP];
      run_window<ST, NW>(f.u, q0 - WS, x);
#pragma unroll
      for (int p = 0; p < RUN_RP; ++p) acc[p] = ST(0);
      run_dot<ST, NW>(w0, x, acc);
#pragma unroll
      for (int p = 0; p < RUN_RP; ++p)
        if (q0 + p < L - H) res[q0 + p] = acc[p];
    }
  } else {
    tile_nonlin_runs<ST, NONLIN, NW>(f.u, f.N, nullptr, hN, L - hN, sd1, ncoef, inv_h);  // N(u)
    __syncthreads();
    {  // a = W0 u + W1 N(u) on [hs + hN, L - hs - hN)
      ST w0[NW], w1[NW];
      run_row<ST, NW>(rows, w0);
      run_row<ST, NW>(rows + DMAX, w1);
      const int end = L - HS - hN;
      for (int q0 = HS + hN + int(threadIdx.x) * RUN_RP; q0 < end; q0 += int(blockDim.x) * RUN_RP) {
        ST acc[RUN_RP];
#pragma unroll
        for (int p = 0; p < RUN_RP; ++p) acc[p] = ST(0);
        {
          ST x[RUN_RP + NW - 1];
          run_window<ST, NW>(f.u, q0 - WS, x);
          run_dot<ST, NW>(w0, x, acc);
        }
        {
          ST x[RUN_RP + NW - 1];
          run_window<ST, NW>(f.N, q0 - WS, x);
          run_dot<ST, NW>(w1, x, acc);
        }
#pragma unroll
        for (int p = 0; p < RUN_RP; ++p)
          if (q0 + p < end) f.a[q0 + p] = acc[p];
      }
    }
    __syncthreads();
    if constexpr (SCHEME == 1) {
      res = f.a;
    } else {
      // N(a) - N(u) on [hs + 2hN, L - hs - 2hN)
      tile_nonlin_runs<ST, NONLIN, NW>(f.a, f.Na, f.N, HS + 2 * hN, L - HS - 2 * hN, sd1, ncoef, inv_h);
      __syncthreads();
      // u+ = a + (W2 (N(a) - N(u))) / dt on [H, L - H)
      ST w2[NW];
      run_row<ST, NW>(rows + 2 * DMAX, w2);
      for (int q0 = H + int(threadIdx.x) * RUN_RP; q0 < L - H; q0 += int(blockDim.x) * RUN_RP) {
        ST x[RUN_RP + NW - 1], acc[RUN_RP];
        run_window<ST, NW>(f.Na, q0 - WS, x);
#pragma unroll
        for (int p = 0; p < RUN_RP; ++p) acc[p] = ST(0);
        run_dot<ST, NW>(w2, x, acc);
#pragma unroll
        for (int p = 0; p < RUN_RP; ++p)
          if (q0 + p < L - H) res[q0 + p] = fma(acc[p], inv_dt, f.a[q0 + p]);
      }
    }
  }
  __syncthreads();
  for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) {
    const ST y = res[q];
    out[gbase + q] = y;
    bad |= !isfinite(y);
  }
}

// NW: the stencil width n of the launch (3 .. 15).
template <typename ST, int SCHEME, int NONLIN, int NW>
__global__ void __launch_bounds__(512) k_apply(ApplyParams a, const ST* __restrict__ u, ST* __restrict__ out,
                                               const ST* __restrict__ W, int wq, unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  ST* sW = reinterpret_cast<ST*>(smem);
  ST* sd1 = sW + MAXW;
  constexpr int n = NW, hs = (NW - 1) >> 1;
  constexpr bool KDV = NONLIN >= 2;                 // a derivative nonlinearity: KdV or Burgers
  const ST ncoef = ST(NONLIN == 2 ? -6 : -1);         // N = ncoef u u_x
  const int hN = KDV ? hs : 0;
  const int H = a.halo;
  const int F = a.tile + 2 * H + RUN_PAD;  // elements per field (slack for the runs of interior tiles)
  ST* su = sd1 + DMAX;
  ST* sN = su + F;
  ST* sa = sN + F;
  ST* sNa = sa + F;
  const TileFields<ST> fields{su, sN, sa, sNa};
  const ST inv_dt = ST(a.inv_dt);
  if (KDV)  // the centre row of h D^(1) from the device tables
    for (int j = threadIdx.x; j < n; j += blockDim.x) sd1[j] = ST(a.dh[hs * LD + j]);
  int64_t cur_inst = -1;
  ST inv_h = ST(0);
  unsigned bad = 0;
  const int64_t ntiles = a.ntiles;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int64_t b = 0, t0, off = 0, N = a.N;
    double h = a.h;
    int bc = a.bc;
    if (a.inst) {
      const int2 tt = a.tiles[tile];
      b = tt.x;
      t0 = tt.y;
      const Instance in = a.inst[b];
      off = in.off;
      N = in.N;
      h = in.h;
      bc = in.bc;
    } else {
      t0 = tile * int64_t(a.tile);
    }
    const int64_t t1 = t0 + a.tile < N ? t0 + a.tile : N;
    const int L = int(t1 - t0) + 2 * H;
    const int64_t base = t0 - H;  // global index of local 0
    const bool dir = bc == BC_DIRICHLET;
    __syncthreads();  // previous tile done with shared memory
    if (b != cur_inst) {
      // Dirichlet needs every row class; periodic and Neumann only the centre row.
      const ST* Wb = W + b * a.w_stride;
      const int nq = SCHEME + 1;
      const int r0 = dir ? 0 : hs + a.shift, r1 = dir ? n : hs + a.shift + 1;
      for (int e = threadIdx.x; e < (r1 - r0) * nq * n; e += blockDim.x) {
        const int r = r0 + e / (nq * n), rem = e % (nq * n);
        sW[(r * 3 + rem / n) * DMAX + rem % n] = Wb[(r * wq + rem / n) * n + rem % n];
      }
      cur_inst = b;
      inv_h = a.inst ? ST(1.0 / h) : ST(a.inv_h);
    }
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
      const int64_t i = base + q;
      ST v = ST(0);
      if (!dir || (i >= 0 && i < N)) v = u[off + grid_index(i, N, bc)];
      su[q] = v;
    }
    __syncthreads();
    // every staged point of an interior tile has a window inside the grid and is no wall
    const bool interior = !dir || (base - n >= 1 && base + L + n <= N - 2);
    if (interior) {
      tile_interior<ST, SCHEME, NONLIN, NW>(a, fields, sW, sd1, L, off + base, ncoef, inv_h, inv_dt, out, bad);
      continue;
    }
    // nonlinear term on [hN, L - hN)
    if (SCHEME != 0) {
      for (int q = hN + threadIdx.x; q < L - hN; q += blockDim.x) {
        const ST x = su[q];
        ST f;
        if (KDV) {
          ST ux = ST(0);
          for (int j = 0; j < n; ++j) ux = fma(sd1[j], su[q - hs + j], ux);
          f = ncoef * x * ux * inv_h;
        } else {
          f = x - x * x * x;
        }
        sN[q] = f;
      }
      __syncthreads();
    }
    // window of local point q: local start and harvest row
    auto window = [&](int q, int& ls, int& r) {
      if (dir) {
        const int64_t i = base + q;
        int64_t st = i - hs - a.shift;
        st = st < 0 ? 0 : (st > N - n ? N - n : st);
        ls = int(st - base);
        r = int(i - st);
      } else {
        ls = q - hs - a.shift;
        r = hs + a.shift;
      }
    };
    if (SCHEME == 0) {
      for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) {
        const int64_t i = base + q;
        ST y;
        if (dir && (i == 0 || i == N - 1)) {
          y = ST(i == 0 ? a.bc_lo : a.bc_hi);
        } else {
          int ls, r;
          window(q, ls, r);
          const ST* w0 = sW + (r * 3) * DMAX;
          ST acc = ST(0);
          for (int j = 0; j < n; ++j) acc = fma(w0[j], su[ls + j], acc);
          y = acc;
        }
        out[off + i] = y;
        bad |= !isfinite(y);
      }
      continue;
    }
    // first stage a = W0 u + W1 N(u) on [hs + hN, L - hs - hN)
    for (int q = hs + hN + threadIdx.x; q < L - hs - hN; q += blockDim.x) {
      const int64_t i = base + q;
      ST y = ST(0);
      if (dir && (i <= 0 || i >= N - 1)) {
        y = i == 0 ? ST(a.bc_lo) : (i == N - 1 ? ST(a.bc_hi) : ST(0));
      } else {
        int ls, r;
        window(q, ls, r);
        const ST* w0 = sW + (r * 3) * DMAX;
        const ST* w1 = w0 + DMAX;
        ST acc = ST(0);
        for (int j = 0; j < n; ++j) acc = fma(w0[j], su[ls + j], acc);
        for (int j = 0; j < n; ++j) acc = fma(w1[j], sN[ls + j], acc);
        y = acc;
      }
      sa[q] = y;
    }
    __syncthreads();
    if (SCHEME == 1) {
      for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) {
        const ST y = sa[q];
        out[off + base + q] = y;
        bad |= !isfinite(y);
      }
      continue;
    }
    // N(a) - N(u) on [hs + 2hN, L - hs - 2hN)
    for (int q = hs + 2 * hN + threadIdx.x; q < L - hs - 2 * hN; q += blockDim.x) {
      const ST x = sa[q];
      ST f;
      if (KDV) {
        ST ux = ST(0);
        for (int j = 0; j < n; ++j) ux = fma(sd1[j], sa[q - hs + j], ux);
        f = ncoef * x * ux * inv_h;
      } else {
        f = x - x * x * x;
      }
      sNa[q] = f - sN[q];
    }
    __syncthreads();
    for (int q = H + threadIdx.x; q < L - H; q += blockDim.x) {
      const int64_t i = base + q;
      ST y;
      if (dir && (i == 0 || i == N - 1)) {
        y = ST(i == 0 ? a.bc_lo : a.bc_hi);
      } else {
        int ls, r;
        window(q, ls, r);
        const ST* w2 = sW + (r * 3 + 2) * DMAX;
        ST acc = ST(0);
        for (int j = 0; j < n; ++j) acc = fma(w2[j], sNa[ls + j], acc);
        y = fma(acc, inv_dt, sa[q]);
      }
      out[off + i] = y;
      bad |= !isfinite(y);
    }
  }
  if (bad) atomicOr(flags, 1u);
}


// Kernel of a launch (lmep_apply.cu: FP32; lmep_apply_f64.cu: FP64).
template <typename ST, int NW>
const void* apply_pick_n(int scheme, int nonlin) {
  if (scheme == 0) return (const void*)k_apply<ST, 0, 0, NW>;
  if (scheme == 1)
    return nonlin == 3 ? (const void*)k_apply<ST, 1, 3, NW>
                       : (nonlin == 2 ? (const void*)k_apply<ST, 1, 2, NW> : (const void*)k_apply<ST, 1, 1, NW>);
  return nonlin == 3 ? (const void*)k_apply<ST, 2, 3, NW>
                     : (nonlin == 2 ? (const void*)k_apply<ST, 2, 2, NW> : (const void*)k_apply<ST, 2, 1, NW>);
}

template <typename ST>
const void* apply_pick(int scheme, int nonlin, int n) {
  switch (n) {
    case 3: return apply_pick_n<ST, 3>(scheme, nonlin);
    case 5: return apply_pick_n<ST, 5>(scheme, nonlin);
    case 7: return apply_pick_n<ST, 7>(scheme, nonlin);
    case 9: return apply_pick_n<ST, 9>(scheme, nonlin);
    case 11: return apply_pick_n<ST, 11>(scheme, nonlin);
    case 13: return apply_pick_n<ST, 13>(scheme, nonlin);
    default: return apply_pick_n<ST, 15>(scheme, nonlin);
  }
}

const void* apply_kernel_f32(int scheme, int nonlin, int n);
const void* apply_kernel_f64(int scheme, int nonlin, int n);

}  // namespace lmep
