// lmep_runs.cuh -- runs of consecutive points per thread for the CTA-tiled
// stencil kernels (lmep_apply_rk4.cuh, lmep_apply_tile.cuh).
//
// On a tile whose points all take the centre row class, a stage's rows sit in
// registers and every thread updates a run of RUN_RP consecutive points from a
// window of RUN_RP + n - 1 values loaded once into registers: n FMAs and about
// (RUN_RP + n - 1) / RUN_RP shared-memory loads per point and stencil.  RUN_RP
// is odd, so the threads' windows start RUN_RP words apart, on 32 different
// banks.  A run may pass the end of its stage's range: its last points read
// the field's slack (RUN_PAD elements after each staged field) and are not
// stored.
#pragma once

namespace lmep {

constexpr int RUN_RP = 9;                 // consecutive points per thread and run
constexpr int RUN_PAD = RUN_RP + 16;      // slack after each staged field (n <= 16)

// Row of NW weights into registers.
template <typename ST, int NW>
__device__ __forceinline__ void run_row(const ST* src, ST (&w)[NW]) {
#pragma unroll
  for (int j = 0; j < NW; ++j) w[j] = src[j];
}

// A run's window: v[s .. s + RUN_RP + NW - 2].
template <typename ST, int NW>
__device__ __forceinline__ void run_window(const ST* v, int s, ST (&x)[RUN_RP + NW - 1]) {
#pragma unroll
  for (int j = 0; j < RUN_RP + NW - 1; ++j) x[j] = v[s + j];
}

// acc[p] += sum_j w[j] x[p + j], taps in order.
template <typename ST, int NW>
__device__ __forceinline__ void run_dot(const ST (&w)[NW], const ST (&x)[RUN_RP + NW - 1], ST (&acc)[RUN_RP]) {
#pragma unroll
  for (int p = 0; p < RUN_RP; ++p)
#pragma unroll
    for (int j = 0; j < NW; ++j) acc[p] = fma(w[j], x[p + j], acc[p]);
}

}  // namespace lmep
