// lmep_warp_kernel.cuh -- the one-warp-per-matrix kernel of steps (a1)-(a6).
//
// A single kernel template k_warp<D, PT> serves four jobs (runtime mode):
//   MODE_FULL        exp(A_p) of caller matrices, whole result   (a4)
//   MODE_CONST       constant-coefficient weight rows, one warp per
//                    (instance, row class)                        (a1)-(a5)
//   MODE_FROZEN_W    frozen-velocity weights of every point       (a1)-(a5)
//   MODE_FROZEN_STEP frozen-velocity step, weights applied at once (a1)-(a6)
// D is the matrix dimension (n, or n + n_phi for the augmented matrix); PT
// the Pade product type (double, or float for the FP32 form).  The state and
// weight dtype ST equals PT.
//
// The derivative matrices of the uniform window are built once per CTA by
// Fornberg's recursion (a2) into shared memory.  Each warp then assembles its
// matrix (a3), exponentiates it (a4) and harvests the needed rows (a5).  In
// MODE_FROZEN_STEP the harvested row is applied to the point's window at once
// (a6), so the weights never reach HBM.
#pragma once

#include "lmep_device.cuh"
#include "lmep_internal.h"

namespace lmep {

constexpr int DH_BYTES = 3 * DMAX * LD * 8;  // h^k D^(k), k = 1..3
constexpr int DHF_BYTES = 3 * DMAX * LD * 4;  // their FP32 copy (FP32 form)
template <typename PT>
constexpr int dh_bytes() { return DH_BYTES + (sizeof(PT) == 4 ? DHF_BYTES : 0); }
constexpr int WARPS = 4;                      // warps per CTA

enum { MODE_FULL = 0, MODE_CONST = 1, MODE_FROZEN_W = 2, MODE_FROZEN_STEP = 3 };

struct WarpJob {
  int mode;
  KParams p;
  int64_t items;        // matrices, (instance, row) pairs or points
  const double* A;      // MODE_FULL input
  double* E;            // MODE_FULL output
  int32_t* ms;          // MODE_FULL (m, s); frozen modes (m, s, a); nullable
  const double* h_inst; // MODE_CONST per-instance spacing, nullable
  const void* u;        // frozen velocities / state
  void* out;            // weights or next state
  unsigned* flags;
  const double* dh;     // h^k D^(k) tables of this n (device, FP64 and FP32), not MODE_FULL
  const float* dhf;
};

// X = cI I + c1h Dh1 + c2h Dh2 + c3h Dh3 on the n x n window, zero-padded to D.
template <int D>
__device__ __forceinline__ void assemble(double* X64, const double* Dh, int n, double cI, double c1h,
                                         double c2h, double c3h, int lane) {
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e - (e / D) * D;
    double x = 0.0;
    if (i < n && j < n) {
      const int o = i * LD + j;
      x = c1h * Dh[o];
      x = fma(c2h, Dh[DMAX * LD + o], x);
      if (c3h != 0.0) x = fma(c3h, Dh[2 * DMAX * LD + o], x);
      if (i == j) x += cI;
    }
    X64[i * LD + j] = x;
  }
}

// Augmented rows (transposed row-restricted form of Sec. 3.1, after Sidje
// 1998 / Al-Mohy & Higham 2011): row n holds dt at column r, row n+q holds dt
// at column n+q-1.
__device__ __forceinline__ void augment(double* X64, int n, int n_phi, int r, double dt, int lane) {
  if (lane == 0) {
    if (n_phi >= 1) X64[n * LD + r] = dt;
    for (int q = 1; q < n_phi; ++q) X64[(n + q) * LD + n + q - 1] = dt;
  }
}

// CTAs per SM: the FP32 form fits 4 CTAs of 4 warps in shared memory and in
// 128 registers per thread; the FP64 path fits 3 (measured faster than 2 CTAs
// with the full register file, despite some spills at n = 13).
template <typename PT>
constexpr int ctas_per_sm() { return sizeof(PT) == 4 ? 4 : 3; }

template <int D, typename PT>
__global__ void __launch_bounds__(32 * WARPS, ctas_per_sm<PT>()) k_warp(WarpJob job) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* Dh = reinterpret_cast<double*>(smem);
  float* Dhf = sizeof(PT) == 4 ? reinterpret_cast<float*>(smem + DH_BYTES) : nullptr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Ws<PT> w(smem + dh_bytes<PT>() + warp * Ws<PT>::BYTES);
  const KParams& p = job.p;
  const int mode = job.mode;
  const int n = p.n;
  if (mode != MODE_FULL) {
    // copy the window's derivative tables (built once per device)
    for (int e = threadIdx.x; e < 3 * DMAX * LD; e += blockDim.x) {
      Dh[e] = job.dh[e];
      if (Dhf) Dhf[e] = job.dhf[e];
    }
  }
  __syncthreads();
  using ST = PT;
  const ST* u = static_cast<const ST*>(job.u);
  ST* out = static_cast<ST*>(job.out);
  const bool dir = p.bc == BC_DIRICHLET;
  unsigned bad = 0;
  for (int64_t it = int64_t(blockIdx.x) * WARPS + warp; it < job.items; it += int64_t(gridDim.x) * WARPS) {
    if (mode == MODE_FULL) {
      for (int e = lane; e < D * D; e += 32) w.X64[(e / D) * LD + e % D] = job.A[it * D * D + e];
      __syncwarp();
      int m, s;
      warp_expm<D, PT>(w, lane, nullptr, 0, true, job.E + it * D * D, D, &m, &s);
      if (job.ms && lane == 0) {
        job.ms[2 * it] = m;
        job.ms[2 * it + 1] = s;
      }
      __syncwarp();
      continue;
    }
    if (mode == MODE_CONST) {
      int64_t b, rr;
      split_index(it, n, 2, b, rr);
      const int r = int(rr);
      const double h = job.h_inst ? job.h_inst[b] : p.h;
      const int q1 = 1 + p.n_phi;
      int rows[4];
      int nrows;
      double c1h = p.dt * p.c1 / h;
      if (p.n_phi == 0) {
        const int kr = recentring_shift(p.c1, p.dt / h, n, r);
        c1h += double(kr);
        rows[0] = r - kr;
        nrows = 1;
      } else {
        rows[0] = r;
        for (int q = 1; q <= p.n_phi; ++q) rows[q] = n + q - 1;
        nrows = q1;
      }
      assemble<D>(w.X64, Dh, n, p.dt * p.c0, c1h, p.dt * p.c2 / (h * h), p.dt * p.c3 / (h * h * h), lane);
      __syncwarp();
      augment(w.X64, n, p.n_phi, r, p.dt, lane);
      __syncwarp();
      warp_expm<D, PT>(w, lane, rows, nrows, false, nullptr, 0, nullptr, nullptr);
      ST* o = out + it * q1 * n;
      for (int e = lane; e < q1 * n; e += 32) o[e] = ST(w.V[(e / n) * DMAX + e % n]);
      __syncwarp();
      continue;
    }
    // frozen velocity: point i of instance b (instances of N points back to back)
    int64_t b, i;
    split_index(it, p.N, p.batch, b, i);
    const ST* ub = u + b * p.N;
    if (dir && (i == 0 || i == p.N - 1)) {  // walls keep their values; no weights
      if (out) {
        if (mode == MODE_FROZEN_STEP) {
          if (lane == 0) out[it] = ST(i == 0 ? p.bc_lo : p.bc_hi);
        } else {
          for (int j = lane; j < n; j += 32) out[it * n + j] = ST(0);
        }
      }
      continue;
    }
    const double ui = double(ub[i]);
    const int k = p.dep ? departure_shift(ui, p.dt, p.h, n, p.dt_h) : 0;
    const int64_t st = window_start(i, p.N, n, p.bc, k);
    const int r = int(i - st);
    const double a1 = p.c1 - p.fa * ui;
    const int kr = recentring_shift(a1, p.dt_h, n, r);
    const double c1h = fma(a1, p.dt_h, double(kr));
    Asm as{Dh, Dhf, n, p.c0dt, c1h, p.c2h, p.c3h, p.c0dt_f, 0.0f, p.c2h_f, p.c3h_f};
    if (sizeof(PT) == 4) {
      as.c1f = __double2float_rn(c1h);  // X is assembled in FP32 inside warp_expm
    } else {
      assemble<D>(w.X64, Dh, n, p.c0dt, c1h, p.c2h, p.c3h, lane);
      __syncwarp();
    }
    const int hr = r - kr;
    // the window values are loaded now so that their latency hides behind the expm
    ST uw = ST(0);
    if (mode == MODE_FROZEN_STEP && lane < n) uw = ub[grid_index(st + lane, p.N, p.bc)];
    int m_, s_, a_;
    warp_expm<D, PT>(w, lane, &hr, 1, false, nullptr, 0, &m_, &s_, &a_, sizeof(PT) == 4 ? &as : nullptr);
    if (job.ms && lane == 0) {
      job.ms[3 * it] = m_;
      job.ms[3 * it + 1] = s_;
      job.ms[3 * it + 2] = a_;
    }
    if (!out) {
      __syncwarp();
      continue;
    }
    if (mode == MODE_FROZEN_STEP) {
      ST acc = ST(0);
      if (lane < n) acc = ST(w.V[lane]) * uw;
      acc = warp_sum(acc);
      if (lane == 0) {
        out[it] = acc;
        bad |= !isfinite(acc);
      }
    } else {
      if (lane < n) out[it * n + lane] = ST(w.V[lane]);
    }
    __syncwarp();
  }
  if (bad) atomicOr(job.flags, 1u);
}

template <int D, typename PT>
cudaError_t run_warp(const WarpJob& job, cudaStream_t s) {
  const size_t smem = dh_bytes<PT>() + WARPS * Ws<PT>::BYTES;
  auto k = k_warp<D, PT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * WARPS, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  const int64_t need = (job.items + WARPS - 1) / WARPS;
  const int grid = int(need < cap ? (need > 0 ? need : 1) : cap);
  k<<<grid, 32 * WARPS, smem, s>>>(job);
  return cudaGetLastError();
}

template <typename PT>
cudaError_t dispatch_warp(int d, const WarpJob& job, cudaStream_t s) {
  switch (d) {
    case 3: return run_warp<3, PT>(job, s);
    case 4: return run_warp<4, PT>(job, s);
    case 5: return run_warp<5, PT>(job, s);
    case 6: return run_warp<6, PT>(job, s);
    case 7: return run_warp<7, PT>(job, s);
    case 8: return run_warp<8, PT>(job, s);
    case 9: return run_warp<9, PT>(job, s);
    case 10: return run_warp<10, PT>(job, s);
    case 11: return run_warp<11, PT>(job, s);
    case 12: return run_warp<12, PT>(job, s);
    case 13: return run_warp<13, PT>(job, s);
    case 14: return run_warp<14, PT>(job, s);
    case 15: return run_warp<15, PT>(job, s);
    case 16: return run_warp<16, PT>(job, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t warp_job_f64(int d, const WarpJob& job, cudaStream_t s);
cudaError_t warp_job_f32(int d, const WarpJob& job, cudaStream_t s);

}  // namespace lmep
