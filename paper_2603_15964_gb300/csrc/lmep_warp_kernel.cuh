// lmep_warp_kernel.cuh -- the one-warp-per-matrix kernel of steps (a1)-(a6).
//
// A single kernel template k_warp<D, PT> serves five jobs (runtime mode):
//   MODE_FULL        exp(A_p) of caller matrices, whole result   (a4)
//   MODE_CONST       constant-coefficient weight rows, one warp per
//                    (instance, row class)                        (a1)-(a5)
//   MODE_FROZEN_W    frozen-velocity weights of every point       (a1)-(a5)
//   MODE_FROZEN_STEP frozen-velocity step, weights applied at once (a1)-(a6)
//   MODE_NODES       weight rows of every node of a non-uniform grid,
//                    one warp per node, its own derivative matrices (a1)-(a5)
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

#include <atomic>

#include "lmep_device.cuh"
#include "lmep_internal.h"

namespace lmep {

constexpr int DH_BYTES = 3 * DMAX * LD * 8;  // h^k D^(k), k = 1..3
constexpr int DHF_BYTES = 3 * DMAX * LD * 4;  // their FP32 copy (FP32 form)
template <typename PT>
constexpr int dh_bytes() { return DH_BYTES + (sizeof(PT) == 4 ? DHF_BYTES : 0); }
constexpr int WARPS = 4;                      // warps per CTA

enum { MODE_FULL = 0, MODE_CONST = 1, MODE_FROZEN_W = 2, MODE_FROZEN_STEP = 3, MODE_NODES = 4 };
// The two frozen-velocity modes (every point of a grid in chunks of 32).
__host__ __device__ constexpr bool frozen_mode(int mode) { return mode == MODE_FROZEN_W || mode == MODE_FROZEN_STEP; }

struct WarpJob {
  int mode;
  KParams p;
  int64_t items;        // matrices, (instance, row) pairs or points
  const double* A;      // MODE_FULL input
  double* E;            // MODE_FULL output
  int32_t* ms;          // MODE_FULL (m, s); frozen modes (m, s, a); nullable
  const double* h_inst; // MODE_CONST per-instance spacing, nullable
  const double* x;      // MODE_NODES: node coordinates (device, N, strictly increasing)
  const void* u;        // frozen velocities / state
  void* out;            // weights or next state
  unsigned* flags;
  const double* dh;     // h^k D^(k) tables of this n (device, FP64 and FP32), not MODE_FULL
  const float* dhf;
  int64_t span;         // frozen modes: consecutive points per warp (set by run_warp)
  // Frozen modes: exp(E) of the point-independent part E = c2h Dh2 + c3h Dh3 of
  // the local matrix (row-major, D x D, then its D absolute row sums) in the
  // product type; sl == 0 when unavailable.  Read as kernel parameters
  // (constant operands).
  int sl;
  union {
    float f[DMAX * DMAX + DMAX];
    double d[DMAX * DMAX + DMAX];
  } slt;
};

// Entry e of the exp(E) table of a launch in the product type PT.
template <typename PT>
__device__ __forceinline__ PT sl_entry(const WarpJob& job, int e) {
  if constexpr (sizeof(PT) == 4) return job.slt.f[e];
  else return job.slt.d[e];
}

// Largest error bound sum_j |l_j| R_j (R_j the absolute row sums of exp(E)) at
// which a frozen-velocity row is taken from the factorised form l(z)^T exp(E);
// the computed row is within a few units of roundoff times the bound of the
// exact one.
constexpr float SL_TAU = 16.0f;

// Row z of the advection exponential on the window: the Lagrange weights l_j(z)
// of the nodes 0..n-1 (Thm. 1: row r of exp(a Dh1) is l(r + a)), by prefix
// and suffix products (no division by z - j, exact at the nodes).
template <int D, typename T>
__device__ __forceinline__ void lagrange_weights(T z, T (&l)[D]) {
  T suf[D];
  suf[D - 1] = T(1);
#pragma unroll
  for (int j = D - 1; j > 0; --j) suf[j - 1] = suf[j] * (z - T(j));
  T pre = T(1);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    l[j] = pre * suf[j] * T(lagrange_den(D, j));
    pre *= z - T(j);
  }
}

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

// Largest error bound beta at which a frozen-velocity row is taken from the
// finite series; above it the row comes from Pade scaling and squaring.  The
// computed series stays within about 2 u beta of the exact row (u the unit
// roundoff of the summation type) on the Burgers distributions (nu = 1e-6 to
// 1e-3, n = 5..13, CFL 1..4), so these keep it below 2e-6 (FP32 sums in the
// FP32 form), 2.5e-10 (FP64 sums in the FP32 form) and 1.5e-14 (FP64 path),
// inside the parity tolerances of 1e-5 (FP32 form) and 1e-12 (FP64 path).
constexpr float SERIES_TAU_F32 = 16.0f;
constexpr float SERIES_TAU_F32_FORM_F64 = 1048576.0f;  // 2^20
constexpr float SERIES_TAU_F64 = 64.0f;

// Frozen-velocity points side by side in the finite series: GS lanes per point.
template <int D>
struct Groups {
  static constexpr int GS = D <= 4 ? 4 : (D <= 8 ? 8 : 16);
  static constexpr int G = 32 / GS;
};
// PT entries between the groups' broadcast buffers (two more for doubles, which
// moves the groups' 16-byte loads to different banks) and per ping-pong half.
template <int D, typename PT>
struct SeriesBuf {
  static constexpr int VS = Groups<D>::GS + (sizeof(PT) == 8 ? 2 : 0);
  static constexpr int VPP = Groups<D>::G * VS;
  static constexpr int WPP = 32;
  static constexpr int BYTES = 2 * VPP * int(sizeof(PT)) + 2 * WPP * 4;
};

// Finite-series rows (product type QT) of the chunk's points in `todo` (bit q
// = point c + q), G at a time: group g = lane / GS takes the g-th remaining
// point.  A row whose error bound is at most tau is stored (MODE_FROZEN_W) or
// applied to its window and handed to its point's lane in `res` (and, with
// statistics, its degree entry set to mcode); the points whose bound is larger
// are returned.  The per-point values hr, c1h, c1f, st and base live in the
// point's own lane.
template <int D, typename QT, typename ST>
__device__ __forceinline__ unsigned series_points(const WarpJob& job, const ST* u, ST* out, const double* Dh,
                                                  const float* Dhf, unsigned todo, int lane, int hr, double c1h,
                                                  float c1f, int64_t st, int64_t base, QT* vb, float* wb, float tau,
                                                  QT e0, int64_t c, int mcode, ST& res) {
  constexpr int GS = Groups<D>::GS, G = Groups<D>::G;
  using SB = SeriesBuf<D, QT>;
  const KParams& p = job.p;
  const int n = p.n;
  const int mode = job.mode;
  const int g = lane / GS, j = lane % GS;
  QT* vg = vb + g * SB::VS;
  float* wg = wb + g * GS;
  bool failed = false;
  while (todo) {
    unsigned t = todo;
    for (int k = 0; k < g; ++k) t &= t - 1;
    const int q = t ? __ffs(t) - 1 : -1;
#pragma unroll
    for (int k = 0; k < G; ++k) todo &= todo - 1;
    const bool has = q >= 0;
    const int qs = has ? q : 0;
    const int hr_q = __shfl_sync(FULL, hr, qs);
    const int64_t st_q = __shfl_sync(FULL, st, qs);
    const int64_t base_q = __shfl_sync(FULL, base, qs);
    Asm as{Dh, Dhf, n, 0.0, 0.0, p.c2h, p.c3h, 0.0f, 0.0f, p.c2h_f, p.c3h_f};
    if constexpr (sizeof(QT) == 4) as.c1f = __shfl_sync(FULL, c1f, qs);
    else as.c1h = __shfl_sync(FULL, c1h, qs);
    // the window values are loaded first so that their latency hides behind the series
    ST uw = ST(0);
    if (mode == MODE_FROZEN_STEP && has && j < n) uw = u[base_q + grid_index(st_q + j, p.N, p.bc)];
    QT row;
    const float beta = group_series_row<D, QT, GS, SB::VPP, SB::WPP>(as, j, hr_q, vg, wg, row);
    row *= e0;
    const bool ok = has && beta <= tau;
    if (mode == MODE_FROZEN_W && out && ok && j < n) out[(c + q) * n + j] = ST(row);
    const QT acc = group_sum<GS>(row * QT(uw));
    // each group's result to its point's lane
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int qk = __shfl_sync(FULL, q, k * GS);
      const QT ak = __shfl_sync(FULL, acc, k * GS);
      const bool okk = __shfl_sync(FULL, ok, k * GS);
      if (lane == qk) {
        if (okk) {
          res = ST(ak);
          if (job.ms && mcode) job.ms[3 * (c + qk)] = mcode;
        } else {
          failed = true;
        }
      }
    }
  }
  return __ballot_sync(FULL, failed);
}

// One chunk of the frozen-velocity modes: the points c .. min(c + 32, end) - 1.
// Lane l first prepares point c + l -- its value (one coalesced load for the
// chunk), departure shift, window, re-centring -- so that the scalar FP64 work
// of 32 points takes one pass.  The rows then come from, in order:
//   1. the finite series in the product type, G points side by side;
//   2. (FP32 form) the finite series in FP64 for the points 1 rejected --
//      at nu = 1e-6 the few next to Dirichlet walls, where the one-sided
//      second-derivative rows have large weights;
//   3. Pade scaling and squaring on the whole warp, one point at a time, for
//      the rest (every point when p.series == 0).
// Each result returns to its point's lane and the chunk leaves in one
// coalesced store.  u and out are the state and the output of the job's
// instance; with a point list (the rejected points of a frozen set, see
// lmep_frozen_set.cu) lane l takes point list[c + l] instead of c + l.
template <int D, typename PT>
__device__ __forceinline__ void frozen_chunk(const WarpJob& job, const Ws<PT>& w, const double* Dh,
                                             const float* Dhf, int64_t c, int64_t end, int lane, unsigned& bad,
                                             const PT* u, PT* out, const int32_t* list = nullptr) {
  using ST = PT;
  constexpr bool F32 = sizeof(PT) == 4;
  const KParams& p = job.p;
  const int n = p.n;
  const int mode = job.mode;
  // ---- lane-parallel preparation of point c + lane
  const bool valid = c + lane < end;
  const int64_t it = list ? (valid ? int64_t(list[c + lane]) : 0) : c + lane;
  int64_t b = 0, i = 0;
  if (valid) split_index(it, p.N, p.batch, b, i);
  const bool wall = valid && p.bc == BC_DIRICHLET && (i == 0 || i == p.N - 1);
  const bool live = valid && !wall;  // walls keep their values and get no weights
  const int64_t base = b * p.N;
  int64_t st;
  int hr;
  double c1h = 0.0;  // FP32 form: formed from c1f below, only for the rows that fall back
  float c1f = 0.0f;
  if constexpr (F32) {
    // in FP32 but for the window's integer decision next to a tie (exact FP64 test)
    const float uf = live ? float(u[base + i]) : 0.0f;
    const int k = p.dep ? departure_shift_f32(uf, p, n) : 0;
    st = window_start(i, p.N, n, p.bc, k);
    const int r = int(i - st);
    const float a1 = p.c1_f - p.fa_f * uf;
    // any re-centring shift in range gives the same row; the rounded one the smallest norm
    const int kr = int(fmaxf(float(r - (n - 1)), fminf(float(r), floorf(fmaf(-a1, p.dt_h_f, 0.5f)))));
    c1f = fmaf(a1, p.dt_h_f, float(kr));
    hr = r - kr;
  } else {
    const double ui = live ? double(u[base + i]) : 0.0;
    const int k = p.dep ? departure_shift(ui, p.dt, p.h, n, p.dt_h) : 0;
    st = window_start(i, p.N, n, p.bc, k);
    const int r = int(i - st);
    const double a1 = p.c1 - p.fa * ui;
    const int kr = recentring_shift(a1, p.dt_h, n, r);
    c1h = fma(a1, p.dt_h, double(kr));
    hr = r - kr;
  }
  ST res = ST(0);
  if (job.ms && live) {  // series rows (m = 0); the other routes overwrite m below
    job.ms[3 * it] = 0;
    job.ms[3 * it + 1] = 0;
    job.ms[3 * it + 2] = 0;
  }
  bool done = false;
  // 0. the factorised row: X = a Dh1 + E with E = c2h Dh2 + c3h Dh3 the same for
  //    every point, and the derivative matrices of the window commute (they are
  //    powers of one differentiation matrix on the local polynomial space), so
  //    e_r^T exp(X) = e_r^T exp(a Dh1) exp(E) = l(r + a)^T exp(E) (Thm. 1 and the
  //    General Exactness theorem); exp(E) comes with the launch
  if (job.sl && live) {
    PT l[D];
    if constexpr (F32) lagrange_weights<D, float>(float(hr) + c1f, l);  // r + a = (r - kr) + (a + kr)
    else lagrange_weights<D, double>(double(hr) + c1h, l);
    PT bound = PT(0);
#pragma unroll
    for (int j = 0; j < D; ++j) bound = fma(abs(l[j]), sl_entry<PT>(job, D * D + j), bound);
    if (bound <= PT(SL_TAU)) {
      const PT e0 = p.c0dt != 0.0 ? PT(exp(p.c0dt)) : PT(1);
      PT acc = PT(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        PT rk = PT(0);
#pragma unroll
        for (int j = 0; j < D; ++j) rk = fma(l[j], sl_entry<PT>(job, j * D + k), rk);
        rk *= e0;
        if (mode == MODE_FROZEN_STEP) acc = fma(rk, PT(u[base + grid_index(st + k, p.N, p.bc)]), acc);
        else if (out) out[it * n + k] = ST(rk);
      }
      res = ST(acc);
      done = true;
      if (job.ms) job.ms[3 * it] = 2;
    }
  }
  unsigned pade = __ballot_sync(FULL, live && !done);
  if (p.series) {
    // e^{dt c0}: the identity term, left out of the nilpotent part
    const double e0 = p.c0dt != 0.0 ? exp(p.c0dt) : 1.0;
    PT* vb = w.M(4);  // broadcast buffers in the Pade workspace, which the series does not use
    float* wb = reinterpret_cast<float*>(vb + 2 * SeriesBuf<D, PT>::VPP);
    pade = series_points<D, PT, ST>(job, u, out, Dh, Dhf, pade, lane, hr, c1h, c1f, st, base, vb, wb,
                                    F32 ? SERIES_TAU_F32 : SERIES_TAU_F64, PT(e0), c, 0, res);
    if constexpr (F32) {
      if (pade) {
        c1h = double(c1f);
        double* vd = reinterpret_cast<double*>(w.M(4));
        float* wd = reinterpret_cast<float*>(vd + 2 * SeriesBuf<D, double>::VPP);
        pade = series_points<D, double, ST>(job, u, out, Dh, Dhf, pade, lane, hr, c1h, c1f, st, base, vd, wd,
                                            SERIES_TAU_F32_FORM_F64, e0, c, 1, res);
      }
    }
  }
  // ---- Pade scaling and squaring, one point at a time on the whole warp
  if (F32 && pade) c1h = double(c1f);
  while (pade) {
    const int q = __ffs(pade) - 1;
    pade &= pade - 1;
    const int hr_q = __shfl_sync(FULL, hr, q);
    const int64_t st_q = __shfl_sync(FULL, st, q);
    const int64_t base_q = __shfl_sync(FULL, base, q);
    const double c1h_q = __shfl_sync(FULL, c1h, q);
    Asm as{Dh, Dhf, n, p.c0dt, c1h_q, p.c2h, p.c3h, p.c0dt_f, 0.0f, p.c2h_f, p.c3h_f};
    if constexpr (F32) as.c1f = __shfl_sync(FULL, c1f, q);  // X is assembled in FP32
    ST uw = ST(0);
    if (mode == MODE_FROZEN_STEP && lane < n) uw = u[base_q + grid_index(st_q + lane, p.N, p.bc)];
    if constexpr (!F32) {
      assemble<D>(w.X64, Dh, n, p.c0dt, c1h_q, p.c2h, p.c3h, lane);
      __syncwarp();
    }
    int mq, sq, aq;
    warp_expm<D, PT>(w, lane, &hr_q, 1, false, nullptr, 0, &mq, &sq, &aq, F32 ? &as : nullptr);
    const PT row = lane < n ? PT(w.V[lane]) : PT(0);
    if (mode == MODE_FROZEN_W && out && lane < n) out[(c + q) * n + lane] = ST(row);
    const ST acc = warp_sum(ST(row) * uw);
    if (lane == q) {
      res = acc;
      if (job.ms) {
        job.ms[3 * it] = mq;
        job.ms[3 * it + 1] = sq;
        job.ms[3 * it + 2] = aq;
      }
    }
    __syncwarp();
  }
  // ---- the chunk's results
  if (out && wall) {
    if (mode == MODE_FROZEN_STEP) out[it] = ST(i == 0 ? p.bc_lo : p.bc_hi);
    else for (int jj = 0; jj < n; ++jj) out[it * n + jj] = ST(0);
  }
  if (out && live && mode == MODE_FROZEN_STEP) {
    out[it] = res;
    bad |= !isfinite(res);
  }
}

// Store the harvested rows (w.V, FP64) of a constant-coefficient or per-node
// harvest: rows k = 0..n_phi of dt^k phi_k, or for ETDRK4 (p.rk4, n_phi = 3,
// Sec. 3) the rows of exp(X), dt alpha, dt beta, dt gamma, formed in FP64 with
// alpha = phi_1 - 3 phi_2 + 4 phi_3, beta = 2 phi_2 - 4 phi_3, gamma = 4 phi_3 - phi_2.
template <typename PT>
__device__ __forceinline__ void emit_rows(const KParams& p, const Ws<PT>& w, PT* o, int lane) {
  const int n = p.n;
  if (p.rk4 && p.n_phi == 3) {
    const double i1 = 1.0 / p.dt, i2 = i1 * i1;
    for (int j = lane; j < n; j += 32) {
      const double w1 = w.V[DMAX + j], w2 = w.V[2 * DMAX + j] * i1, w3 = w.V[3 * DMAX + j] * i2;
      o[j] = PT(w.V[j]);
      o[n + j] = PT(w1 - 3.0 * w2 + 4.0 * w3);
      o[2 * n + j] = PT(2.0 * w2 - 4.0 * w3);
      o[3 * n + j] = PT(4.0 * w3 - w2);
    }
  } else {
    for (int e = lane; e < (1 + p.n_phi) * n; e += 32) o[e] = PT(w.V[(e / n) * DMAX + e % n]);
  }
}

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
  if (job.sl) {
    // factorised launches: the few rows that fall back read the tables from global memory
    Dh = const_cast<double*>(job.dh);
    if (Dhf) Dhf = const_cast<float*>(job.dhf);
  } else if (mode != MODE_FULL && mode != MODE_NODES) {
    // copy the window's derivative tables (built once per device)
    for (int e = threadIdx.x; e < 3 * DMAX * LD; e += blockDim.x) {
      Dh[e] = job.dh[e];
      if (Dhf) Dhf[e] = job.dhf[e];
    }
  }
  __syncthreads();
  using ST = PT;
  ST* out = static_cast<ST*>(job.out);
  unsigned bad = 0;
  if (frozen_mode(mode)) {
    static_assert(SeriesBuf<D, PT>::BYTES <= DMAX * Ws<PT>::LDM * int(sizeof(PT)) &&
                      SeriesBuf<D, double>::BYTES <= DMAX * Ws<PT>::LDM * int(sizeof(PT)),
                  "the series buffers fit in one product matrix");
    // one contiguous range of points per warp (every warp of the grid is resident),
    // in chunks of equal size up to 32
    const int64_t begin = (int64_t(blockIdx.x) * WARPS + warp) * job.span;
    const int64_t end = begin + job.span < job.items ? begin + job.span : job.items;
    const int64_t csz = (job.span + (job.span + 31) / 32 - 1) / ((job.span + 31) / 32);
    for (int64_t c = begin; c < end; c += csz)
      frozen_chunk<D, PT>(job, w, Dh, Dhf, c, c + csz < end ? c + csz : end, lane, bad,
                          static_cast<const PT*>(job.u), static_cast<PT*>(job.out));
    if (bad) atomicOr(job.flags, 1u);
    return;
  }
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
    if (mode == MODE_NODES) {
      // non-uniform grid (Sec. 4.3.3): the window's own derivative matrices, in local
      // coordinates xi = (x - x_s) / hl (hl the window's mean spacing), built by
      // Fornberg's recursion into the product-matrix area of the workspace, which the
      // exponential does not use before it reads X
      int64_t st = it - (n - 1) / 2;
      st = st < 0 ? 0 : (st > p.N - n ? p.N - n : st);
      const int r = int(it - st);
      const double x0 = job.x[st];
      const double hl = (job.x[st + n - 1] - x0) / double(n - 1);
      static_assert(Ws<PT>::VEC_OFF - Ws<PT>::PRD_OFF >= 3 * DMAX * LD * 8,
                    "the window's derivative tables fit between X and the harvested rows");
      double* Dn = reinterpret_cast<double*>(w.P);
      if (lane < n) {
        double xs[DMAX], c[4][DMAX];
        for (int m = 0; m < DMAX; ++m) xs[m] = m < n ? (job.x[st + m] - x0) / hl : 0.0;
        fornberg_row_nodes(xs[lane], xs, n, c);
        for (int k = 1; k <= 3; ++k)
          for (int m = 0; m < DMAX; ++m) Dn[(k - 1) * DMAX * LD + lane * LD + m] = m < n ? c[k][m] : 0.0;
      }
      __syncwarp();
      assemble<D>(w.X64, Dn, n, p.dt * p.c0, p.dt * p.c1 / hl, p.dt * p.c2 / (hl * hl),
                  p.dt * p.c3 / (hl * hl * hl), lane);
      __syncwarp();
      augment(w.X64, n, p.n_phi, r, p.dt, lane);
      __syncwarp();
      int rows[4];
      rows[0] = r;
      for (int q = 1; q <= p.n_phi; ++q) rows[q] = n + q - 1;
      warp_expm<D, PT>(w, lane, rows, 1 + p.n_phi, false, nullptr, 0, nullptr, nullptr);
      emit_rows(p, w, out + it * (p.w_rows > 0 ? p.w_rows : 1 + p.n_phi) * n + int64_t(p.w_row0) * n, lane);
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
      const int wr = p.w_rows > 0 ? p.w_rows : q1;
      emit_rows(p, w, out + it * wr * n + int64_t(p.w_row0) * n, lane);
      __syncwarp();
      continue;
    }
  }
  if (bad) atomicOr(job.flags, 1u);
}

// exp(E) of the point-independent part E = c2h Dh2 + c3h Dh3 of a
// frozen-velocity local matrix, computed by one warp (FP64 Pade scaling and
// squaring) into out (D x D row-major, global), then Dh2 exp(E) into out2:
// the direction of d exp(E) / d c2h (Dh2 commutes with E).  Dh is the
// warp's shared copy of the derivative tables, filled here from dh.
template <int D>
__device__ __forceinline__ void exp_const_warp(const KParams& p, const double* dh, double* Dh, const Ws<double>& w,
                                               double* out, double* out2, int lane) {
  for (int e = lane; e < 3 * DMAX * LD; e += 32) Dh[e] = dh[e];
  __syncwarp();
  assemble<D>(w.X64, Dh, p.n, 0.0, 0.0, p.c2h, p.c3h, lane);
  __syncwarp();
  int m, s;
  warp_expm<D, double>(w, lane, nullptr, 0, true, out, D, &m, &s);
  __syncwarp();  // orders the global writes of exp(E) before the product below
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e - (e / D) * D;
    double acc = 0.0;
    for (int k = 0; k < D; ++k) acc = fma(Dh[DMAX * LD + i * LD + k], out[k * D + j], acc);
    out2[e] = acc;
  }
  __syncwarp();
}

// Resident CTAs per SM of k_warp<D, PT>, set up once per device (the shared
// memory attribute and the occupancy query are host calls worth skipping on
// every launch); 0 on failure, with the error in *err.
template <int D, typename PT>
int warp_ctas_per_sm(size_t smem, cudaError_t* err) {
  static std::atomic<int> cache[64];
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess || dev < 0 || dev >= 64) {
    if (*err == cudaSuccess) *err = cudaErrorInvalidDevice;
    return 0;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  auto k = k_warp<D, PT>;
  *err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (*err != cudaSuccess) return 0;
  int per_sm = 1;
  *err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * WARPS, smem);
  if (*err != cudaSuccess) return 0;
  v = per_sm < 1 ? 1 : per_sm;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

template <int D, typename PT>
cudaError_t run_warp(const WarpJob& job_in, cudaStream_t s) {
  const size_t smem = dh_bytes<PT>() + WARPS * Ws<PT>::BYTES;
  cudaError_t e = cudaSuccess;
  const int per_sm = warp_ctas_per_sm<D, PT>(smem, &e);
  if (per_sm == 0) return e;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  WarpJob job = job_in;
  int64_t need;
  need = (job.items + WARPS - 1) / WARPS;
  if (frozen_mode(job.mode)) {
    // frozen modes: every warp of the grid (all resident) takes one contiguous
    // range of points, so that the SMs finish together
    const int64_t g = need < cap ? (need > 0 ? need : 1) : cap;
    job.span = (job.items + g * WARPS - 1) / (g * WARPS);
    if (job.span < 1) job.span = 1;
  }
  const int grid = int(need < cap ? (need > 0 ? need : 1) : cap);
  k_warp<D, PT><<<grid, 32 * WARPS, smem, s>>>(job);
  return cudaGetLastError();
}

// The instantiations are split by width over two translation units per
// product type (d <= 9 and d >= 10), which keeps every unit's compile time short.
template <typename PT>
cudaError_t dispatch_warp_lo(int d, const WarpJob& job, cudaStream_t s) {
  switch (d) {
    case 3: return run_warp<3, PT>(job, s);
    case 4: return run_warp<4, PT>(job, s);
    case 5: return run_warp<5, PT>(job, s);
    case 6: return run_warp<6, PT>(job, s);
    case 7: return run_warp<7, PT>(job, s);
    case 8: return run_warp<8, PT>(job, s);
    case 9: return run_warp<9, PT>(job, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename PT>
cudaError_t dispatch_warp_hi(int d, const WarpJob& job, cudaStream_t s) {
  switch (d) {
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

cudaError_t warp_job_f32_hi(int d, const WarpJob& job, cudaStream_t s);
cudaError_t warp_job_f64_hi(int d, const WarpJob& job, cudaStream_t s);
cudaError_t warp_job_f64(int d, const WarpJob& job, cudaStream_t s);
cudaError_t warp_job_f32(int d, const WarpJob& job, cudaStream_t s);

}  // namespace lmep
