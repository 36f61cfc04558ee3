// lmep_adjoint.cu -- step (a7): one reverse step of the frozen-velocity scheme.
//
// Forward (per updated point i): u+_i = w_i . u[window_i], w_i = row r_i of
// exp(X_i), X_i = dt (c0 + c1 D1 + c2 D2 + c3 D3 - fa u_i D1).  The paper has
// no adjoint; this is the exact transpose of the step's linearisation:
//   lam_k  = sum_i lam+_i w_i[k - start_i]  +  lam+_k (dw_k/du_k . u[window_k])
//   dJ/dnu += sum_i lam+_i (dw_i/dnu . u[window_i]).
// dw/du_i and dw/dnu are rows of the Frechet derivative L(X, E) of the
// matrix exponential in the directions E = -dt fa/h Dh1 and E = dt/h^2 Dh2
// (Higham, Functions of Matrices, 2008, Sec. 3.2).  L is obtained by
// differentiating every step of Pade-13 scaling and squaring with the
// product rule (the approach of Al-Mohy & Higham, SIMAX 30(4), 2009):
//   powers  A_2k and their derivatives M_2k,
//   U, V and L_U, L_V,
//   R = Q^-1 P and L = Q^-1 [(L_U + L_V) + (L_U - L_V) R],
//   squaring  L <- R L + L R,  R <- R^2.
// With the exp(E) table of the handle (E = c2h Dh2 + c3h Dh3, the point-
// independent part of X) the derivatives are taken in closed form instead:
// the row is w = e^{dt c0} l(z)^T exp(E) with z = r + dt (c1 - fa u_i) / h
// (the derivative matrices commute, Thm. 1), so
//   dw/du_i = -dt fa / h e^{dt c0} l'(z)^T exp(E),
//   dw/dnu  =  dt / h^2  e^{dt c0} l(z)^T Dh2 exp(E),
// one point per thread (k_adjoint_fact); points whose bound
// sum_j |l_j| |row j of exp(E)|_1 exceeds 16 are marked and take the Pade
// derivatives in k_adjoint_points.
// The Pade Frechet path runs in FP64; the factorised path in the product type of
// the state (FP64, or FP32 for the FP32 form) with dnu summed in FP64; lam is
// stored in the state dtype.
// The exact re-centring of the forward step (row r of exp(X) equals row r-k
// of exp(X + k Dh1)) shifts X by a constant matrix, so the directions E are
// unchanged and the same identity holds for L.
#include <climits>
#include <cstdio>
#include <type_traits>

#include "lmep_device.cuh"
#include "lmep_internal.h"

namespace lmep {

namespace {

constexpr int AW = 2;                      // warps per CTA
constexpr int DHB = 3 * DMAX * LD * 8;     // Dh1..Dh3 bytes (DMAX x LD layout of the tables)
constexpr int NMAT = 20;                   // matrices per warp

// Per-warp workspace sized for the window: d x d matrices with row stride
// d + 1 and the Gauss-Jordan block [Q | 5 right-hand sides] with row stride
// 6 d + 1, so that small stencils fit several warps per SM.
template <int D>
struct AdjWs {
  static constexpr int LDA = D + 1;
  static constexpr int MAT = D * LDA;
  static constexpr int LDGA = 6 * D + 1;
  static constexpr int BYTES = (NMAT * MAT + D * LDGA) * 8;
};

template <int D>
__device__ __forceinline__ void mm(const double* A, const double* B, double* C, int lane, double beta = 0.0) {
  constexpr int LA = AdjWs<D>::LDA;
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e - (e / D) * D;
    double acc = beta == 0.0 ? 0.0 : beta * C[i * LA + j];
#pragma unroll
    for (int k = 0; k < D; ++k) acc = fma(A[i * LA + k], B[k * LA + j], acc);
    C[i * LA + j] = acc;
  }
  __syncwarp();
}

// C = a0 M0 + a1 M1 + a2 M2 + cI I   (any Mi may be null)
template <int D>
__device__ __forceinline__ void lc(double* C, double a0, const double* M0, double a1, const double* M1,
                                   double a2, const double* M2, double cI, int lane) {
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e - (e / D) * D, o = i * AdjWs<D>::LDA + j;
    double x = (i == j) ? cI : 0.0;
    if (M0) x = fma(a0, M0[o], x);
    if (M1) x = fma(a1, M1[o], x);
    if (M2) x = fma(a2, M2[o], x);
    C[o] = x;
  }
  __syncwarp();
}

// Gauss-Jordan with partial pivoting on G = [Q | B1 | ... | B_nb] (row stride 6 D + 1,
// the right-hand-side blocks contiguous after Q).
template <int D>
__device__ void gj_multi(double* G, int nb, int lane) {
  constexpr int ldg = AdjWs<D>::LDGA;
  const int W = D * (1 + nb);
  for (int k = 0; k < D; ++k) {
    long long key = -1;
    int idx = k;
    if (lane >= k && lane < D) {
      key = __double_as_longlong(G[lane * ldg + k]) & 0x7fffffffffffffffll;
      idx = lane;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const long long ok = __shfl_xor_sync(FULL, key, o);
      const int oi = __shfl_xor_sync(FULL, idx, o);
      if (ok > key || (ok == key && oi < idx)) {
        key = ok;
        idx = oi;
      }
    }
    if (idx != k) {
      for (int j = lane; j < W; j += 32) {
        const double t = G[k * ldg + j];
        G[k * ldg + j] = G[idx * ldg + j];
        G[idx * ldg + j] = t;
      }
    }
    __syncwarp();
    const double inv = 1.0 / G[k * ldg + k];
    for (int j = k + 1 + lane; j < W; j += 32) G[k * ldg + j] *= inv;
    __syncwarp();
    const int nc = W - k - 1;
    for (int e = lane; e < (D - 1) * nc; e += 32) {
      const int ii = e / nc, cc = e - (e / nc) * nc;
      const int i = ii + (ii >= k ? 1 : 0);
      const int j = k + 1 + cc;
      G[i * ldg + j] = fma(-G[i * ldg + k], G[k * ldg + j], G[i * ldg + j]);
    }
    __syncwarp();
  }
}

// Window offset of a point left to k_adjoint_points by k_adjoint_fact.
constexpr int32_t ADJ_MARK = INT32_MIN;

// Warps take chunks of 32 consecutive points; with fix != 0 only the points
// that k_adjoint_fact marked (st_out == ADJ_MARK), otherwise every point.
template <int D, typename ST>
__global__ void __launch_bounds__(32 * AW) k_adjoint_points(KParams p, const ST* __restrict__ u,
                                                            const ST* __restrict__ lam_next, ST* __restrict__ Wout,
                                                            ST* __restrict__ gu_out, int32_t* __restrict__ st_out,
                                                            double* dnu, int fix, const int* marks) {
  extern __shared__ __align__(16) unsigned char smem[];
  // after k_adjoint_fact: nothing marked (the usual case), so every CTA leaves
  if (fix && *marks == 0) return;
  double* Dh = reinterpret_cast<double*>(smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int LA = AdjWs<D>::LDA;
  double* base = reinterpret_cast<double*>(smem + DHB + warp * AdjWs<D>::BYTES);
  auto Mt = [&](int q) { return base + q * AdjWs<D>::MAT; };
  double* X = Mt(0);
  double* A2 = Mt(1);
  double* A4 = Mt(2);
  double* A6 = Mt(3);
  double* W1 = Mt(4);
  double* Z1 = Mt(5);
  double* Wm = Mt(6);   // W = A6 W1 + W2, later R
  double* T = Mt(7);
  double* E[2] = {Mt(8), Mt(9)};
  double* M2[2] = {Mt(10), Mt(11)};
  double* M4[2] = {Mt(12), Mt(13)};
  double* M6[2] = {Mt(14), Mt(15)};
  double* LU[2] = {Mt(16), Mt(17)};
  double* LV[2] = {Mt(18), Mt(19)};
  double* G = base + NMAT * AdjWs<D>::MAT;
  constexpr int ldg = AdjWs<D>::LDGA;
  __shared__ double dnu_blk;
  if (threadIdx.x == 0) dnu_blk = 0.0;
  fornberg_block(Dh, p.n);
  __syncthreads();
  const int n = p.n;
  const bool dir = p.bc == BC_DIRICHLET;
  constexpr double b13 = pade_b(13, 13), b12 = pade_b(13, 12), b11 = pade_b(13, 11), b10 = pade_b(13, 10),
                   b9 = pade_b(13, 9), b8 = pade_b(13, 8), b7 = pade_b(13, 7), b6 = pade_b(13, 6),
                   b5 = pade_b(13, 5), b4 = pade_b(13, 4), b3 = pade_b(13, 3), b2 = pade_b(13, 2),
                   b1 = pade_b(13, 1), b0 = pade_b(13, 0);
  double dnu_acc = 0.0;
  const int64_t items = p.N * (p.batch > 1 ? p.batch : 1);
  for (int64_t c = (int64_t(blockIdx.x) * AW + warp) * 32; c < items; c += int64_t(gridDim.x) * AW * 32) {
   const bool mine = c + lane < items && (!fix || st_out[c + lane] == ADJ_MARK);
   unsigned todo = __ballot_sync(FULL, mine);
   while (todo) {
    const int64_t it = c + (__ffs(todo) - 1);
    todo &= todo - 1;
    // the squaring phase swaps these scratch roles in place: every point starts from the same layout
    T = Mt(7);
    for (int q = 0; q < 2; ++q) {
      LU[q] = Mt(16 + q);
      LV[q] = Mt(18 + q);
    }
    int64_t bb, i;
    split_index(it, p.N, p.batch, bb, i);
    const ST* ub = u + bb * p.N;
    if (dir && (i == 0 || i == p.N - 1)) {
      for (int j = lane; j < n; j += 32) Wout[j * items + it] = ST(0);
      if (lane == 0) {
        gu_out[it] = ST(0);
        st_out[it] = 0;
      }
      continue;
    }
    const double ui = double(ub[i]);
    const int k = p.dep ? departure_shift(ui, p.dt, p.h, n, p.dt_h) : 0;
    const int64_t st = window_start(i, p.N, n, p.bc, k);
    const int r = int(i - st);
    const double a1 = p.c1 - p.fa * ui;
    const int kr = recentring_shift(a1, p.dt_h, n, r);
    const int hr = r - kr;
    // X (re-centred) and the two directions
    const double c1h = p.dt * a1 / p.h + double(kr);
    const double c2h = p.dt * p.c2 / (p.h * p.h), c3h = p.dt * p.c3 / (p.h * p.h * p.h);
    for (int e = lane; e < D * D; e += 32) {
      const int a = e / D, b = e - (e / D) * D, od = a * LD + b, o = a * LA + b;
      double x = c1h * Dh[od];
      x = fma(c2h, Dh[DMAX * LD + od], x);
      if (c3h != 0.0) x = fma(c3h, Dh[2 * DMAX * LD + od], x);
      if (a == b) x += p.dt * p.c0;
      X[o] = x;
      E[0][o] = -(p.dt * p.fa / p.h) * Dh[od];
      E[1][o] = (p.dt / (p.h * p.h)) * Dh[DMAX * LD + od];
    }
    __syncwarp();
    double cs = 0.0;
    if (lane < D)
      for (int a = 0; a < D; ++a) cs += fabs(X[a * LA + lane]);
    const double nrm = warp_max(cs);
    int s = 0;
    {
      double t = nrm;
      while (t > THETA13 && s < 1023) { t *= 0.5; ++s; }
    }
    const double sc = ldexp(1.0, -s);
    for (int e = lane; e < D * D; e += 32) {
      const int o = (e / D) * LA + e % D;
      X[o] *= sc;
      E[0][o] *= sc;
      E[1][o] *= sc;
    }
    __syncwarp();
    mm<D>(X, X, A2, lane);
    mm<D>(A2, A2, A4, lane);
    mm<D>(A4, A2, A6, lane);
    for (int q = 0; q < 2; ++q) {
      mm<D>(X, E[q], M2[q], lane);
      mm<D>(E[q], X, M2[q], lane, 1.0);
      mm<D>(A2, M2[q], M4[q], lane);
      mm<D>(M2[q], A2, M4[q], lane, 1.0);
      mm<D>(A4, M2[q], M6[q], lane);
      mm<D>(M4[q], A2, M6[q], lane, 1.0);
    }
    lc<D>(W1, b13, A6, b11, A4, b9, A2, 0.0, lane);
    lc<D>(Z1, b12, A6, b10, A4, b8, A2, 0.0, lane);
    lc<D>(Wm, b7, A6, b5, A4, b3, A2, b1, lane);      // W2
    mm<D>(A6, W1, Wm, lane, 1.0);                      // W = A6 W1 + W2
    // derivatives: LW = A6 LW1 + M6 W1 + LW2 ; LU = X LW + E W ; LV = A6 LZ1 + M6 Z1 + LZ2
    for (int q = 0; q < 2; ++q) {
      lc<D>(T, b13, M6[q], b11, M4[q], b9, M2[q], 0.0, lane);          // LW1
      lc<D>(LV[q], b7, M6[q], b5, M4[q], b3, M2[q], 0.0, lane);         // LW2 (temporarily in LV)
      mm<D>(A6, T, LV[q], lane, 1.0);
      mm<D>(M6[q], W1, LV[q], lane, 1.0);                               // LW
      mm<D>(X, LV[q], LU[q], lane);
      mm<D>(E[q], Wm, LU[q], lane, 1.0);                                // LU
      lc<D>(T, b12, M6[q], b10, M4[q], b8, M2[q], 0.0, lane);           // LZ1
      lc<D>(LV[q], b6, M6[q], b4, M4[q], b2, M2[q], 0.0, lane);         // LZ2
      mm<D>(A6, T, LV[q], lane, 1.0);
      mm<D>(M6[q], Z1, LV[q], lane, 1.0);                               // LV
    }
    // U = X W (into T), V = A6 Z1 + Z2 (into W1)
    mm<D>(X, Wm, T, lane);
    lc<D>(W1, b6, A6, b4, A4, b2, A2, b0, lane);
    mm<D>(A6, Z1, W1, lane, 1.0);
    // G = [V-U | V+U | LU+LV (u) | LU-LV (u) | LU+LV (nu) | LU-LV (nu)]
    for (int e = lane; e < D * D; e += 32) {
      const int a = e / D, b = e - (e / D) * D, o = a * LA + b;
      const double Uv = T[o], Vv = W1[o];
      G[a * ldg + b] = Vv - Uv;
      G[a * ldg + D + b] = Vv + Uv;
      for (int q = 0; q < 2; ++q) {
        G[a * ldg + (2 + 2 * q) * D + b] = LU[q][o] + LV[q][o];
        G[a * ldg + (3 + 2 * q) * D + b] = LU[q][o] - LV[q][o];
      }
    }
    __syncwarp();
    gj_multi<D>(G, 5, lane);
    // R into Wm, L_q = Y1 + Y2 R into LU[q]
    double* R = Wm;
    for (int e = lane; e < D * D; e += 32) {
      const int a = e / D, b = e - (e / D) * D, o = a * LA + b;
      R[o] = G[a * ldg + D + b];
      for (int q = 0; q < 2; ++q) {
        LU[q][o] = G[a * ldg + (2 + 2 * q) * D + b];
        LV[q][o] = G[a * ldg + (3 + 2 * q) * D + b];
      }
    }
    __syncwarp();
    for (int q = 0; q < 2; ++q) mm<D>(LV[q], R, LU[q], lane, 1.0);
    // squaring: L <- R L + L R ; R <- R R
    for (int t = 0; t < s; ++t) {
      for (int q = 0; q < 2; ++q) {
        mm<D>(R, LU[q], LV[q], lane);
        mm<D>(LU[q], R, LV[q], lane, 1.0);
        double* sw = LU[q];
        LU[q] = LV[q];
        LV[q] = sw;
      }
      mm<D>(R, R, T, lane);
      double* sw = R;
      R = T;
      T = sw;
    }
    // outputs: w = R[hr], g_q = L_q[hr] . u[window]
    double uj = 0.0;
    if (lane < n) uj = double(ub[grid_index(st + lane, p.N, p.bc)]);
    const double gu = warp_sum(lane < n ? LU[0][hr * LA + lane] * uj : 0.0);
    const double gn = warp_sum(lane < n ? LU[1][hr * LA + lane] * uj : 0.0);
    if (lane < n) Wout[lane * items + it] = ST(R[hr * LA + lane]);
    __syncwarp();  // every lane has read this chunk's marks before lane 0 overwrites st_out
    if (lane == 0) {
      gu_out[it] = ST(gu);
      st_out[it] = int32_t(st - i);
      dnu_acc += double(lam_next[it]) * gn;
    }
    __syncwarp();
   }
  }
  if (lane == 0 && dnu_acc != 0.0) atomicAdd(&dnu_blk, dnu_acc);
  __syncthreads();
  if (threadIdx.x == 0 && dnu_blk != 0.0) atomicAdd(dnu, dnu_blk);
}

// The factorised tables of one launch, as kernel parameters: exp(E), its
// absolute row sums and Dh2 exp(E), row-major D x D.
template <int D>
struct AdjTables {
  double ex[D * D];
  double rs[D];
  double d2ex[D * D];
};
// The FP32 form's tables (exp(E), its absolute row sums and Dh2 exp(E) rounded
// to FP32): with the loops unrolled, the rows are constant-bank operands.
template <int D>
struct AdjTablesF {
  float ex[D * D];
  float rs[D];
  float d2ex[D * D];
};
template <int D, typename ST>
using AdjTab = typename std::conditional<sizeof(ST) == 4, AdjTablesF<D>, AdjTables<D>>::type;

// One point per thread: the row w, g_u = dw/du_i . u[window] and the window
// offset into the scratch arrays of k_adjoint_gather, lam+_i dw/dnu . u[window]
// into dnu; a point whose bound exceeds the threshold gets st_out = ADJ_MARK.
// The window and the departure position z are formed in FP64; the FP32 form
// (ST = float) then takes the weights, their derivatives and the three rows in
// FP32 (the precision of its forward rows), and every form sums dnu in FP64.
template <int D, typename ST>
__global__ void __launch_bounds__(128) k_adjoint_fact(KParams p, AdjTab<D, ST> t, const ST* __restrict__ u,
                                                      const ST* __restrict__ lam_next, ST* __restrict__ Wout,
                                                      ST* __restrict__ gu_out, int32_t* __restrict__ st_out,
                                                      double* dnu, int* marks) {
  const int n = p.n;
  const bool dir = p.bc == BC_DIRICHLET;
  const int64_t items = p.N * (p.batch > 1 ? p.batch : 1);
  const double e0 = p.c0dt != 0.0 ? exp(p.c0dt) : 1.0;
  // d z / d u_i = -dt fa / h; the FP32 form takes it from its FP32 roundings (no FP64 division per thread)
  const double su = sizeof(ST) == 4 ? double(-p.fa_f * p.dt_h_f) : -p.dt * p.fa / p.h;
  double dnu_acc = 0.0;
  for (int64_t it = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; it < items;
       it += int64_t(gridDim.x) * blockDim.x) {
    int64_t bb, i;
    split_index(it, p.N, p.batch, bb, i);
    const ST* ub = u + bb * p.N;
    if (dir && (i == 0 || i == p.N - 1)) {
      for (int j = 0; j < n; ++j) Wout[j * items + it] = ST(0);
      gu_out[it] = ST(0);
      st_out[it] = 0;
      continue;
    }
    using CT = ST;  // arithmetic type of the rows
    int64_t st;
    CT zc;
    if constexpr (sizeof(CT) == 4) {
      // the FP32 form's window and departure position, as its forward step forms them
      const float uf = float(ub[i]);
      const int k = p.dep ? departure_shift_f32(uf, p, n) : 0;
      st = window_start(i, p.N, n, p.bc, k);
      const int r = int(i - st);
      const float a1 = p.c1_f - p.fa_f * uf;
      const int kr = int(fmaxf(float(r - (n - 1)), fminf(float(r), floorf(fmaf(-a1, p.dt_h_f, 0.5f)))));
      zc = float(r - kr) + fmaf(a1, p.dt_h_f, float(kr));
    } else {
      const double ui = double(ub[i]);
      const int k = p.dep ? departure_shift(ui, p.dt, p.h, n, p.dt_h) : 0;
      st = window_start(i, p.N, n, p.bc, k);
      zc = double(i - st) + p.dt * (p.c1 - p.fa * ui) / p.h;
    }
    // Lagrange weights l_j(z) and l_j'(z) by prefix and suffix products carried with
    // their derivatives (exact at the nodes)
    CT suf[D], sufd[D];
    suf[D - 1] = CT(1);
    sufd[D - 1] = CT(0);
#pragma unroll
    for (int j = D - 1; j > 0; --j) {
      sufd[j - 1] = fma(sufd[j], zc - CT(j), suf[j]);
      suf[j - 1] = suf[j] * (zc - CT(j));
    }
    CT l[D], ld[D];
    CT pre = CT(1), pred = CT(0), bound = CT(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const CT c = CT(lagrange_den(D, j));
      l[j] = pre * suf[j] * c;
      ld[j] = fma(pred, suf[j], pre * sufd[j]) * c;
      bound = fma(abs(l[j]), t.rs[j], bound);
      pred = fma(pred, zc - CT(j), pre);
      pre *= zc - CT(j);
    }
    if (!(bound <= CT(16))) {
      st_out[it] = ADJ_MARK;
      atomicAdd(marks, 1);
      continue;
    }
    // g_u = l'(z)^T exp(E) u and g_nu = l(z)^T Dh2 exp(E) u are (first and
    // second) differences of the window's values, far smaller than the values.
    // The first row maps the constant 1 to 0 and the node index q to 1, the
    // second maps both to 0 (exp(E) keeps polynomials of degree 1, Lagrange
    // interpolation reproduces them), so the FP32 form takes both on the
    // residual r_q = (u_q - u_0) - s q of the window's linear interpolant (the
    // difference u_q - u_0 rounds relative to itself), the linear part adding
    // exactly s to g_u: the products then round only the small residual.
    CT u_lin = CT(0), s_lin = CT(0);
    if constexpr (sizeof(CT) == 4) {
      u_lin = CT(ub[grid_index(st, p.N, p.bc)]);
      s_lin = (CT(ub[grid_index(st + D - 1, p.N, p.bc)]) - u_lin) * CT(1.0 / (D - 1));
    }
    CT gu = CT(0), gn = CT(0);
#pragma unroll
    for (int q = 0; q < D; ++q) {
      CT w = CT(0), wu = CT(0), wn = CT(0);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        w = fma(l[j], t.ex[j * D + q], w);
        wu = fma(ld[j], t.ex[j * D + q], wu);
        wn = fma(l[j], t.d2ex[j * D + q], wn);
      }
      const CT uv = CT(ub[grid_index(st + q, p.N, p.bc)]);
      const CT uq = sizeof(CT) == 4 ? fma(-s_lin, CT(q), uv - u_lin) : uv;
      Wout[q * items + it] = ST(CT(e0) * w);
      gu = fma(wu, uq, gu);
      gn = fma(wn, uq, gn);
    }
    st_out[it] = int32_t(st - i);
    if constexpr (sizeof(CT) == 4) {
      gu_out[it] = ST(CT(e0 * su) * (gu + s_lin));
      dnu_acc += double(CT(lam_next[it]) * gn);  // scaled by e0 dt / h^2 below
    } else {
      gu_out[it] = ST(e0 * su * gu);
      dnu_acc = fma(double(lam_next[it]), e0 * (p.dt / (p.h * p.h)) * double(gn), dnu_acc);
    }
  }
  if constexpr (sizeof(ST) == 4) {
    if (dnu_acc != 0.0) dnu_acc *= e0 * (p.dt / (p.h * p.h));
  }
  dnu_acc = warp_sum(dnu_acc);
  if ((threadIdx.x & 31) == 0 && dnu_acc != 0.0) atomicAdd(dnu, dnu_acc);
}

// lam[k] = sum over points i whose window holds k of lam+_i w_i[k - start_i] + lam+_k g_u,k
template <typename ST>
__global__ void k_adjoint_gather(KParams p, const ST* __restrict__ lam_next, const ST* __restrict__ W,
                                 const ST* __restrict__ gu, const int32_t* __restrict__ st_rel,
                                 ST* __restrict__ lam, unsigned* flags) {
  const int n = p.n;
  const bool dir = p.bc == BC_DIRICHLET;
  unsigned bad = 0;
  const int64_t items = p.N * (p.batch > 1 ? p.batch : 1);
  for (int64_t kg = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; kg < items; kg += int64_t(gridDim.x) * blockDim.x) {
    const int64_t base = (kg / p.N) * p.N;  // first point of this instance
    const int64_t k = kg - base;
    ST acc = ST(0);
    for (int d = -(n - 1); d <= n - 1; ++d) {
      int64_t i = k + d;
      if (dir) {
        if (i < 1 || i > p.N - 2) continue;
      } else {
        i = grid_index(i, p.N, BC_PERIODIC);
      }
      const int64_t sti = i + st_rel[base + i];
      int64_t j = k - sti;
      if (!dir) j = grid_index(j, p.N, BC_PERIODIC);
      if (j >= 0 && j < n) acc = fma(lam_next[base + i], W[j * items + base + i], acc);
    }
    if (!dir || (k >= 1 && k <= p.N - 2)) acc = fma(lam_next[kg], gu[kg], acc);
    lam[kg] = acc;
    bad |= !isfinite(double(acc));
  }
  if (bad) atomicOr(flags, 1u);
}

template <int D, typename ST>
cudaError_t run_adjoint(const KParams& p, const void* u, const void* lam_next, void* lam, double* dnu,
                        void* scratch, unsigned* flags, cudaStream_t s, const double* sl) {
  const int64_t items = p.N * (p.batch > 1 ? p.batch : 1);
  // scratch: the rows W[n][items] (row element j of every point together, so
  // that one point per thread stores coalesced), g_u[items], window offsets
  // st[items], then the count of points marked for the Pade derivatives
  ST* W = static_cast<ST*>(scratch);
  ST* gu = W + items * p.n;
  int32_t* st = reinterpret_cast<int32_t*>(gu + items);
  int* marks = reinterpret_cast<int*>(st + items);
  int fix = 0;
  if (sl) {
    cudaError_t em = cudaMemsetAsync(marks, 0, sizeof(int), s);
    if (em != cudaSuccess) return em;
    AdjTab<D, ST> t;
    using TT = typename std::remove_reference<decltype(t.ex[0])>::type;
    for (int e = 0; e < D * D; ++e) t.ex[e] = TT(sl[e]);
    for (int j = 0; j < D; ++j) t.rs[j] = TT(sl[D * D + j]);
    for (int e = 0; e < D * D; ++e) t.d2ex[e] = TT(sl[D * D + D + e]);
    int64_t gf = (items + 4 * 128 - 1) / (4 * 128);  // at least 4 points per thread: the prologue is shared
    if (gf > int64_t(device_info().sms) * 16) gf = int64_t(device_info().sms) * 16;
    k_adjoint_fact<D, ST><<<int(gf), 128, 0, s>>>(p, t, static_cast<const ST*>(u), static_cast<const ST*>(lam_next),
                                                  W, gu, st, dnu, marks);
    cudaError_t ef = cudaGetLastError();
    if (ef != cudaSuccess) return ef;
    fix = 1;
  }
  const size_t smem = DHB + AW * AdjWs<D>::BYTES;
  auto k1 = k_adjoint_points<D, ST>;
  cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, 32 * AW, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = int64_t(device_info().sms) * per_sm;
  const int64_t need = (items + 32 * AW - 1) / (32 * AW);  // chunks of 32 points per warp
  if (need < grid) grid = need;
  k1<<<int(grid), 32 * AW, smem, s>>>(p, static_cast<const ST*>(u), static_cast<const ST*>(lam_next), W, gu, st,
                                      dnu, fix, marks);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int blk = 256;
  int64_t g2 = (items + blk - 1) / blk;
  if (g2 > int64_t(device_info().sms) * 16) g2 = int64_t(device_info().sms) * 16;
  k_adjoint_gather<ST><<<int(g2), blk, 0, s>>>(p, static_cast<const ST*>(lam_next), W, gu, st, static_cast<ST*>(lam),
                                              flags);
  return cudaGetLastError();
}

}  // namespace

size_t adjoint_scratch_bytes(int64_t N, int n, bool mixed) {
  const size_t es = mixed ? 4 : 8;
  return size_t(N) * size_t(n + 1) * es + size_t(N) * 4 + 256;
}

cudaError_t launch_adjoint(const KParams& p, const void* u, const void* lam_next, void* lam, double* dnu,
                           void* scratch, bool mixed, unsigned* flags, cudaStream_t s, const double* sl) {
#define ADJ_CASE(DD)                                                                              \
  case DD:                                                                                        \
    return mixed ? run_adjoint<DD, float>(p, u, lam_next, lam, dnu, scratch, flags, s, sl)        \
                 : run_adjoint<DD, double>(p, u, lam_next, lam, dnu, scratch, flags, s, sl);
  switch (p.n) {
    ADJ_CASE(3)
    ADJ_CASE(5)
    ADJ_CASE(7)
    ADJ_CASE(9)
    ADJ_CASE(11)
    ADJ_CASE(13)
    ADJ_CASE(15)
    default: return cudaErrorInvalidValue;
  }
#undef ADJ_CASE
}

}  // namespace lmep
