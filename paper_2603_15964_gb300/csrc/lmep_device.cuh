// lmep_device.cuh -- device building blocks of the LMEP hot path (sm_103a).
//
// One warp owns one small matrix (dimension d <= 16) in shared memory:
//   * Fornberg derivative weights on the integer window nodes (Sec. 2.1 step 1),
//   * stencil window / harvest row selection (Sec. 2.1 steps 1 and 3),
//   * Pade [m/m] scaling and squaring exp(X) (Sec. 2.1 step 2), with the
//     polynomial products in PT (double, or float for the FP32 form), the
//     denominator solve by Gauss-Jordan elimination with partial pivoting in
//     FP64, and the squaring phase in FP64.
//     Degree: m in {3,5,7,9} when ||X||_1 <= theta_m (Higham 2005,
//     Algorithm 2.3, theta_m of its Table 2.3), else m = 13.  Scaling for
//     m = 13: Al-Mohy & Higham, "A new scaling and squaring algorithm for the
//     matrix exponential", SIMAX 31(3), 2009: s from
//     alpha = min_{p<=5} max(||X^p||^(1/p), ||X^(p+1)||^(1/(p+1))) (their
//     Thm. 4.2; the norms are computed exactly from the powers), plus their
//     correction ell for non-normal X from ||(|X_s|)^27||_1.  The local LMEP
//     operators are nilpotent up to rounding, so alpha << ||X||_1 and s is
//     usually 0.  Because only a few rows of exp(X) are harvested, the last
//     2^b factors of the squaring phase act on those rows only, and with
//     s = 0 a single row is obtained from one transposed solve y^T Q = e_r^T,
//     w = y^T P.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lmep {

constexpr int DMAX = 16;        // largest matrix handled by one warp
constexpr int LD = 17;          // leading dimension of a d x d matrix in shared memory
constexpr int LDG = 2 * DMAX + 1;  // leading dimension of the d x 2d Gauss-Jordan block
constexpr unsigned FULL = 0xffffffffu;

// Backward-error bounds theta_m of Higham (2005), Table 2.3.
constexpr double THETA3 = 1.495585217958292e-2;
constexpr double THETA5 = 2.539398330063230e-1;
constexpr double THETA7 = 9.504178996162932e-1;
constexpr double THETA9 = 2.097847961257068e0;
constexpr double THETA13 = 5.371920351148152e0;

// Coefficient of x^j in the numerator of the [m/m] Pade approximant of e^x,
// normalised to b_0 = 1: b_{j+1} = b_j (m - j) / ((2m - j)(j + 1)).
__host__ __device__ constexpr double pade_b(int m, int j) {
  double b = 1.0;
  for (int t = 0; t < j; ++t) b = b * double(m - t) / (double(2 * m - t) * double(t + 1));
  return b;
}

// 1 / prod_{m != j} (j - m): the denominators of the Lagrange basis on the
// integer nodes 0..n-1.
__host__ __device__ constexpr double lagrange_den(int n, int j) {
  double d = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) d *= double(j - m);
  return 1.0 / d;
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// ---------------------------------------------------------------- Fornberg (a2)
// Weights c[k][j] of d^k/dx^k (k = 0..3) at z from the integer nodes 0..n-1,
// built by adding one node at a time (Fornberg 1988 recursion, in-place form
// with descending derivative order).  Per thread; used once per CTA.
__device__ inline void fornberg_row(double z, int n, double c[4][DMAX]) {
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < DMAX; ++j) c[k][j] = 0.0;
  c[0][0] = 1.0;
  double c1 = 1.0, c4 = -z;
  for (int i = 1; i < n; ++i) {
    const int mn = i < 3 ? i : 3;
    double c2 = 1.0;
    const double c5 = c4;
    c4 = double(i) - z;
    for (int j = 0; j < i; ++j) {
      const double c3 = double(i - j);
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k) c[k][i] = c1 * (k * c[k - 1][i - 1] - c5 * c[k][i - 1]) / c2;
        c[0][i] = -c1 * c5 * c[0][i - 1] / c2;
      }
      for (int k = mn; k >= 1; --k) c[k][j] = (c4 * c[k][j] - k * c[k - 1][j]) / c3;
      c[0][j] = c4 * c[0][j] / c3;
    }
    c1 = c2;
  }
}

// The same recursion on arbitrary distinct nodes xs[0..n-1] (non-uniform
// windows, Sec. 4.3.3): c[k][j] are the weights of d^k/dx^k at z.
__device__ inline void fornberg_row_nodes(double z, const double* xs, int n, double c[4][DMAX]) {
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < DMAX; ++j) c[k][j] = 0.0;
  c[0][0] = 1.0;
  double c1 = 1.0, c4 = xs[0] - z;
  for (int i = 1; i < n; ++i) {
    const int mn = i < 3 ? i : 3;
    double c2 = 1.0;
    const double c5 = c4;
    c4 = xs[i] - z;
    for (int j = 0; j < i; ++j) {
      const double c3 = xs[i] - xs[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k) c[k][i] = c1 * (k * c[k - 1][i - 1] - c5 * c[k][i - 1]) / c2;
        c[0][i] = -c1 * c5 * c[0][i - 1] / c2;
      }
      for (int k = mn; k >= 1; --k) c[k][j] = (c4 * c[k][j] - k * c[k - 1][j]) / c3;
      c[0][j] = c4 * c[0][j] / c3;
    }
    c1 = c2;
  }
}

// Fill Dh[k-1][i*LD + j] = h^k D^(k)[i][j] (k = 1..3) for the uniform window of
// width n in shared memory.  Threads 0..n-1 of the block each build one row.
// Caller synchronises.
__device__ inline void fornberg_block(double* Dh, int n, float* Dhf = nullptr) {
  const int t = threadIdx.x;
  if (t < n) {
    double c[4][DMAX];
    fornberg_row(double(t), n, c);
    for (int k = 1; k <= 3; ++k)
      for (int j = 0; j < n; ++j) {
        Dh[(k - 1) * DMAX * LD + t * LD + j] = c[k][j];
        if (Dhf) Dhf[(k - 1) * DMAX * LD + t * LD + j] = float(c[k][j]);
      }
  }
}

// ---------------------------------------------------------------- stencils (a1)
enum { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_NEUMANN = 2 };

// Window start of point i (global index of window node 0 before wrap or
// reflection) with an upstream shift k; the harvest row is i - start.
__device__ __forceinline__ int64_t window_start(int64_t i, int64_t N, int n, int bc, int k) {
  const int hs = (n - 1) >> 1;
  int64_t s = i - hs - k;
  if (bc == BC_DIRICHLET) s = s < 0 ? 0 : (s > N - n ? N - n : s);
  return s;
}
// Map a possibly out-of-range index to the grid (periodic wrap, even reflection).
__device__ __forceinline__ int64_t grid_index(int64_t q, int64_t N, int bc) {
  if (bc == BC_PERIODIC) {
    // a window (n <= N nodes) wraps at most once; the general remainder (a
    // slow 64-bit division) only runs for indices further away
    if (q >= 0 && q < N) return q;
    if (q < 0 && q >= -N) return q + N;
    if (q >= N && q < 2 * N) return q - N;
    q %= N;
    return q < 0 ? q + N : q;
  }
  if (bc == BC_NEUMANN) {
    if (q < 0) q = -q;
    if (q > N - 1) q = 2 * (N - 1) - q;
    return q;
  }
  return q;
}
// it = b N + i with 0 <= i < N: no division for one instance, a 32-bit one
// when the index fits, the 64-bit division otherwise.
__device__ __forceinline__ void split_index(int64_t it, int64_t N, int64_t batch, int64_t& b, int64_t& i) {
  if (batch <= 1) {
    b = 0;
    i = it;
  } else if (it < (int64_t(1) << 32) && N < (int64_t(1) << 32)) {
    const uint32_t q = uint32_t(it) / uint32_t(N);
    b = q;
    i = it - int64_t(q) * N;
  } else {
    b = it / N;
    i = it - b * N;
  }
}

// Departure-centring shift clamp(floor(u dt / h + 1/2), -hs, hs), evaluated
// with explicitly rounded FP64 operations, (u dt) / h + 1/2, so that the
// integer decision is reproducible bit for bit.  dt_h = dt / h gives a cheap
// estimate first; the exact division runs only when the estimate lies within
// 1e-9 of an integer, where the two roundings could disagree.
// Rare-path helpers kept out of line: inlined, the compiler may turn these
// long FP64 sequences into predicated code that occupies the FP64 pipe on
// every call even when the branch is not taken.
static __device__ __noinline__ double departure_exact(double u, double dt, double h) {
  return __dadd_rn(__ddiv_rn(__dmul_rn(u, dt), h), 0.5);
}
static __device__ __noinline__ double drcp_slow(double x) { return __drcp_rn(x); }

__device__ __forceinline__ int departure_shift(double u, double dt, double h, int n, double dt_h) {
  const int hs = (n - 1) >> 1;
  double t = fma(u, dt_h, 0.5);
  const double f = t - floor(t);
  if (!(f > 1e-9 && f < 1.0 - 1e-9)) t = departure_exact(u, dt, h);
  // fmin/fmax return the non-NaN operand, so a non-finite state still gives a
  // window inside the clamp range (the non-finite result is flagged later).
  const double k = fmax(double(-hs), fmin(double(hs), floor(t)));
  return int(k);
}
// departure_shift of a float state for the FP32 form: the estimate in FP32 (error
// below 4e-7 (|t| + 1) for t = u dt / h + 1/2), the exact FP64 decision when it
// lies within 1e-6 (|t| + 1) of an integer (or is not finite).
template <typename P>
__device__ __forceinline__ int departure_shift_f32(float u, const P& p, int n) {
  const int hs = (n - 1) >> 1;
  const float t = fmaf(u, p.dt_h_f, 0.5f);
  const float f = t - floorf(t);
  const float m = 1e-6f * (fabsf(t) + 1.0f);
  if (!(f > m && f < 1.0f - m)) return departure_shift(double(u), p.dt, p.h, n, p.dt_h);
  return int(fmaxf(float(-hs), fminf(float(hs), floorf(t))));
}

// Exact integer re-centring of an exponential row: row r of exp(X(a)) equals
// row r - k of exp(X(a) + k Dh1) (both evaluate e^{dt L} p at the same
// departure point, Thm. 2).  k is the rounded local Courant number
// -a1 dt / h, kept so that row r - k exists; any k in range gives the same
// row, the rounded one the smallest matrix norm.
__device__ __forceinline__ int recentring_shift(double a1, double dt_h, int n, int r) {
  const double k = fmax(double(r - (n - 1)), fmin(double(r), floor(fma(-a1, dt_h, 0.5))));
  return int(k);
}

// ---------------------------------------------------------------- warp expm (a4)
// Per-warp shared workspace layout (bytes).  Buffers whose lifetimes do not
// overlap share storage, which keeps the workspace small enough for 3 (FP64)
// or 4 (FP32 form) CTAs of 4 warps per SM:
//   X64 | R1   double d x d (LD)    input X; after the Pade products the
//                                   solution R (or P in the one-row solve)
//   PRD | G    5 x PT d x d (LD)    X, X^2, X^4, X^6, temporary; after the
//                                   products the FP64 block [Q | P] (LDG)
//   R2         double d x d (LD)    squaring ping-pong
//   VEC        double 4 x 16        harvested rows
template <typename PT>
struct Ws {
  static constexpr int X64_OFF = 0;
  static constexpr int PRD_OFF = X64_OFF + DMAX * LD * 8;
  static constexpr int LDM = sizeof(PT) == 4 ? 20 : LD;   // row stride of the PT matrices
  static constexpr int PRD_BYTES = 5 * DMAX * LDM * int(sizeof(PT));
  static constexpr int G_BYTES = DMAX * LDG * 8;
  static constexpr int R2_OFF = PRD_OFF + (PRD_BYTES > G_BYTES ? PRD_BYTES : G_BYTES);
  static constexpr int VEC_OFF = R2_OFF + DMAX * LD * 8;
  static constexpr int BYTES = VEC_OFF + 4 * DMAX * 8;
  double* X64;
  PT* P;  // 5 product matrices back to back
  double* G;
  double* R1;
  double* R2;
  double* V;
  __device__ explicit Ws(unsigned char* base)
      : X64(reinterpret_cast<double*>(base + X64_OFF)),
        P(reinterpret_cast<PT*>(base + PRD_OFF)),
        G(reinterpret_cast<double*>(base + PRD_OFF)),
        R1(reinterpret_cast<double*>(base + X64_OFF)),
        R2(reinterpret_cast<double*>(base + R2_OFF)),
        V(reinterpret_cast<double*>(base + VEC_OFF)) {}
  __device__ PT* M(int q) const { return P + q * DMAX * LDM; }
};

// Element slots of a d x d matrix spread over a warp: lane owns e = lane + 32 t.
template <int D>
struct Slots {
  static constexpr int S = (D * D + 31) / 32;
  int i[S], j[S];
  bool ok[S];
  __device__ explicit Slots(int lane) {
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const int e = lane + 32 * t;
      ok[t] = e < D * D;
      i[t] = ok[t] ? e / D : 0;
      j[t] = ok[t] ? e - (e / D) * D : 0;
    }
  }
};

// acc = A B for the lane's slots (A stride LDA, B stride LDB).
template <int D, int LDA, int LDB, typename T>
__device__ __forceinline__ void mm_slots(const T* __restrict__ A, const T* __restrict__ B,
                                         T (&acc)[Slots<D>::S], const Slots<D>& sl) {
  constexpr int S = Slots<D>::S;
#pragma unroll
  for (int t = 0; t < S; ++t) acc[t] = T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int t = 0; t < S; ++t) acc[t] = fma(A[sl.i[t] * LDA + k], B[k * LDB + sl.j[t]], acc[t]);
  }
}

template <int D, typename T>
__device__ __forceinline__ void store_slots(T* __restrict__ C, const T (&v)[Slots<D>::S],
                                            const Slots<D>& sl) {
#pragma unroll
  for (int t = 0; t < Slots<D>::S; ++t)
    if (sl.ok[t]) C[sl.i[t] * LD + sl.j[t]] = v[t];
}

// Per-lane output positions of a D x D product in the Pade phase.
//  * double: the element slots above (lane owns e = lane + 32 t), row stride 17;
//    FP64 products are bound by the FP64 pipe, so padding would only add work.
//  * float: register blocks.  The matrix is padded to DP x DP (DP = 8 or 16);
//    lane l owns rows {rq, rq + DP/RB, ..} (rq = l / 4) and the CB consecutive
//    columns from cq * CB (cq = l % 4).  Per k it loads RB row-broadcast
//    scalars of A and one CB-wide vector of B (row stride 20 floats keeps the
//    vectors 16-byte aligned and the 8 broadcast rows on distinct banks), so a
//    product costs ~4x fewer shared-memory wavefronts than the slot layout.
template <int D, typename PT>
struct Lay;

template <int D>
struct Lay<D, double> {
  static constexpr int N = Slots<D>::S;
  static constexpr int LDM = LD;
  int i[N], j[N];
  bool ok[N];
  __device__ explicit Lay(int lane) {
    const Slots<D> sl(lane);
#pragma unroll
    for (int t = 0; t < N; ++t) {
      i[t] = sl.i[t];
      j[t] = sl.j[t];
      ok[t] = sl.ok[t];
    }
  }
  __device__ __forceinline__ void mm(const double* __restrict__ A, const double* __restrict__ B,
                                     double (&acc)[N]) const {
#pragma unroll
    for (int t = 0; t < N; ++t) acc[t] = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
#pragma unroll
      for (int t = 0; t < N; ++t) acc[t] = fma(A[i[t] * LDM + k], B[k * LDM + j[t]], acc[t]);
    }
  }
};

template <int D>
struct Lay<D, float> {
  static constexpr int DP = D <= 8 ? 8 : 16;
  static constexpr int RB = DP == 8 ? 1 : 2;
  static constexpr int CB = DP == 8 ? 2 : 4;
  static constexpr int RS = DP / RB;  // row stride between a lane's rows (= 8)
  static constexpr int N = RB * CB;
  static constexpr int LDM = 20;
  int rq, cq;
  int i[N], j[N];
  bool ok[N];
  __device__ explicit Lay(int lane) : rq(lane >> 2), cq(lane & 3) {
#pragma unroll
    for (int t = 0; t < N; ++t) {
      i[t] = rq + RS * (t / CB);
      j[t] = cq * CB + (t % CB);
      ok[t] = i[t] < D && j[t] < D;
    }
  }
  __device__ __forceinline__ void mm(const float* __restrict__ A, const float* __restrict__ B,
                                     float (&acc)[N]) const {
#pragma unroll
    for (int t = 0; t < N; ++t) acc[t] = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float a[RB], b[CB];
#pragma unroll
      for (int r = 0; r < RB; ++r) a[r] = A[(rq + RS * r) * LDM + k];
      if constexpr (CB == 4) {
        const float4 v = *reinterpret_cast<const float4*>(B + k * LDM + cq * 4);
        b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
      } else {
        const float2 v = *reinterpret_cast<const float2*>(B + k * LDM + cq * 2);
        b[0] = v.x; b[1] = v.y;
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) acc[r * CB + c] = fmaf(a[r], b[c], acc[r * CB + c]);
    }
  }
};

template <int D, typename T>
__device__ __forceinline__ void lay_store(const Lay<D, T>& L, T* __restrict__ C, const T (&v)[Lay<D, T>::N]) {
#pragma unroll
  for (int t = 0; t < Lay<D, T>::N; ++t)
    if (L.ok[t]) C[L.i[t] * Lay<D, T>::LDM + L.j[t]] = v[t];
}

// v = c0*M0 + c1*M1 + c2*M2 (+ cI on the diagonal) at the lane's positions (add: v += ...).
template <int D, typename T>
__device__ __forceinline__ void lincomb(const Lay<D, T>& L, T (&v)[Lay<D, T>::N], const T* M0, T c0,
                                        const T* M1, T c1, const T* M2, T c2, T cI, bool add) {
#pragma unroll
  for (int t = 0; t < Lay<D, T>::N; ++t) {
    const int o = L.i[t] * Lay<D, T>::LDM + L.j[t];
    T x = add ? v[t] : T(0);
    if (M0) x = fma(c0, M0[o], x);
    if (M1) x = fma(c1, M1[o], x);
    if (M2) x = fma(c2, M2[o], x);
    if (L.i[t] == L.j[t]) x += cI;
    v[t] = x;
  }
}

// Odd part U and even part V of p_m(X) at the lane's positions; X is PRD slot
// 0 and X^2, X^4, X^6 (as far as m needs them) are in slots 1..3.  Products
// follow Higham (2005) eqs. (2.10)-(2.11); the degree only changes which
// powers exist and which coefficients multiply them, so every degree shares
// the same product call sites.  Uses PRD slot 4 and the R2 buffer as scratch.
template <int D, typename PT>
__device__ __forceinline__ void pade_uv(const Ws<PT>& w, int m, const Lay<D, PT>& L, PT (&U)[Lay<D, PT>::N],
                                        PT (&V)[Lay<D, PT>::N]) {
  constexpr int N = Lay<D, PT>::N;
  PT* X = w.M(0);
  PT* A2 = w.M(1);
  PT* A4 = w.M(2);
  PT* A6 = w.M(3);
  PT* T = w.M(4);
  PT* T2 = reinterpret_cast<PT*>(w.R2);
  PT acc[N], A8[N];
  PT b[14];
#pragma unroll
  for (int j = 0; j < 14; ++j) b[j] = PT(0);
  switch (m) {
    case 3:
#pragma unroll
      for (int j = 0; j <= 3; ++j) b[j] = PT(pade_b(3, j));
      break;
    case 5:
#pragma unroll
      for (int j = 0; j <= 5; ++j) b[j] = PT(pade_b(5, j));
      break;
    case 7:
#pragma unroll
      for (int j = 0; j <= 7; ++j) b[j] = PT(pade_b(7, j));
      break;
    case 9:
#pragma unroll
      for (int j = 0; j <= 9; ++j) b[j] = PT(pade_b(9, j));
      break;
    default:
#pragma unroll
      for (int j = 0; j <= 13; ++j) b[j] = PT(pade_b(13, j));
  }
  if (m == 13) {
    // U-inner = A6 (b13 A6 + b11 A4 + b9 A2) + b7 A6 + b5 A4 + b3 A2 + b1 I
    // V       = A6 (b12 A6 + b10 A4 + b8 A2) + b6 A6 + b4 A4 + b2 A2 + b0 I
    lincomb<D>(L, acc, A6, b[13], A4, b[11], A2, b[9], PT(0), false);
    lay_store<D>(L, T, acc);
    lincomb<D>(L, acc, A6, b[12], A4, b[10], A2, b[8], PT(0), false);
    lay_store<D>(L, T2, acc);
    __syncwarp();
    L.mm(A6, T, acc);
    lincomb<D>(L, acc, A6, b[7], A4, b[5], A2, b[3], b[1], true);
    L.mm(A6, T2, V);
    lincomb<D>(L, V, A6, b[6], A4, b[4], A2, b[2], b[0], true);
    __syncwarp();
    lay_store<D>(L, T, acc);  // U-inner for the last product
  } else {
    const PT* P2 = A2;
    const PT* P4 = m >= 5 ? A4 : nullptr;
    const PT* P6 = m >= 7 ? A6 : nullptr;
    if (m == 9) L.mm(A6, A2, A8);
    lincomb<D>(L, acc, P6, b[7], P4, b[5], P2, b[3], b[1], false);
    lincomb<D>(L, V, P6, b[6], P4, b[4], P2, b[2], b[0], false);
    if (m == 9) {
#pragma unroll
      for (int t = 0; t < N; ++t) {
        acc[t] = fma(b[9], A8[t], acc[t]);
        V[t] = fma(b[8], A8[t], V[t]);
      }
    }
    lay_store<D>(L, T, acc);
  }
  __syncwarp();
  L.mm(X, T, U);
  __syncwarp();
}

// 1/x by Newton-Raphson for the reciprocal, r <- r + r (1 - x r), from an FP32
// seed (__frcp_rn of x rounded to 20 mantissa bits, relative error < 2^-19):
// each step squares the relative error, so two steps reach the FP64 rounding
// level; one step (relative error < 2^-38) is used for the FP32 form, whose
// inputs carry FP32 rounding errors five orders of magnitude larger.  The float <-> double conversions act on the bit patterns (exact for
// the seed), so only the four Newton FMAs use the FP64 pipe.  Outside the
// normal float range the correctly rounded __drcp_rn is used instead.
template <int STEPS>
__device__ __forceinline__ double recip_nr(double x) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (e <= 1 || e >= 253) return drcp_slow(x);
  const float xf = __int_as_float((hi & int(0x80000000)) | (e << 23) | ((hi & 0xfffff) << 3));
  const int rb = __float_as_int(__frcp_rn(xf));
  const int re = ((rb >> 23) & 0xff) - 127 + 1023;
  double r = __hiloint2double((rb & int(0x80000000)) | (re << 20) | ((rb & 0x7fffff) >> 3), (rb & 7) << 29);
#pragma unroll
  for (int it = 0; it < STEPS; ++it) r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// Solve Q R = P in place on G = [Q | P] (NC = D + number of right-hand
// sides <= 32 columns) by Gauss-Jordan elimination with partial pivoting
// (FP64).  On return G[:, D:NC] holds R.  Pivot magnitudes are compared as
// IEEE bit patterns (monotonic for non-negative doubles).  The step loop is
// unrolled, so every step's element count and index divisions are constants
// and each step issues exactly ceil((D - 1)(NC - k - 1) / 32) FP64 FMAs.
template <int D, int NEWTON, int NC>
__device__ void gauss_jordan(double* G, int lane) {
  static_assert(NC <= 32, "one column per lane for swaps and scaling");
#pragma unroll
  for (int k = 0; k < D; ++k) {
    long long key = -1;
    int idx = k;
    if (lane >= k && lane < D) {
      key = __double_as_longlong(G[lane * LDG + k]) & 0x7fffffffffffffffll;
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
    if (idx != k && k + lane < NC) {
      const int j = k + lane;
      const double a = G[k * LDG + j];
      G[k * LDG + j] = G[idx * LDG + j];
      G[idx * LDG + j] = a;
    }
    __syncwarp();
    const double inv = recip_nr<NEWTON>(G[k * LDG + k]);
    if (k + 1 + lane < NC) G[k * LDG + k + 1 + lane] *= inv;
    __syncwarp();
    const int nc = NC - k - 1;
    const int tot = (D - 1) * nc;
#pragma unroll
    for (int q = 0; q < (tot + 31) / 32; ++q) {
      const int e = lane + 32 * q;
      if (e < tot) {
        const int ii = e / nc;
        const int i = ii + (ii >= k ? 1 : 0);
        const int j = k + 1 + (e - ii * nc);
        G[i * LDG + j] = fma(-G[i * LDG + k], G[k * LDG + j], G[i * LDG + j]);
      }
    }
    __syncwarp();
  }
}

// Row-vector phase: V[q][:] <- V[q][:] * R, nrows rows, FP64.  R has stride ldr.
template <int D>
__device__ __forceinline__ void rows_times(double* V, const double* R, int ldr, int nrows, int lane) {
  if (nrows == 1) {
    // split the k-sum over the two half-warps, then combine with one shuffle
    constexpr int K0 = (D + 1) / 2;
    const int j = lane & 15, half = lane >> 4;
    double acc = 0.0;
    if (j < D) {
      if (half == 0) {
#pragma unroll
        for (int k = 0; k < K0; ++k) acc = fma(V[k], R[k * ldr + j], acc);
      } else {
#pragma unroll
        for (int k = K0; k < D; ++k) acc = fma(V[k], R[k * ldr + j], acc);
      }
    }
    acc += __shfl_xor_sync(FULL, acc, 16);
    __syncwarp();
    if (half == 0 && j < D) V[j] = acc;
    __syncwarp();
    return;
  }
  double res[2] = {0.0, 0.0};
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int o = lane + 32 * p;
    if (o < nrows * D) {
      const int q = o / D, j = o - (o / D) * D;
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fma(V[q * DMAX + k], R[k * ldr + j], acc);
      res[p] = acc;
    }
  }
  __syncwarp();
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int o = lane + 32 * p;
    if (o < nrows * D) V[(o / D) * DMAX + (o - (o / D) * D)] = res[p];
  }
  __syncwarp();
}

// float -> double with integer operations only (exact): the FP64 pipe, which
// also executes the hardware conversion, stays free.  Zero, subnormal, Inf
// and NaN inputs take the hardware conversion.
__device__ __forceinline__ double f2d_bits(float f) {
  const int b = __float_as_int(f);
  const int e = (b >> 23) & 0xff;
  if (e == 0 || e == 0xff) {
    if ((b & 0x7fffffff) == 0) return __hiloint2double(b & int(0x80000000), 0);
    return double(f);
  }
  return __hiloint2double((b & int(0x80000000)) | ((e + 896) << 20) | ((b & 0x7fffff) >> 3), (b & 7) << 29);
}

// X = cI I + c1h Dh1 + c2h Dh2 + c3h Dh3 on the n x n window (zero-padded to
// D) from the window's derivative matrices Dh (stride LD, DMAX rows per
// order), in FP64 and, for the FP32 form, directly in FP32 from an FP32 copy
// of Dh.  The FP32 form assembles X in FP32 and needs the FP64 matrix only
// to settle a Pade degree next to a threshold.
struct Asm {
  const double* Dh;
  const float* Dhf;
  int n;
  double cI, c1h, c2h, c3h;
  float cIf, c1f, c2f, c3f;
};

template <int D>
__device__ __forceinline__ void assemble64(double* X64, const Asm& a, int lane) {
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e - (e / D) * D;
    double x = 0.0;
    if (i < a.n && j < a.n) {
      const int o = i * LD + j;
      x = a.c1h * a.Dh[o];
      x = fma(a.c2h, a.Dh[DMAX * LD + o], x);
      if (a.c3h != 0.0) x = fma(a.c3h, a.Dh[2 * DMAX * LD + o], x);
      if (i == j) x += a.cI;
    }
    X64[i * LD + j] = x;
  }
}

// |x| as a float from the top word of a double with integer operations only
// (exponent rebias, mantissa truncated to 20 bits; relative error < 2^-20).
// Used where only a magnitude estimate is needed, to keep the FP64 pipe free.
__device__ __forceinline__ float approx_abs_f32(double x) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __int_as_float(0x7f800000);
  return __int_as_float((e << 23) | ((hi & 0xfffff) << 3));
}
__device__ __forceinline__ float approx_abs_f32(float x) { return fabsf(x); }
// x as a float with integer operations only (mantissa truncated to 20 bits,
// relative error < 2^-20; underflow to zero, overflow to Inf).  For estimates.
__device__ __forceinline__ float approx_f32(double x) {
  const int hi = __double2hiint(x);
  const int sg = hi & int(0x80000000);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __int_as_float(sg);
  if (e >= 255) return __int_as_float(sg | 0x7f800000);
  return __int_as_float(sg | (e << 23) | ((hi & 0xfffff) << 3));
}

// 1-norm (max column sum) of a D x D matrix in shared memory, all lanes.
template <int D, typename T>
__device__ __forceinline__ double norm1_smem(const T* M, int lane) {
  double cs = 0.0;
  if (lane < D) {
#pragma unroll
    for (int i = 0; i < D; ++i) cs += fabs(double(M[i * LD + lane]));
  }
  return warp_max(cs);
}

// Powers X^2, X^4, X^6 into PRD slots 1..3 (PT) from X in slot 0, degree m
// and scaling s.  m = 13 uses the Al-Mohy & Higham (2009) choice of s (see the
// file header); the powers are then scaled by exact powers of two.
template <int D, typename PT>
__device__ void powers_and_scaling(const Ws<PT>& w, const Lay<D, PT>& L, int lane, double nrm, float nrmf,
                                   bool exact64, int& m, int& s) {
  constexpr int S = Lay<D, PT>::N;
  constexpr int LM = Lay<D, PT>::LDM;
  PT* X = w.M(0);
  PT* A2 = w.M(1);
  PT* A4 = w.M(2);
  PT* A6 = w.M(3);
  PT* T = w.M(4);
  PT acc[S];
  s = 0;
  // The FP32 form decides on its FP32 norm (at least 1e-4 relative away from
  // every threshold, so the decision equals the FP64 one); exact64 marks an
  // FP64 norm, compared in FP64.
  const bool f32dec = sizeof(PT) == 4 && !exact64;
  if (f32dec) {
    if (nrmf <= float(THETA3)) m = 3;
    else if (nrmf <= float(THETA5)) m = 5;
    else if (nrmf <= float(THETA7)) m = 7;
    else if (nrmf <= float(THETA9)) m = 9;
    else m = 13;
  } else {
    if (nrm <= THETA3) m = 3;
    else if (nrm <= THETA5) m = 5;
    else if (nrm <= THETA7) m = 7;
    else if (nrm <= THETA9) m = 9;
    else m = 13;
  }
  // Norms of powers overflow FP32 for very large ||X||: there, and for
  // non-finite input, scale by the norm first (Higham 2005) and stop.
  const bool by_norm = m == 13 && (f32dec ? !(nrmf <= 8192.0f) : !(nrm <= 8192.0));
  if (by_norm) {
    double t = f32dec ? double(nrmf) : nrm;
    while (t > THETA13 && s < 1023) { t *= 0.5; ++s; }
    const PT sc = PT(ldexp(1.0, -s));
#pragma unroll
    for (int q = 0; q < S; ++q)
      if (L.ok[q]) X[L.i[q] * LM + L.j[q]] *= sc;
    __syncwarp();
  }
  L.mm(X, X, acc);
  lay_store<D>(L, A2, acc);
  __syncwarp();
  if (m >= 5) {
    L.mm(A2, A2, acc);
    lay_store<D>(L, A4, acc);
    __syncwarp();
  }
  if (m >= 7) {
    L.mm(A4, A2, acc);
    lay_store<D>(L, A6, acc);
    __syncwarp();
  }
  if (m != 13 || by_norm) return;
  // ||X||_1 <= theta_13 needs no squaring: alpha <= ||X||_1 (d_p <= ||X||_1 by
  // submultiplicativity) gives s0 = 0, and ||(|X|)^27||_1 <= ||X||_1^27 bounds
  // the ell term by |c27| ||X||_1^26 <= 2^-53 for ||X||_1 <= 5.43 > theta_13,
  // so ell = 0.  Only larger norms need the powers' norms and the ell estimate.
  if (f32dec ? nrmf <= float(THETA13) : nrm <= THETA13) return;
  // log2 d_p = log2 ||X^p|| / p, p = 1..6, with X^3 = X^2 X (into T) and
  // X^5 = X^4 X (into the R2 buffer, free at this point).  Only the exponent
  // of alpha matters, so the arithmetic is FP32 (the estimate is inflated by
  // 2^-12 to stay an upper bound); the six column-sum maxima are reduced
  // together.
  PT* A5 = reinterpret_cast<PT*>(w.R2);
  float cs[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if constexpr (sizeof(PT) == 8) {
    // FP64 path: the two odd powers only feed these norm estimates, so they
    // are formed in FP32 from FP32 copies of X, X^2 and X^4 (slot 4 and R2,
    // which are contiguous, hold the copies; R1 holds X^3; X^5 overwrites the
    // X^2 copy) and the FP64 pipe is spared two products.
    static_assert(Ws<double>::R2_OFF == Ws<double>::PRD_OFF + 5 * DMAX * LD * 8, "slot 4 and R2 adjoin");
    const Lay<D, float> LQ(lane);
    constexpr int LQM = Lay<D, float>::LDM;
    constexpr int NQ = Lay<D, float>::N;
    float* Xf = reinterpret_cast<float*>(T);
    float* A2f = Xf + DMAX * LQM;
    float* A4f = A2f + DMAX * LQM;
    float* A3f = reinterpret_cast<float*>(w.R1);
    for (int e = lane; e < D * D; e += 32) {
      const int i = e / D, j = e - (e / D) * D;
      Xf[i * LQM + j] = approx_f32(X[i * LM + j]);
      A2f[i * LQM + j] = approx_f32(A2[i * LM + j]);
      A4f[i * LQM + j] = approx_f32(A4[i * LM + j]);
    }
    __syncwarp();
    float q[NQ];
    LQ.mm(A2f, Xf, q);
    lay_store<D>(LQ, A3f, q);
    LQ.mm(A4f, Xf, q);
    __syncwarp();
    lay_store<D>(LQ, A2f, q);  // X^5
    __syncwarp();
    if (lane < D) {
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const int o = i * LM + lane, of = i * LQM + lane;
        cs[2] += approx_abs_f32(A2[o]);
        cs[3] += fabsf(A3f[of]);
        cs[4] += approx_abs_f32(A4[o]);
        cs[5] += fabsf(A2f[of]);
        cs[6] += approx_abs_f32(A6[o]);
      }
    }
  } else {
    L.mm(A2, X, acc);
    lay_store<D>(L, T, acc);
    L.mm(A4, X, acc);
    lay_store<D>(L, A5, acc);
    __syncwarp();
    if (lane < D) {
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const int o = i * LM + lane;
        cs[2] += approx_abs_f32(A2[o]);
        cs[3] += approx_abs_f32(T[o]);
        cs[4] += approx_abs_f32(A4[o]);
        cs[5] += approx_abs_f32(A5[o]);
        cs[6] += approx_abs_f32(A6[o]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
#pragma unroll
    for (int p = 2; p <= 6; ++p) cs[p] = fmaxf(cs[p], __shfl_xor_sync(FULL, cs[p], o));
  }
  float lg[7];
  lg[1] = log2f(sizeof(PT) == 4 ? nrmf : float(nrm));
#pragma unroll
  for (int p = 2; p <= 6; ++p) lg[p] = log2f(cs[p]) / float(p);
  float la = lg[1];  // log2 alpha = min_p max(lg_p, lg_{p+1})
#pragma unroll
  for (int p = 1; p <= 5; ++p) la = fminf(la, fmaxf(lg[p], lg[p + 1]));
  la += 1.0f / 4096.0f;
  const float lt = 2.425436f;  // log2(theta_13) rounded down
  int s0 = la > lt ? int(ceilf(la - lt)) : 0;
  // ell: log2 ||(|X|)^27||_1 = log2 max_j (1^T |X|^27)_j.  With Y = |X| / ||X||_1
  // (so that nothing overflows), 1^T Y^27 = ((1^T (Y^4)^6) Y^2) Y: two FP32
  // products (Y^2, Y^4 of a nonnegative matrix, no cancellation) and eight
  // renormalised row-vector steps.  Lane j keeps column j of the current
  // matrix in registers; the vector is broadcast through shared memory.
  __syncwarp();
  // Always FP32 (an exponent estimate), in the FP32 register-block layout, in
  // buffers that are free at this point (X^3, X^5 and the double input).
  const Lay<D, float> LF(lane);
  constexpr int LMF = Lay<D, float>::LDM;
  constexpr int NF = Lay<D, float>::N;
  float* Y = reinterpret_cast<float*>(T);
  float* Y2 = reinterpret_cast<float*>(A5);
  float* Y4 = reinterpret_cast<float*>(w.R1);
  {
    const float sc = 1.0f / (sizeof(PT) == 4 ? nrmf : float(nrm));
#pragma unroll
    for (int q = 0; q < NF; ++q)
      if (LF.ok[q]) Y[LF.i[q] * LMF + LF.j[q]] = approx_abs_f32(X[LF.i[q] * LM + LF.j[q]]) * sc;
  }
  __syncwarp();
  float accf[NF];
  LF.mm(Y, Y, accf);
  lay_store<D>(LF, Y2, accf);
  __syncwarp();
  LF.mm(Y2, Y2, accf);
  lay_store<D>(LF, Y4, accf);
  __syncwarp();
  float* vs = reinterpret_cast<float*>(w.V);
  if (lane < D) vs[lane] = 1.0f;
  __syncwarp();
  float l27 = 27.0f * lg[1];
  // Column `lane` of Y^4 stays in registers for its six steps.  Every column
  // sum of Y is at most 1, so the iterates never grow; they are renormalised
  // after every second step only.  Two unnormalised steps shrink the vector
  // by at most ||Y^8||_1: if that underflows, ||Y^27||_1 < 2^-378 and ell is 0
  // for every norm this branch sees (||X||_1 <= 8192), which is what a zero
  // maximum reports below.
  float y4c[D];
#pragma unroll
  for (int k = 0; k < D; ++k) y4c[k] = lane < D ? Y4[k * LMF + lane] : 0.0f;
  for (int it = 0; it < 8; ++it) {
    const float* M = it == 6 ? Y2 : Y;
    float a0 = 0.0f, a1 = 0.0f;
    if (it < 6) {
#pragma unroll
      for (int k = 0; k < D; k += 2) {
        a0 = fmaf(vs[k], y4c[k], a0);
        if (k + 1 < D) a1 = fmaf(vs[k + 1], y4c[k + 1], a1);
      }
    } else {
#pragma unroll
      for (int k = 0; k < D; k += 2) {
        a0 = fmaf(vs[k], lane < D ? M[k * LMF + lane] : 0.0f, a0);
        if (k + 1 < D) a1 = fmaf(vs[k + 1], lane < D ? M[(k + 1) * LMF + lane] : 0.0f, a1);
      }
    }
    float vj = a0 + a1;
    if (it & 1) {
      float mx = vj;
#pragma unroll
      for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
      if (!(mx > 0.0f)) { l27 = -1e30f; break; }
      l27 += log2f(mx);
      vj *= __frcp_rn(mx);
    }
    __syncwarp();
    if (lane < D) vs[lane] = vj;
    __syncwarp();
  }
  // ell = max(0, ceil(log2(|c27| ||(|X_s|)^27|| / ||X_s|| / u) / 26)), u = 2^-53
  constexpr float LOG2_C27 = -116.447f;  // log2((13!)^2 / (26! 27!))
  const float la27 = LOG2_C27 + l27 - 27.0f * float(s0) - (lg[1] - float(s0));
  int ell = int(ceilf((la27 + 53.0f) / 26.0f));
  if (!(ell > 0)) ell = 0;
  s = s0 + ell;
  if (s > 0) {
    PT c1, c2, c4, c6;
    if constexpr (sizeof(PT) == 4) {
      c1 = ldexpf(1.0f, -s);
      c2 = ldexpf(1.0f, -2 * s);
      c4 = ldexpf(1.0f, -4 * s);
      c6 = ldexpf(1.0f, -6 * s);
    } else {
      c1 = ldexp(1.0, -s);
      c2 = ldexp(1.0, -2 * s);
      c4 = ldexp(1.0, -4 * s);
      c6 = ldexp(1.0, -6 * s);
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
      if (L.ok[q]) {
        const int o = L.i[q] * LM + L.j[q];
        X[o] *= c1;
        A2[o] *= c2;
        A4[o] *= c4;
        A6[o] *= c6;
      }
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------- finite series (a4)
// Without the identity term the local matrix X = c1h Dh1 + c2h Dh2 + c3h Dh3
// is a polynomial without constant term in the differentiation matrix of the
// window's interpolating polynomial (degree < n, Sec. 2): X^n = 0, and a row
// of its exponential is the finite sum
//   e_r^T exp(X) = sum_{k < n} e_r^T X^k / k!
// exactly: n - 2 vector-matrix products instead of the Pade products, the
// solve and the squarings.  In floating point the terms can cancel (a large
// ||X|| with a row of order one); the computed row then differs from the exact
// one by about u * beta, beta = sum_k ||e_r^T |X|^k||_1 / k! (u the unit
// roundoff of PT), which is accumulated in FP32 next to the series and
// returned.  The caller keeps the row when beta is small and otherwise falls
// back to Pade scaling and squaring.
//
// Several points run side by side in one warp, GS lanes each (a group of
// aligned lanes; column j = lane % GS of the group's point, j < n holds column
// j of X in registers).  The row vector is broadcast through the group's
// ping-pong buffers (VPP PT / WPP floats apart, 16-byte aligned, read back
// with 16-byte loads), so that one __syncwarp per term orders their reuse.  The FP32 form runs two FMA chains
// per term (latency); the FP64 path one (the FP64 pipe is the limit).  `row`
// receives element j of the row (0 for j >= n); the cI term is not included
// (it factors out as e^cI).  All lanes of the warp must call this together.
// Sum over the GS aligned lanes of a group; every lane of the group receives
// the same value (each butterfly stage adds the same two operands on both sides).
template <int GS, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = GS / 2; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// |x| of a column entry for the bound: free in FP32 (an operand modifier), an
// integer-only truncation for doubles (keeps the FP64 pipe free).
template <typename PT>
struct AbsCol {
  float a;
  __device__ __forceinline__ void set(PT x) {
    if constexpr (sizeof(PT) == 8) a = approx_abs_f32(x);
  }
  __device__ __forceinline__ float get(PT x) const {
    if constexpr (sizeof(PT) == 8) return a;
    else return fabsf(x);
  }
};

template <int D, typename PT, int GS, int VPP, int WPP>
__device__ __forceinline__ float group_series_row(const Asm& as, int j, int r, PT* vb, float* wb, PT& row) {
  constexpr bool F32 = sizeof(PT) == 4;
  static_assert(D <= GS && GS % 4 == 0, "one lane per column; whole float4 / double2 broadcasts");
  constexpr int VW = F32 ? 4 : 2;  // PT entries per 16-byte broadcast load
  PT x[D];
  AbsCol<PT> ax[D];
  const bool col = j < as.n;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    PT v = PT(0);
    if (col && i < as.n) {
      const int o = i * LD + j;
      if constexpr (F32) {
        v = as.c1f * as.Dhf[o];
        v = fmaf(as.c2f, as.Dhf[DMAX * LD + o], v);
        v = fmaf(as.c3f, as.Dhf[2 * DMAX * LD + o], v);
      } else {
        v = as.c1h * as.Dh[o];
        v = fma(as.c2h, as.Dh[DMAX * LD + o], v);
        if (as.c3h != 0.0) v = fma(as.c3h, as.Dh[2 * DMAX * LD + o], v);
      }
    }
    x[i] = v;
    ax[i].set(v);
  }
  // k = 1: row r of X
  PT v = PT(0);
  float wv = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i)
    if (i == r) {
      v = x[i];
      wv = ax[i].get(x[i]);
    }
  PT acc = (j == r ? PT(1) : PT(0)) + v;
  float sw = wv;
#pragma unroll
  for (int k = 2; k < D; ++k) {
    PT* vk = vb + (k & 1) * VPP;
    float* wk = wb + (k & 1) * WPP;
    vk[j] = v;
    wk[j] = wv;
    __syncwarp();
    PT s0 = PT(0), s1 = PT(0);
    float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
    for (int q = 0; q < (D + VW - 1) / VW; ++q) {
      PT vv[VW];
      if constexpr (F32) {
        const float4 t = reinterpret_cast<const float4*>(vk)[q];
        vv[0] = t.x; vv[1] = t.y; vv[2] = t.z; vv[3] = t.w;
      } else {
        const double2 t = reinterpret_cast<const double2*>(vk)[q];
        vv[0] = t.x; vv[1] = t.y;
      }
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int i = q * VW + e;
        if (i < D) {
          if (F32 && (i & 1)) s1 = fma(vv[e], x[i], s1);
          else s0 = fma(vv[e], x[i], s0);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < (D + 3) / 4; ++q) {
      const float4 t = reinterpret_cast<const float4*>(wk)[q];
      const float ww[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * q + e;
        if (i < D) {
          if (i & 1) t1 = fmaf(ww[e], ax[i].get(x[i]), t1);
          else t0 = fmaf(ww[e], ax[i].get(x[i]), t0);
        }
      }
    }
    v = (F32 ? s0 + s1 : s0) * PT(1.0 / double(k));
    wv = (t0 + t1) * float(1.0 / double(k));
    acc += v;
    sw += wv;
  }
  row = acc;
  const float beta = 1.0f + group_sum<GS>(sw);
  __syncwarp();  // the buffers are free for the caller
  return beta;
}

// exp(X) for X = w.X64 (D x D, double).  Writes the harvested rows
// rows[0..nrows) into w.V[q*DMAX + j] (double) when full == false, or the
// whole exponential into E (stride lde) when full == true.  m_out, s_out and
// a_out receive the Pade degree, the squarings and the full squarings.
template <int D, typename PT>
__device__ __noinline__ void warp_expm(const Ws<PT>& w, int lane, const int* rows, int nrows, bool full,
                                       double* E, int lde, int* m_out, int* s_out, int* a_out = nullptr,
                                       const Asm* as = nullptr) {
  constexpr int S = Slots<D>::S;
  constexpr int NL = Lay<D, PT>::N;
  constexpr int LM = Lay<D, PT>::LDM;
  const Slots<D> sl(lane);
  const Lay<D, PT> L(lane);
  constexpr bool F32 = sizeof(PT) == 4;
  // ||X||_1 picks the Pade degree.  The FP32 form estimates it in FP32 and
  // falls back to the FP64 sum only next to a threshold, where the estimate
  // (relative error below 1e-5) could pick another degree.  With an
  // assembly descriptor the FP32 form builds X in FP32 directly and the FP64
  // matrix only for that fallback.
  PT* X = w.M(0);
  double nrm = 0.0;
  float nrmf = 0.0f;
  bool exact64 = !F32;
  if (F32) {
    if (as) {
      const float* Df = as->Dhf;
#pragma unroll
      for (int t = 0; t < NL; ++t) {
        if (L.ok[t]) {
          const int i = L.i[t], j = L.j[t];
          float x = 0.0f;
          if (i < as->n && j < as->n) {
            const int o = i * LD + j;
            x = as->c1f * Df[o];
            x = fmaf(as->c2f, Df[DMAX * LD + o], x);
            x = fmaf(as->c3f, Df[2 * DMAX * LD + o], x);
            if (i == j) x += as->cIf;
          }
          X[i * LM + j] = PT(x);
        }
      }
      __syncwarp();
    }
    float cs = 0.0f;
    if (lane < D) {
#pragma unroll
      for (int i = 0; i < D; ++i) cs += as ? fabsf(float(X[i * LM + lane])) : approx_abs_f32(w.X64[i * LD + lane]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) cs = fmaxf(cs, __shfl_xor_sync(FULL, cs, o));
    nrmf = cs;
    const float th[6] = {float(THETA3), float(THETA5), float(THETA7), float(THETA9), float(THETA13), 8192.0f};
    bool near = !(cs > 0.0f) || !(cs < 3.0e38f);
#pragma unroll
    for (int q = 0; q < 6; ++q) near |= fabsf(cs - th[q]) <= 1e-4f * th[q];
    if (near) {
      if (as) {
        assemble64<D>(w.X64, *as, lane);
        __syncwarp();
      }
      nrm = norm1_smem<D>(w.X64, lane);
      nrmf = float(nrm);
      exact64 = true;
    }
  } else {
    nrm = norm1_smem<D>(w.X64, lane);
  }
  if (!(F32 && as)) {
#pragma unroll
    for (int t = 0; t < NL; ++t)
      if (L.ok[t]) X[L.i[t] * LM + L.j[t]] = PT(w.X64[L.i[t] * LD + L.j[t]]);
  }
  __syncwarp();
  int m, s;
  powers_and_scaling<D, PT>(w, L, lane, nrm, nrmf, exact64, m, s);
  PT U[NL], V[NL];
  pade_uv<D, PT>(w, m, L, U, V);
  int a = s;
  if (!full && s == 0 && nrows == 1) {
    // one row of Q^-1 P: y^T Q = e_r^T (Gauss-Jordan on [Q^T | e_r]), w = y^T P.
    // Q = V - U is formed exactly in FP64.  In the FP32 form the numerator
    // P = V + U and the product y^T P stay FP32 (FP32 accumulation).
    PT* Pm = reinterpret_cast<PT*>(w.R1);
#pragma unroll
    for (int t = 0; t < NL; ++t) {
      if (L.ok[t]) {
        double u, v;
        if constexpr (F32) {
          u = f2d_bits(U[t]);
          v = f2d_bits(V[t]);
        } else {
          u = U[t];
          v = V[t];
        }
        w.G[L.j[t] * LDG + L.i[t]] = v - u;
        if (F32) Pm[L.i[t] * LM + L.j[t]] = V[t] + U[t];
        else w.R1[L.i[t] * LD + L.j[t]] = v + u;
      }
    }
    if (lane < D) w.G[lane * LDG + D] = lane == rows[0] ? 1.0 : 0.0;
    __syncwarp();
    gauss_jordan<D, F32 ? 1 : 2, D + 1>(w.G, lane);
    if (F32) {
      float* ys = reinterpret_cast<float*>(w.V) + 2 * DMAX;
      if (lane < D) ys[lane] = float(w.G[lane * LDG + D]);
      __syncwarp();
      constexpr int K0 = (D + 1) / 2;
      const int j = lane & 15, half = lane >> 4;
      float acc = 0.0f;
      if (j < D) {
        if (half == 0) {
#pragma unroll
          for (int k = 0; k < K0; ++k) acc = fmaf(ys[k], float(Pm[k * LM + j]), acc);
        } else {
#pragma unroll
          for (int k = K0; k < D; ++k) acc = fmaf(ys[k], float(Pm[k * LM + j]), acc);
        }
      }
      acc += __shfl_xor_sync(FULL, acc, 16);
      __syncwarp();
      if (half == 0 && j < D) w.V[j] = double(acc);
      __syncwarp();
    } else {
      if (lane < D) w.V[lane] = w.G[lane * LDG + D];
      __syncwarp();
      rows_times<D>(w.V, w.R1, LD, 1, lane);
    }
    a = 0;
  } else {
    // [Q | P] = [V - U | V + U] in FP64
#pragma unroll
    for (int t = 0; t < NL; ++t) {
      if (L.ok[t]) {
        double u, v;
        if constexpr (F32) {
          u = f2d_bits(U[t]);
          v = f2d_bits(V[t]);
        } else {
          u = U[t];
          v = V[t];
        }
        w.G[L.i[t] * LDG + L.j[t]] = v - u;
        w.G[L.i[t] * LDG + D + L.j[t]] = v + u;
      }
    }
    __syncwarp();
    gauss_jordan<D, 2, 2 * D>(w.G, lane);
    // squaring phase in FP64: R = G[:, D:2D] copied to R1, full squarings
    // ping-pong between R1 and R2, then the remaining 2^b factors act on the
    // harvested rows only.
#pragma unroll
    for (int t = 0; t < S; ++t)
      if (sl.ok[t]) w.R1[sl.i[t] * LD + sl.j[t]] = w.G[sl.i[t] * LDG + D + sl.j[t]];
    __syncwarp();
    if (!full) {
      // a full squarings + 2^(s-a) - 1 row products, minimising FP64 instructions;
      // at most 2^6 - 1 row products, larger s always squares in full
      const int cost_full = S * D;
      const int cost_vec = nrows == 1 ? (D + 1) / 2 + 1 : D * ((nrows * D + 31) / 32);
      int best = 1 << 30;
      for (int aa = (s > 6 ? s - 6 : 0); aa <= s; ++aa) {
        const int c = aa * cost_full + ((1 << (s - aa)) - 1) * cost_vec;
        if (c < best) { best = c; a = aa; }
      }
    }
    double* R = w.R1;
    double* Rn = w.R2;
    for (int q = 0; q < a; ++q) {
      double acc[S];
      mm_slots<D, LD, LD>(R, R, acc, sl);
#pragma unroll
      for (int t = 0; t < S; ++t)
        if (sl.ok[t]) Rn[sl.i[t] * LD + sl.j[t]] = acc[t];
      __syncwarp();
      double* tmp = R;
      R = Rn;
      Rn = tmp;
    }
    if (full) {
#pragma unroll
      for (int t = 0; t < S; ++t)
        if (sl.ok[t]) E[sl.i[t] * lde + sl.j[t]] = R[sl.i[t] * LD + sl.j[t]];
    } else {
      for (int o = lane; o < nrows * D; o += 32) {
        const int q = o / D, j = o - (o / D) * D;
        w.V[q * DMAX + j] = R[rows[q] * LD + j];
      }
      __syncwarp();
      for (int q = 0; q < (1 << (s - a)) - 1; ++q) rows_times<D>(w.V, R, LD, nrows, lane);
    }
  }
  __syncwarp();
  if (m_out) *m_out = m;
  if (s_out) *s_out = s;
  if (a_out) *a_out = a;
}

}  // namespace lmep
