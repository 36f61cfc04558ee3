/*
 * lmep_oracle.c -- FP64 CPU oracle of the frozen-velocity LMEP step, in plain C.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests/ and by bench.py's CPU-baseline
 * leg through oracle/cpu.py.  It shares no code with the CUDA library and
 * includes none of its headers.  The same steps as the numpy oracle
 * (oracle/lmep.py), written out once more in C so that the oracle can be
 * timed on all host cores (OpenMP over grid points) and can check every point
 * of a full-size step:
 *
 *  Sec. 2.1 step 1  window of point i: Dirichlet start clamp(i - hs - k, 0, N - n),
 *                   harvest row i - start (one-sided edge rows near the walls);
 *                   periodic centred and wrapped; Neumann centred with even
 *                   reflection about the wall node; departure centring
 *                   k = clamp(floor(u_i dt / h + 1/2), -hs, hs).
 *  Sec. 2.1 step 1  derivative matrices of the window: D1[i][j] = l_j'(i) of the
 *                   Lagrange basis on the integer nodes 0..n-1 (closed form),
 *                   D2 = D1 D1 and D3 = D1 D2 (on P_{n-1} the k-th derivative is
 *                   the k-th power of the first).
 *  Thm. 2 proof     X = dt (c0 I + c1 D1/h + c2 D2/h^2 + c3 D3/h^3 - fa u_i D1/h),
 *                   re-centred by the integer k_r nearest the local Courant number
 *                   (row r of exp(X) equals row r - k_r of exp(X + k_r D1)).
 *  Sec. 2.1 step 2  exp(X) by Pade [m/m] scaling and squaring (Higham 2005,
 *                   Algorithm 2.3: m in {3,5,7,9} when ||X||_1 <= theta_m, else
 *                   m = 13 with s = ceil(log2(||X||_1 / theta_13)); LU with
 *                   partial pivoting; s squarings).
 *  Sec. 2.1 step 3  the harvested row applied to the window: u_i+ = w . u[window].
 * Dirichlet walls keep bc_lo / bc_hi.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NMAX 16

static const double THETA[5] = {1.495585217958292e-2, 2.539398330063230e-1, 9.504178996162932e-1,
                                2.097847961257068e0, 5.371920351148152e0};
static const int DEGREE[5] = {3, 5, 7, 9, 13};

/* C = A B for n x n row-major matrices (C distinct from A and B). */
static void matmul(int n, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
      C[i * n + j] = s;
    }
}

static double norm1(int n, const double* A) {
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fabs(A[i * n + j]);
    if (s > best) best = s;
  }
  return best;
}

/* b_j of the [m/m] Pade numerator of e^x: (2m - j)! m! / ((2m)! j! (m - j)!). */
static void pade_coefficients(int m, double* b) {
  b[0] = 1.0;
  for (int j = 0; j < m; ++j) b[j + 1] = b[j] * (double)(m - j) / ((double)(2 * m - j) * (double)(j + 1));
}

/* Solve Q R = P (n x n) in place: R returned in P.  Gaussian elimination with
 * partial pivoting, then back substitution. */
static void lu_solve(int n, double* Q, double* P) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(Q[i * n + k]) > fabs(Q[piv * n + k])) piv = i;
    if (piv != k)
      for (int j = 0; j < n; ++j) {
        double t = Q[k * n + j];
        Q[k * n + j] = Q[piv * n + j];
        Q[piv * n + j] = t;
        t = P[k * n + j];
        P[k * n + j] = P[piv * n + j];
        P[piv * n + j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      const double l = Q[i * n + k] / Q[k * n + k];
      for (int j = k; j < n; ++j) Q[i * n + j] -= l * Q[k * n + j];
      for (int j = 0; j < n; ++j) P[i * n + j] -= l * P[k * n + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    for (int j = 0; j < n; ++j) {
      double s = P[k * n + j];
      for (int q = k + 1; q < n; ++q) s -= Q[k * n + q] * P[q * n + j];
      P[k * n + j] = s / Q[k * n + k];
    }
}

/* E = exp(A), n x n (Higham 2005, Algorithm 2.3). */
static void expm(int n, const double* A, double* E) {
  double As[NMAX * NMAX], I[NMAX * NMAX], A2[NMAX * NMAX], A4[NMAX * NMAX], A6[NMAX * NMAX];
  double U[NMAX * NMAX], V[NMAX * NMAX], T[NMAX * NMAX], T2[NMAX * NMAX], b[14];
  const int nn = n * n;
  const double a = norm1(n, A);
  int m = 13, s = 0;
  for (int q = 0; q < 4; ++q)
    if (a <= THETA[q]) {
      m = DEGREE[q];
      break;
    }
  if (m == 13 && a > THETA[4]) s = (int)ceil(log2(a / THETA[4]));
  const double scale = ldexp(1.0, -s);
  for (int e = 0; e < nn; ++e) As[e] = A[e] * scale;
  for (int e = 0; e < nn; ++e) I[e] = 0.0;
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  pade_coefficients(m, b);
  matmul(n, As, As, A2);
  if (m < 13) {
    /* odd = sum b_{2j+1} A^{2j}, even = sum b_{2j} A^{2j}, j <= (m-1)/2; U = A odd, V = even */
    double P[NMAX * NMAX], odd[NMAX * NMAX];
    for (int e = 0; e < nn; ++e) {
      P[e] = I[e];
      odd[e] = b[1] * I[e];
      V[e] = b[0] * I[e];
    }
    for (int j = 1; j <= (m - 1) / 2; ++j) {
      matmul(n, P, A2, T);
      memcpy(P, T, sizeof(double) * nn);
      for (int e = 0; e < nn; ++e) {
        odd[e] += b[2 * j + 1] * P[e];
        V[e] += b[2 * j] * P[e];
      }
    }
    matmul(n, As, odd, U);
  } else {
    matmul(n, A2, A2, A4);
    matmul(n, A4, A2, A6);
    for (int e = 0; e < nn; ++e) T[e] = b[13] * A6[e] + b[11] * A4[e] + b[9] * A2[e];
    matmul(n, A6, T, T2);
    for (int e = 0; e < nn; ++e) T2[e] += b[7] * A6[e] + b[5] * A4[e] + b[3] * A2[e] + b[1] * I[e];
    matmul(n, As, T2, U);
    for (int e = 0; e < nn; ++e) T[e] = b[12] * A6[e] + b[10] * A4[e] + b[8] * A2[e];
    matmul(n, A6, T, V);
    for (int e = 0; e < nn; ++e) V[e] += b[6] * A6[e] + b[4] * A4[e] + b[2] * A2[e] + b[0] * I[e];
  }
  double Q[NMAX * NMAX];
  for (int e = 0; e < nn; ++e) {
    Q[e] = V[e] - U[e];
    E[e] = V[e] + U[e];
  }
  lu_solve(n, Q, E);
  for (int q = 0; q < s; ++q) {
    matmul(n, E, E, T);
    memcpy(E, T, sizeof(double) * nn);
  }
}

/* D[k] (k = 1..3, n x n each) on the integer nodes 0..n-1. */
static void derivative_matrices(int n, double* D1, double* D2, double* D3) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double v;
      if (i == j) {
        v = 0.0;
        for (int m = 0; m < n; ++m)
          if (m != j) v += 1.0 / (double)(j - m);
      } else {
        /* l_j'(x_i) = prod_{m != i, j} (i - m) / prod_{m != j} (j - m) */
        double num = 1.0, den = 1.0;
        for (int m = 0; m < n; ++m) {
          if (m != j) den *= (double)(j - m);
          if (m != i && m != j) num *= (double)(i - m);
        }
        v = num / den;
      }
      D1[i * n + j] = v;
    }
  matmul(n, D1, D1, D2);
  matmul(n, D1, D2, D3);
}

static int64_t wrap(int64_t q, int64_t N, int bc) {
  if (bc == 0) {
    q %= N;
    return q < 0 ? q + N : q;
  }
  if (bc == 2) {
    if (q < 0) q = -q;
    if (q > N - 1) q = 2 * (N - 1) - q;
  }
  return q;
}

/* One frozen-velocity step at the points pts[0..npts) (all N points when pts is
 * NULL, out then indexed by point): out[k] = the updated value of point pts[k].
 * bc: 0 periodic, 1 Dirichlet, 2 Neumann.  threads <= 0: the OpenMP default.
 * Returns 0, or -1 for an unsupported width. */
int lmep_oracle_frozen_step(int64_t N, double h, int bc, int n, int dep, double dt, double c0, double c1,
                            double c2, double c3, double fa, double bc_lo, double bc_hi, const double* u,
                            const int64_t* pts, int64_t npts, double* out, int threads) {
  if (n < 3 || n > 15 || n % 2 == 0) return -1;
  double D1[NMAX * NMAX], D2[NMAX * NMAX], D3[NMAX * NMAX];
  derivative_matrices(n, D1, D2, D3);
  const int hs = (n - 1) / 2;
  const int64_t count = pts ? npts : N;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
  for (int64_t q = 0; q < count; ++q) {
    const int64_t i = pts ? pts[q] : q;
    if (bc == 1 && (i == 0 || i == N - 1)) {
      out[q] = i == 0 ? bc_lo : bc_hi;
      continue;
    }
    const double ui = u[i];
    int k = 0;
    if (dep) {
      double t = floor(ui * dt / h + 0.5);
      if (t < -hs) t = -hs;
      if (t > hs) t = hs;
      k = (int)t;
    }
    int64_t start = i - hs - k;
    if (bc == 1) start = start < 0 ? 0 : (start > N - n ? N - n : start);
    const int r = (int)(i - start);
    /* re-centring by the integer nearest the local Courant number, kept so that row r - kr exists */
    const double a1 = c1 - fa * ui;
    double kr = floor(-dt * a1 / h + 0.5);
    if (kr > r) kr = r;
    if (kr < r - (n - 1)) kr = r - (n - 1);
    double X[NMAX * NMAX], E[NMAX * NMAX];
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        const int e = a * n + b;
        X[e] = (dt * a1 / h) * D1[e] + (dt * c2 / (h * h)) * D2[e] + (dt * c3 / (h * h * h)) * D3[e] +
               kr * D1[e];
        if (a == b) X[e] += dt * c0;
      }
    expm(n, X, E);
    const int row = r - (int)kr;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += E[row * n + j] * u[wrap(start + j, N, bc)];
    out[q] = acc;
  }
  return 0;
}

/* The oracle's thread count after an OpenMP region (1 without OpenMP). */
int lmep_oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
