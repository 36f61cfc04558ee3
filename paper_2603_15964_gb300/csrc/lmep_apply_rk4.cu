// lmep_apply_rk4.cu -- step (a6) for the ETDRK4 scheme (Sec. 3).
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
#include <cstdio>

#include "lmep_device.cuh"
#include "lmep_internal.h"

namespace lmep {

namespace {

constexpr int RK4_ROWS = 6;                       // E, A, B, G, E2, P2 per row class
constexpr int RK4_MAXW = DMAX * RK4_ROWS * DMAX;  // every row class (Dirichlet), width <= 16

struct Rk4Params {
  int64_t N;
  double h, dt, bc_lo, bc_hi;
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

template <typename ST, int NONLIN>
__global__ void __launch_bounds__(256) k_apply_rk4(Rk4Params a, const ST* __restrict__ u, ST* __restrict__ out,
                                                   const ST* __restrict__ W, const double* __restrict__ dh,
                                                   unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool DER = NONLIN >= 2;
  ST* sW = reinterpret_cast<ST*>(smem);
  ST* sD1 = sW + RK4_MAXW;
  ST* su = sD1 + DMAX * DMAX;
  const int n = a.n, hs = (n - 1) >> 1;
  const int H = a.halo;
  const int Lmax = a.tile + 2 * H;
  ST* sNu = su + Lmax;
  ST* sa = sNu + Lmax;
  ST* sNa = sa + Lmax;  // N(a), then N(a) + N(b)
  ST* sb = sNa + Lmax;
  ST* sNb = sb + Lmax;
  ST* sc = sNb + Lmax;
  ST* sNc = sc + Lmax;
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
  const ST inv_h = ST(1.0 / a.h);
  const ST lo_v = ST(a.bc_lo), hi_v = ST(a.bc_hi);
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
      su[q] = v;
    }
    __syncthreads();
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
    eval_n(su, sNu, lo);                     // N(u)
    __syncthreads();
    lo += rs;
    half_stage(su, sNu, sa, lo);             // a = E2 u + P2 N(u)
    __syncthreads();
    lo += rN;
    eval_n(sa, sNa, lo);                     // N(a)
    __syncthreads();
    lo += rs;
    half_stage(su, sNa, sb, lo);             // b = E2 u + P2 N(a)
    __syncthreads();
    lo += rN;
    eval_n(sb, sNb, lo);                     // N(b)
    __syncthreads();
    for (int q = lo + threadIdx.x; q < L - lo; q += blockDim.x) {
      sb[q] = ST(2) * sNb[q] - sNu[q];       // 2 N(b) - N(u)   (b is no longer needed)
      sNa[q] = sNa[q] + sNb[q];              // N(a) + N(b)
    }
    __syncthreads();
    lo += rs;
    half_stage(sa, sb, sc, lo);              // c = E2 a + P2 (2 N(b) - N(u))
    __syncthreads();
    lo += rN;
    eval_n(sc, sNc, lo);                     // N(c)
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
        for (int j = 0; j < n; ++j) acc = fma(e[j], su[ls + j], acc);
        for (int j = 0; j < n; ++j) acc = fma(e[DMAX + j], sNu[ls + j], acc);
        for (int j = 0; j < n; ++j) acc = fma(e[2 * DMAX + j], sNa[ls + j], acc);
        for (int j = 0; j < n; ++j) acc = fma(e[3 * DMAX + j], sNc[ls + j], acc);
        y = acc;
      }
      out[i] = y;
      bad |= !isfinite(y);
    }
  }
  if (bad) atomicOr(flags, 1u);
}

template <typename ST>
const void* rk4_kernel(int nonlin) {
  if (nonlin == 1) return (const void*)k_apply_rk4<ST, 1>;
  if (nonlin == 2) return (const void*)k_apply_rk4<ST, 2>;
  return (const void*)k_apply_rk4<ST, 3>;
}

size_t rk4_smem(int tile, int halo, bool mixed) {
  const size_t es = mixed ? 4 : 8;
  return (size_t(RK4_MAXW) + DMAX * DMAX + 8 * (size_t(tile) + 2 * size_t(halo))) * es;
}

}  // namespace

int rk4_halo(int n, int nonlin, int bc) {
  const int hs = (n - 1) / 2;
  const int rs = bc == BC_DIRICHLET ? 2 * hs : hs;  // one-sided windows reach n - 1 next to a wall
  const int rN = nonlin >= 2 ? rs : 0;
  return 4 * rs + 4 * rN;
}

cudaError_t launch_apply_rk4(int64_t N, double h, int bc, int n, int nonlin, double dt, double bc_lo, double bc_hi,
                             const void* u, void* out, const void* W, bool mixed, unsigned* flags, cudaStream_t s) {
  Rk4Params a{};
  a.N = N;
  a.h = h;
  a.dt = dt;
  a.bc_lo = bc_lo;
  a.bc_hi = bc_hi;
  a.n = n;
  a.bc = bc;
  a.halo = rk4_halo(n, nonlin, bc);
  const int hs = (n - 1) / 2;
  a.rs = bc == BC_DIRICHLET ? 2 * hs : hs;
  a.rN = nonlin >= 2 ? a.rs : 0;
  const size_t cap = size_t(device_info().smem_optin);
  int tile = mixed ? 2048 : 1024;
  while (tile > 64 && rk4_smem(tile, a.halo, mixed) > cap) tile /= 2;
  a.tile = tile;
  a.ntiles = (N + tile - 1) / tile;
  const size_t smem = rk4_smem(tile, a.halo, mixed);
  const void* k = mixed ? rk4_kernel<float>(nonlin) : rk4_kernel<double>(nonlin);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t cap_ctas = int64_t(device_info().sms) * per_sm;
  const int grid = int(a.ntiles < cap_ctas ? a.ntiles : cap_ctas);
  const double* dh;
  const float* dhf;
  if ((e = fornberg_of(n, &dh, &dhf)) != cudaSuccess) return e;
  void* args[] = {&a, (void*)&u, &out, (void*)&W, (void*)&dh, &flags};
  return cudaLaunchKernel(k, dim3(grid), dim3(256), args, smem, s);
}

}  // namespace lmep
