// lmep_apply.cu -- step (a6): banded application of stored weights.
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
// wall values are never updated.
#include <cstdio>
#include <type_traits>

#include "lmep_device.cuh"
#include "lmep_internal.h"
#include "lmep_stream.cuh"

namespace lmep {

constexpr int MAXW = DMAX * 3 * DMAX;  // n * (1 + n_phi) * n, n <= 15, n_phi <= 2

// Halo staged on each side of a tile: the stages shrink the valid range by
// hs (a stencil) or hN (the KdV derivative).  Dirichlet adds hs so that the
// one-sided windows of points next to a wall stay inside the staged range
// even when the last tile is shorter than a stencil.
int apply_halo(int n, int scheme, int nonlin, int bc) {
  const int hs = (n - 1) / 2;
  const int hN = nonlin >= 2 ? hs : 0;
  int H = scheme == 0 ? hs : (scheme == 1 ? hs + hN : 2 * hs + 2 * hN);
  if (bc == BC_DIRICHLET) H += hs;
  return H;
}

size_t apply_smem_bytes(int tile, int halo, int scheme, bool mixed) {
  const size_t es = mixed ? 4 : 8;
  const size_t L = size_t(tile) + 2 * size_t(halo);
  const size_t arrays = scheme == 0 ? 1 : (scheme == 1 ? 3 : 4);
  return (MAXW + DMAX) * es + arrays * L * es;
}

template <typename ST, int SCHEME, int NONLIN>
__global__ void __launch_bounds__(512) k_apply(ApplyParams a, const ST* __restrict__ u, ST* __restrict__ out,
                                               const ST* __restrict__ W, int wq, unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  ST* sW = reinterpret_cast<ST*>(smem);
  ST* sd1 = sW + MAXW;
  const int n = a.n, hs = (n - 1) >> 1;
  constexpr bool KDV = NONLIN >= 2;                 // a derivative nonlinearity: KdV or Burgers
  const ST ncoef = ST(NONLIN == 2 ? -6 : -1);         // N = ncoef u u_x
  const int hN = KDV ? hs : 0;
  const int H = a.halo;
  const int Lmax = a.tile + 2 * H;
  ST* su = sd1 + DMAX;
  ST* sN = su + Lmax;
  ST* sa = sN + Lmax;
  ST* sNa = sa + Lmax;
  const ST inv_dt = ST(1.0 / a.dt);
  if (KDV) {
    if (threadIdx.x == 0) {
      double c[4][DMAX];
      fornberg_row(double(hs), n, c);
      for (int j = 0; j < n; ++j) sd1[j] = ST(c[1][j]);
    }
  }
  int64_t cur_inst = -1;
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
    }
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
      const int64_t i = base + q;
      ST v = ST(0);
      if (!dir || (i >= 0 && i < N)) v = u[off + grid_index(i, N, bc)];
      su[q] = v;
    }
    __syncthreads();
    const ST inv_h = ST(1.0 / h);
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
        bad |= !isfinite(double(y));
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
        bad |= !isfinite(double(y));
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
      bad |= !isfinite(double(y));
    }
  }
  if (bad) atomicOr(flags, 1u);
}

// ------------------------------------------------------------------ streaming fast path
// Geometry of the warp-streaming kernel (lmep_apply_stream.cu): a warp takes
// 128 staged points per round; for ETDRK2 the first stage runs on all 128 and
// the second updates the inner 128 - 2 hr of them.  A tile of `tile` staged
// points per round-set (tile / 128 rounds) updates fast_tile_out points.
int fast_tile_out(int tile, int n, int scheme) {
  const int hr = ((n - 1) / 2 + 3) / 4 * 4;
  const int rounds = tile / 128 > 0 ? tile / 128 : 1;
  return rounds * (scheme == 2 ? 128 - 2 * hr : 128);
}

int apply_fast_halo(int n, int scheme) {
  const int hs = (n - 1) / 2;
  const int hr = (hs + 3) / 4 * 4;
  return scheme == 2 ? 2 * hr : hr;
}

template <typename ST>
__global__ void k_pair_tables(const ST* __restrict__ W, int64_t w_stride, int wq, int n, int scheme, int64_t B,
                              int stride, ST* __restrict__ tab) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= B * stride) return;
  const int64_t b = i / stride;
  const int e = int(i % stride);
  tab[i] = pair_table_entry(W, w_stride, wq, n, scheme, b, e);
}

int pair_table_stride(int n) { return (3 * 2 * ((n + 1) / 2) * 2 + 3) / 4 * 4; }

cudaError_t launch_pair_tables(const void* W, int64_t w_stride, int wq, int n, int scheme, int64_t B, void* tab,
                               bool mixed, cudaStream_t s) {
  const int stride = pair_table_stride(n);
  const int64_t total = B * stride;
  if (total == 0) return cudaSuccess;
  const int block = 256;
  const unsigned grid = unsigned((total + block - 1) / block);
  if (mixed)
    k_pair_tables<float><<<grid, block, 0, s>>>(static_cast<const float*>(W), w_stride, wq, n, scheme, B, stride,
                                                static_cast<float*>(tab));
  else
    k_pair_tables<double><<<grid, block, 0, s>>>(static_cast<const double*>(W), w_stride, wq, n, scheme, B, stride,
                                                 static_cast<double*>(tab));
  return cudaGetLastError();
}

template <typename ST>
static const void* pick(int scheme, int nonlin) {
  if (scheme == 0) return (const void*)k_apply<ST, 0, 0>;
  if (scheme == 1)
    return nonlin == 3 ? (const void*)k_apply<ST, 1, 3>
                       : (nonlin == 2 ? (const void*)k_apply<ST, 1, 2> : (const void*)k_apply<ST, 1, 1>);
  return nonlin == 3 ? (const void*)k_apply<ST, 2, 3>
                     : (nonlin == 2 ? (const void*)k_apply<ST, 2, 2> : (const void*)k_apply<ST, 2, 1>);
}

// The fast kernels hard-wire the Allen-Cahn nonlinearity for ETD schemes; with
// no nonlinearity every ETD step reduces to u+ = W0 u, the linear kernel (the
// weight stride wq is passed separately and keeps the stored layout).
static int fast_scheme(const ApplyParams& a) { return a.nonlin == 0 ? 0 : a.scheme; }

static const void* kernel_of(const ApplyParams& a, bool mixed) {
  if (a.fast) return stream_kernel(fast_scheme(a), a.n, mixed);
  return mixed ? pick<float>(a.scheme, a.nonlin) : pick<double>(a.scheme, a.nonlin);
}

static size_t smem_of(const ApplyParams& a, bool mixed, int block) {
  if (a.fast) return size_t(a.warp_smem) * size_t(block / 32);
  return apply_smem_bytes(a.tile, a.halo, a.scheme, mixed);
}

// Pipeline depth of the streaming kernel: 4 slots per warp, or 3 when 4 do
// not fit `block` threads' worth of warps in shared memory.
bool apply_configure(ApplyParams& a, bool mixed, int block) {
  a.stages = 0;
  a.warp_smem = 0;
  const size_t cap = size_t(device_info().smem_optin);
  if (!a.fast) return apply_smem_bytes(a.tile, a.halo, a.scheme, mixed) <= cap;
  for (int st = STREAM_MAX_STAGES; st >= 3; --st) {
    const size_t w = stream_warp_smem(a, mixed, st, fast_scheme(a));
    if (w * size_t(block / 32) <= cap) {
      a.stages = st;
      a.warp_smem = int(w);
      return true;
    }
  }
  return false;
}

int apply_grid(const ApplyParams& a, int block, int ctas_per_sm, bool mixed) {
  const void* k = kernel_of(a, mixed);
  const size_t smem = smem_of(a, mixed, block);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
  if (per_sm < 1) per_sm = 1;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  // the streaming kernel gives every warp its own tiles
  const int64_t units = a.fast ? (a.ntiles + block / 32 - 1) / (block / 32) : a.ntiles;
  return int(units < cap ? (units > 0 ? units : 1) : cap);
}

cudaError_t launch_apply(const ApplyParams& a, const void* u, void* out, const void* W, bool mixed,
                         int block, int grid, unsigned* flags, cudaStream_t s) {
  const size_t smem = smem_of(a, mixed, block);
  int wq = a.wq;
  const void* k = kernel_of(a, mixed);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  ApplyParams ap = a;
  void* args[] = {&ap, (void*)&u, &out, (void*)&W, (void*)&wq, &flags};
  return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace lmep
