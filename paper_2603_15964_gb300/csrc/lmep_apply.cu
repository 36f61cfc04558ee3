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

namespace lmep {

constexpr int MAXW = DMAX * 3 * DMAX;  // n * (1 + n_phi) * n, n <= 15, n_phi <= 2

// Halo staged on each side of a tile: the stages shrink the valid range by
// hs (a stencil) or hN (the KdV derivative).  Dirichlet adds hs so that the
// one-sided windows of points next to a wall stay inside the staged range
// even when the last tile is shorter than a stencil.
int apply_halo(int n, int scheme, int nonlin, int bc) {
  const int hs = (n - 1) / 2;
  const int hN = nonlin == 2 ? hs : 0;
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
  constexpr bool KDV = NONLIN == 2;
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
      const int r0 = dir ? 0 : hs, r1 = dir ? n : hs + 1;
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
          f = ST(-6) * x * ux * inv_h;
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
        int64_t st = i - hs;
        st = st < 0 ? 0 : (st > N - n ? N - n : st);
        ls = int(st - base);
        r = int(i - st);
      } else {
        ls = q - hs;
        r = hs;
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
        f = ST(-6) * x * ux * inv_h;
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

// ------------------------------------------------------------------ register-tiled fast path
// Periodic or Neumann tiles with a pointwise nonlinearity (none, Allen-Cahn),
// stencil width NW fixed at compile time.  The centre-row weights live in
// registers; each thread produces 4 consecutive outputs from windows read with
// 16-byte shared-memory vector loads, and N(.) is recomputed from the window
// values instead of being staged.  Halos are multiples of 4 so every window
// load is aligned; a tile stages round_up(len, 4) + 2H values.
int apply_fast_halo(int n, int scheme) {
  const int hs = (n - 1) / 2;
  const int hr = (hs + 3) / 4 * 4;
  return scheme == 2 ? 2 * hr : hr;
}

template <typename ST>
__device__ __forceinline__ ST nl_ac(ST x) { return x * fma(-x, x, ST(1)); }  // u - u^3

// Load `CNT` consecutive elements of shared memory starting at a 16-byte aligned
// position into registers with vector loads.
template <typename ST, int CNT>
__device__ __forceinline__ void load_window(const ST* __restrict__ src, ST (&x)[CNT]) {
  using V = typename std::conditional<sizeof(ST) == 4, float4, double2>::type;
  constexpr int VW = 16 / int(sizeof(ST));
#pragma unroll
  for (int v = 0; v < CNT / VW; ++v) {
    const V t = *reinterpret_cast<const V*>(src + v * VW);
    if constexpr (sizeof(ST) == 4) {
      x[v * 4] = t.x; x[v * 4 + 1] = t.y; x[v * 4 + 2] = t.z; x[v * 4 + 3] = t.w;
    } else {
      x[v * 2] = t.x; x[v * 2 + 1] = t.y;
    }
  }
}

template <typename ST, int CNT>
__device__ __forceinline__ void store_vec(ST* __restrict__ dst, const ST (&y)[CNT]) {
  using V = typename std::conditional<sizeof(ST) == 4, float4, double2>::type;
  constexpr int VW = 16 / int(sizeof(ST));
#pragma unroll
  for (int v = 0; v < CNT / VW; ++v) {
    if constexpr (sizeof(ST) == 4)
      *reinterpret_cast<V*>(dst + v * 4) = make_float4(y[v * 4], y[v * 4 + 1], y[v * 4 + 2], y[v * 4 + 3]);
    else
      *reinterpret_cast<V*>(dst + v * 2) = make_double2(y[v * 2], y[v * 2 + 1]);
  }
}

constexpr int FAST_P = 8;  // consecutive outputs per thread in the fast path

template <typename ST, int SCHEME, int NW>
__global__ void __launch_bounds__(512) k_apply_fast(ApplyParams a, const ST* __restrict__ u, ST* __restrict__ out,
                                                    const ST* __restrict__ W, int wq, unsigned* flags) {
  using V = typename std::conditional<sizeof(ST) == 4, float4, double2>::type;
  constexpr int P = FAST_P;
  constexpr int HS = (NW - 1) / 2;
  constexpr int HR = (HS + 3) / 4 * 4;
  constexpr int H = SCHEME == 2 ? 2 * HR : HR;
  constexpr int VW = 16 / int(sizeof(ST));
  constexpr int WIN = P + 2 * HR;  // window of one P-output group (multiple of 4)
  constexpr int OFF = HR - HS;     // first window element used by output 0
  extern __shared__ __align__(16) unsigned char smem[];
  const int Lmax = a.tile + 2 * H;
  ST* su = reinterpret_cast<ST*>(smem);
  ST* sa = su + Lmax;
  const bool ac = a.nonlin == 1;
  const ST inv_dt = ST(1.0 / a.dt);
  ST w0[NW], w1[NW], w2[NW];
  int64_t cur_inst = -1;
  unsigned bad = 0;
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    int64_t b = 0, t0, off = 0, N = a.N;
    int bc = a.bc;
    if (a.inst) {
      const int2 tt = a.tiles[tile];
      b = tt.x;
      t0 = tt.y;
      const Instance in = a.inst[b];
      off = in.off;
      N = in.N;
      bc = in.bc;
    } else {
      t0 = tile * int64_t(a.tile);
    }
    const int len = int((t0 + a.tile < N ? t0 + a.tile : N) - t0);
    const int lenp = (len + P - 1) / P * P;
    const int Lp = lenp + 2 * H;
    const int64_t base = t0 - H;
    if (b != cur_inst) {
      const ST* Wb = W + b * a.w_stride + int64_t(HS) * wq * NW;
#pragma unroll
      for (int j = 0; j < NW; ++j) {
        w0[j] = Wb[j];
        w1[j] = SCHEME >= 1 ? Wb[NW + j] : ST(0);
        w2[j] = SCHEME >= 2 ? Wb[2 * NW + j] : ST(0);
      }
      cur_inst = b;
    }
    __syncthreads();  // previous tile done with shared memory
    // Stage [base, base + Lp) in 16-byte chunks: instance starts and tile
    // starts are 16-byte aligned, so every chunk inside the instance is one
    // aligned vector load; chunks that cross an instance end wrap (periodic)
    // or reflect (Neumann) element by element.
    for (int c = threadIdx.x; c < Lp / VW; c += blockDim.x) {
      const int64_t i0 = base + int64_t(c) * VW;
      if (i0 >= 0 && i0 + VW <= N) {
        *reinterpret_cast<V*>(su + c * VW) = __ldg(reinterpret_cast<const V*>(u + off + i0));
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          int64_t i = i0 + e;
          if (i < 0 || i >= N) {
            if (bc == BC_PERIODIC) i = i < 0 ? i + N : i - N;
            else i = i < 0 ? -i : 2 * (N - 1) - i;
          }
          su[c * VW + e] = u[off + i];
        }
      }
    }
    __syncthreads();
    if (SCHEME == 2) {
      // first stage a on [HR, Lp - HR); windows [q - HR, q + P + HR) are staged
      const int ng = (Lp - 2 * HR) / P;
      for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int q = HR + P * g;
        ST x[WIN], nx[WIN], y[P];
        load_window<ST, WIN>(su + q - HR, x);
#pragma unroll
        for (int e = 0; e < WIN; ++e) nx[e] = ac ? nl_ac(x[e]) : ST(0);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          ST acc = ST(0);
#pragma unroll
          for (int j = 0; j < NW; ++j) {
            acc = fma(w0[j], x[OFF + p + j], acc);
            acc = fma(w1[j], nx[OFF + p + j], acc);
          }
          y[p] = acc;
        }
        store_vec<ST, P>(sa + q, y);
      }
      __syncthreads();
    }
    // outputs on [H, H + lenp)
    const int ng = lenp / P;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
      const int q = H + P * g;
      ST x[WIN], y[P];
      load_window<ST, WIN>(su + q - HR, x);
      if (SCHEME == 2) {
        ST z[WIN], d[WIN];
        load_window<ST, WIN>(sa + q - HR, z);
        // d = N(a) - N(u) on the window, then u+ = a + (W2 / dt) d
#pragma unroll
        for (int e = 0; e < WIN; ++e) d[e] = ac ? nl_ac(z[e]) - nl_ac(x[e]) : ST(0);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          ST acc = ST(0);
#pragma unroll
          for (int j = 0; j < NW; ++j) acc = fma(w2[j], d[OFF + p + j], acc);
          y[p] = fma(acc, inv_dt, z[HR + p]);
        }
      } else {
        ST nx[WIN];
#pragma unroll
        for (int e = 0; e < WIN; ++e) nx[e] = (SCHEME == 1 && ac) ? nl_ac(x[e]) : ST(0);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          ST acc = ST(0);
#pragma unroll
          for (int j = 0; j < NW; ++j) {
            acc = fma(w0[j], x[OFF + p + j], acc);
            if (SCHEME == 1) acc = fma(w1[j], nx[OFF + p + j], acc);
          }
          y[p] = acc;
        }
      }
      ST* o = out + off + t0 + P * g;
      if (P * g + P <= len) {
        store_vec<ST, P>(o, y);
#pragma unroll
        for (int p = 0; p < P; ++p) bad |= !isfinite(double(y[p]));
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (P * g + p < len) {
            o[p] = y[p];
            bad |= !isfinite(double(y[p]));
          }
        }
      }
    }
  }
  if (bad) atomicOr(flags, 1u);
}

template <typename ST, int SCHEME>
static const void* pick_fast_n(int n) {
  switch (n) {
    case 3: return (const void*)k_apply_fast<ST, SCHEME, 3>;
    case 5: return (const void*)k_apply_fast<ST, SCHEME, 5>;
    case 7: return (const void*)k_apply_fast<ST, SCHEME, 7>;
    case 9: return (const void*)k_apply_fast<ST, SCHEME, 9>;
    case 11: return (const void*)k_apply_fast<ST, SCHEME, 11>;
    case 13: return (const void*)k_apply_fast<ST, SCHEME, 13>;
    default: return (const void*)k_apply_fast<ST, SCHEME, 15>;
  }
}

template <typename ST>
static const void* pick_fast(int scheme, int n) {
  if (scheme == 0) return pick_fast_n<ST, 0>(n);
  if (scheme == 1) return pick_fast_n<ST, 1>(n);
  return pick_fast_n<ST, 2>(n);
}

template <typename ST>
static const void* pick(int scheme, int nonlin) {
  if (scheme == 0) return (const void*)k_apply<ST, 0, 0>;
  if (scheme == 1) return nonlin == 2 ? (const void*)k_apply<ST, 1, 2> : (const void*)k_apply<ST, 1, 1>;
  return nonlin == 2 ? (const void*)k_apply<ST, 2, 2> : (const void*)k_apply<ST, 2, 1>;
}

static const void* kernel_of(const ApplyParams& a, bool mixed) {
  if (a.fast) return mixed ? pick_fast<float>(a.scheme, a.n) : pick_fast<double>(a.scheme, a.n);
  return mixed ? pick<float>(a.scheme, a.nonlin) : pick<double>(a.scheme, a.nonlin);
}

static size_t smem_of(const ApplyParams& a, bool mixed) {
  const size_t es = mixed ? 4 : 8;
  if (a.fast) return size_t(a.scheme == 2 ? 2 : 1) * size_t(a.tile + 2 * a.halo) * es;
  return apply_smem_bytes(a.tile, a.halo, a.scheme, mixed);
}

int apply_grid(const ApplyParams& a, int block, int ctas_per_sm, bool mixed) {
  const void* k = kernel_of(a, mixed);
  const size_t smem = smem_of(a, mixed);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
  if (per_sm < 1) per_sm = 1;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  return int(a.ntiles < cap ? (a.ntiles > 0 ? a.ntiles : 1) : cap);
}

cudaError_t launch_apply(const ApplyParams& a, const void* u, void* out, const void* W, bool mixed,
                         int block, int grid, unsigned* flags, cudaStream_t s) {
  const size_t smem = smem_of(a, mixed);
  int wq = a.wq;
  const void* k = kernel_of(a, mixed);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  ApplyParams ap = a;
  void* args[] = {&ap, (void*)&u, &out, (void*)&W, (void*)&wq, &flags};
  return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace lmep
