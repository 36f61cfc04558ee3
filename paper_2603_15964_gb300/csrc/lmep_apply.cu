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

// ------------------------------------------------------------------ pipelined fast path
// Periodic or Neumann tiles with a pointwise nonlinearity (none, Allen-Cahn),
// stencil width NW fixed at compile time.  Persistent CTAs walk their tiles
// with two stage buffers: while a tile is computed, the next one is already
// on its way into the other buffer through one bulk asynchronous copy (TMA
// engine, completion counted on an mbarrier), so the SM keeps a whole tile of
// loads in flight instead of one round trip per thread.  The few staged values
// outside an instance (periodic wrap, Neumann reflection) and its ragged last
// elements are read with plain loads into registers at the same time and
// written into the stage buffer after the current tile is done.
//
// Compute: the centre-row weights live in registers; each thread produces 4
// consecutive outputs from windows read with 16-byte shared-memory vector
// loads, and N(.) is evaluated once per window element.  Halos are multiples
// of 4 so every window load is aligned; a tile stages round_up(len, 4) + 2H
// values.
// Points updated per tile by the fast kernel: for ETDRK2 the first stage
// spans the tile's outputs plus one stencil halo on each side, so a tile of
// `tile` staged points updates tile - 2 hr of them and both stages split
// evenly over the threads.
int fast_tile_out(int tile, int n, int scheme) {
  const int hr = ((n - 1) / 2 + 3) / 4 * 4;
  return scheme == 2 ? tile - 2 * hr : tile;
}

int apply_fast_halo(int n, int scheme) {
  const int hs = (n - 1) / 2;
  const int hr = (hs + 3) / 4 * 4;
  return scheme == 2 ? 2 * hr : hr;
}

template <typename ST>
__device__ __forceinline__ ST nl_ac(ST x) { return x * fma(-x, x, ST(1)); }  // u - u^3

// ---- two-lane arithmetic.  FP32 pairs use the packed f32x2 instructions
// (two IEEE single-precision operations per instruction); FP64 pairs are two
// scalar operations.  Lane "lo" is the lower address.
template <typename ST>
struct PairOps;

template <>
struct PairOps<float> {
  using T = unsigned long long;
  static __device__ __forceinline__ T make(float a, float b) {
    T r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
  }
  static __device__ __forceinline__ void split(T r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
  }
  static __device__ __forceinline__ T fma(T a, T b, T c) {
    T d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
  }
  static __device__ __forceinline__ T mul(T a, T b) {
    T d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
  }
  static __device__ __forceinline__ T sub(T a, T b) {
    T d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
  }
  static __device__ __forceinline__ float sum(T r) {
    float a, b;
    split(r, a, b);
    return a + b;
  }
  // `CNT` pairs from 16-byte aligned shared memory
  template <int CNT>
  static __device__ __forceinline__ void load(const float* src, T (&x)[CNT]) {
    static_assert(CNT % 2 == 0, "pairs come in 16-byte vectors");
#pragma unroll
    for (int v = 0; v < CNT / 2; ++v) {
      const ulonglong2 t = reinterpret_cast<const ulonglong2*>(src)[v];
      x[2 * v] = t.x;
      x[2 * v + 1] = t.y;
    }
  }
  static __device__ __forceinline__ void store2(float* dst, T a, T b) {
    reinterpret_cast<ulonglong2*>(dst)[0] = make_ulonglong2(a, b);
  }
};

template <>
struct PairOps<double> {
  using T = double2;
  static __device__ __forceinline__ T make(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ void split(T r, double& a, double& b) {
    a = r.x;
    b = r.y;
  }
  static __device__ __forceinline__ T fma(T a, T b, T c) {
    return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
  }
  static __device__ __forceinline__ T mul(T a, T b) { return make_double2(a.x * b.x, a.y * b.y); }
  static __device__ __forceinline__ T sub(T a, T b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ double sum(T r) { return r.x + r.y; }
  template <int CNT>
  static __device__ __forceinline__ void load(const double* src, T (&x)[CNT]) {
#pragma unroll
    for (int v = 0; v < CNT; ++v) x[v] = reinterpret_cast<const double2*>(src)[v];
  }
  static __device__ __forceinline__ void store2(double* dst, T a, T b) {
    reinterpret_cast<double2*>(dst)[0] = a;
    reinterpret_cast<double2*>(dst)[1] = b;
  }
};

// ---- mbarrier and bulk-copy primitives (PTX, sm_90+)
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return unsigned(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Order this thread's earlier generic-proxy shared-memory accesses before
// later bulk (async-proxy) writes to the same buffers.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// dst, src and bytes are multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Wait for the phase with the given parity to complete; gives up after a
// bounded number of polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned addr = smem_u32(bar);
  for (int it = 0; it < (1 << 20); ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Geometry of one tile: staged range [base, base + Lp) of instance coordinates,
// of which [lo, hi) is copied in bulk and the rest is read element by element.
struct TileGeo {
  int64_t off, N, t0, base, lo, hi;
  int b, bc, len, Lp;
};

// Descriptor of a tile: from the batch's tile table, or computed for a single
// instance.
__device__ __forceinline__ TileDesc load_desc(const ApplyParams& a, int64_t tile) {
  TileDesc d;
  if (a.desc) {
    const longlong2* p = reinterpret_cast<const longlong2*>(a.desc + tile);
    const longlong2 v0 = __ldg(p), v1 = __ldg(p + 1);
    d.off = v0.x;
    d.N = v0.y;
    d.t0 = v1.x;
    d.b = int(v1.y & 0xffffffff);
    d.bc = int(v1.y >> 32);
  } else {
    d.off = 0;
    d.N = a.N;
    d.t0 = tile * int64_t(a.tile);
    d.b = 0;
    d.bc = a.bc;
  }
  return d;
}

template <int H, int P, int VW>
__device__ __forceinline__ TileGeo tile_geo(const ApplyParams& a, const TileDesc& d) {
  TileGeo g;
  g.b = d.b;
  g.off = d.off;
  g.N = d.N;
  g.bc = d.bc;
  g.t0 = d.t0;
  g.len = int((g.t0 + a.tile < g.N ? g.t0 + a.tile : g.N) - g.t0);
  g.Lp = (g.len + P - 1) / P * P + 2 * H;
  g.base = g.t0 - H;
  g.lo = g.base > 0 ? g.base : 0;
  const int64_t nv = g.N - g.N % VW;
  g.hi = g.base + g.Lp < nv ? g.base + g.Lp : nv;
  if (g.hi < g.lo) g.hi = g.lo;
  return g;
}

// Staged position handled element by element by thread e (or -1), with the
// global index it reads (wrap for periodic, reflection about the wall node
// for Neumann).
__device__ __forceinline__ int edge_pos(const TileGeo& g, int e, int64_t* src) {
  const int nlo = int(g.lo - g.base);
  const int q = e < nlo ? e : int(g.hi - g.base) + (e - nlo);
  if (q >= g.Lp) return -1;
  int64_t i = g.base + q;
  if (i < 0 || i >= g.N) {
    if (g.bc == BC_PERIODIC) i = i < 0 ? i + g.N : i - g.N;
    else i = i < 0 ? -i : 2 * (g.N - 1) - i;
  }
  *src = g.off + i;
  return q;
}

constexpr int FAST_P = 4;           // consecutive outputs per thread
constexpr int FAST_MAX_STAGES = 4;  // stage buffers (bulk copies in flight + 1)
constexpr int FAST_HEADER = 64 + 32 * FAST_MAX_STAGES;  // mbarriers, abort word, tile descriptors

// Weight-pair tables.  A window of staged values is read as aligned pairs
// (x[2i], x[2i+1]); output p with stencil start s takes the pairs
// i = floor(s/2) + t, t < NT, against the weight pairs
//   even s: (w[2t], w[2t+1]),   odd s: (w[2t-1], w[2t])   (w outside [0, NW) is 0),
// so every product is a two-lane FMA whose lanes are summed at the end.
// The weights of the nonlinear terms are stored negated: the kernel evaluates
// -N(u) = u^3 - u, which takes one instruction less per pair than N(u).
template <int NW>
struct PairTable {
  static constexpr int NT = (NW + 1) / 2;
  static constexpr int ENTRIES = 3 * 2 * NT * 2;         // {W0, W1, W2} x {even, odd} x NT pairs
  static constexpr int STRIDE = (ENTRIES + 3) / 4 * 4;  // elements per table (16-byte multiple)
};

// Value of pair-table entry e for instance b, from the centre row of its
// stored weights W[b][row][k][j] (k < wq weight sets of n taps).
template <typename ST>
__device__ __forceinline__ ST pair_table_entry(const ST* __restrict__ W, int64_t w_stride, int wq, int n, int scheme,
                                               int64_t b, int e) {
  const int nt = (n + 1) / 2;
  const int k = e / (4 * nt);
  const int ph = (e / (2 * nt)) & 1;
  const int t = (e >> 1) % nt;
  const int wi = 2 * t + (e & 1) - ph;
  if (k > scheme || k > 2 || wi < 0 || wi >= n) return ST(0);
  const ST w = W[b * w_stride + int64_t((n - 1) / 2) * wq * n + k * n + wi];
  return k ? -w : w;
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

template <typename ST, int SCHEME, int NW>
__global__ void __launch_bounds__(512) k_apply_tma(ApplyParams a, const ST* __restrict__ u, ST* __restrict__ out,
                                                   const ST* __restrict__ W, int wq, unsigned* flags) {
  using PO = PairOps<ST>;
  using T = typename PO::T;
  constexpr int P = FAST_P;
  constexpr int HS = (NW - 1) / 2;
  constexpr int HR = (HS + 3) / 4 * 4;
  constexpr int H = SCHEME == 2 ? 2 * HR : HR;
  constexpr int VW = 16 / int(sizeof(ST));
  constexpr int WIN = P + 2 * HR;  // window of one P-output group (multiple of 4)
  constexpr int WP = WIN / 2;      // pairs per window
  constexpr int OFF = HR - HS;     // stencil start of output 0 inside the window
  constexpr int NT = PairTable<NW>::NT;
  constexpr int TS = PairTable<NW>::STRIDE;
  constexpr int TE = PairTable<NW>::ENTRIES;
  // Shared memory: a header with NS mbarriers, an abort word and NS tile
  // descriptors; NS weight-pair tables; NS stage buffers; for ETDRK2 the first
  // stage a and the difference D = N(a) - N(u) (stored negated).  Tile j of
  // this CTA lives in slot j mod NS; tiles j+1 .. j+NS-1 are in flight while j
  // is computed.  A slot's data and (for batches) its pair table arrive by bulk
  // copy; the few staged values outside the instance are read with plain loads
  // one tile later and stored one tile after that, so no global load latency
  // sits on a tile's critical path.
  extern __shared__ __align__(128) unsigned char smem[];
  const int NS = a.stages;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  int& s_abort = *reinterpret_cast<int*>(smem + 8 * FAST_MAX_STAGES);
  TileDesc* meta = reinterpret_cast<TileDesc*>(smem + 64);
  const int Lmax = a.tile + 2 * H;
  ST* wtab = reinterpret_cast<ST*>(smem + FAST_HEADER);
  ST* buf = wtab + NS * TS;
  ST* sa = buf + NS * Lmax;
  ST* sd = sa + Lmax;
  const ST* ptab = static_cast<const ST*>(a.ptab);
  const T ZERO = PO::make(ST(0), ST(0));
  const T M1 = PO::make(ST(-1), ST(-1));
  const ST inv_dt_s = ST(1.0 / a.dt);
  const T INV = PO::make(inv_dt_s, inv_dt_s);
  T chk = ZERO;  // fma(out, 0, chk) turns any Inf/NaN output into NaN
  if (blockIdx.x >= a.ntiles) return;
  if (threadIdx.x == 0) {
    for (int j = 0; j < NS; ++j) mbar_init(&bar[j], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  // thread 0: bulk copies of a tile (and its pair table) into slot j
  auto issue = [&](const TileDesc& d, const TileGeo& g, int j) {
    meta[j] = d;
    const unsigned bytes = unsigned(g.hi - g.lo) * unsigned(sizeof(ST));
    const unsigned tbytes = ptab ? unsigned(TS * sizeof(ST)) : 0u;
    mbar_expect_tx(&bar[j], bytes + tbytes);
    if (bytes) bulk_g2s(buf + int64_t(j) * Lmax + (g.lo - g.base), u + g.off + g.lo, bytes, &bar[j]);
    if (tbytes) bulk_g2s(wtab + j * TS, ptab + int64_t(g.b) * TS, tbytes, &bar[j]);
  };
  // prologue: the first NS-1 tiles of this CTA, edges stored directly
  for (int j = 0; j < NS - 1; ++j) {
    const int64_t t = blockIdx.x + int64_t(j) * gridDim.x;
    if (t >= a.ntiles) break;
    const TileDesc d = load_desc(a, t);
    const TileGeo gj = tile_geo<H, P, VW>(a, d);
    if (threadIdx.x == 0) issue(d, gj, j);
    int64_t src;
    const int q = edge_pos(gj, threadIdx.x, &src);
    if (q >= 0) buf[int64_t(j) * Lmax + q] = __ldg(u + src);
  }
  if (!ptab && int(threadIdx.x) < TE)  // one instance: one table, built once
    wtab[threadIdx.x] = pair_table_entry(W, a.w_stride, wq, NW, SCHEME, 0, threadIdx.x);
  int64_t tile = blockIdx.x;
  TileDesc dnext{};  // descriptor of the next tile to fetch, loaded one tile ahead
  {
    const int64_t t = tile + int64_t(NS - 1) * gridDim.x;
    if (t < a.ntiles) dnext = load_desc(a, t);
  }
  int pend_q = -1;  // edge value loaded during the previous tile, stored after this one
  ST pend_v = ST(0);
  // slot of the current tile (k mod NS) and the parity of each slot's next wait
  int s = 0;
  unsigned parity = 0;
  for (;;) {
    const int sf = s == 0 ? NS - 1 : s - 1;  // slot of tile k + NS - 1, released when tile k - 1 ended
    const int64_t ftile = tile + int64_t(NS - 1) * gridDim.x;
    int eq = -1;
    ST ev = ST(0);
    if (ftile < a.ntiles) {
      const TileGeo gf = tile_geo<H, P, VW>(a, dnext);
      if (threadIdx.x == 0) issue(dnext, gf, sf);
      int64_t src;
      eq = edge_pos(gf, threadIdx.x, &src);
      if (eq >= 0) ev = __ldg(u + src);
      if (ftile + gridDim.x < a.ntiles) dnext = load_desc(a, ftile + gridDim.x);
    }
    if (threadIdx.x == 0 && !mbar_wait(&bar[s], (parity >> s) & 1u)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    parity ^= 1u << s;
    const TileGeo g = tile_geo<H, P, VW>(a, meta[s]);
    const ST* cur = buf + int64_t(s) * Lmax;
    const T* wp = reinterpret_cast<const T*>(wtab + (ptab ? s * TS : 0));  // [k][phase][t]
    const int lenp = g.Lp - 2 * H;
    if (SCHEME == 2) {
      // first stage on [HR, Lp - HR): a = W0 u + W1 N(u) and D = N(a) - N(u)
      T w0[2][NT], w1[2][NT];
#pragma unroll
      for (int ph = 0; ph < 2; ++ph)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          w0[ph][t] = wp[(0 * 2 + ph) * NT + t];
          w1[ph][t] = wp[(1 * 2 + ph) * NT + t];
        }
      const int ng = (g.Lp - 2 * HR) / P;
      for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
        const int q = HR + P * gi;
        T x[WP], nx[WP];
        PO::template load<WP>(cur + q - HR, x);
#pragma unroll
        for (int i = 0; i < WP; ++i) nx[i] = PO::mul(x[i], PO::fma(x[i], x[i], M1));  // -N(u)
        ST y[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int st = OFF + p, i0 = st >> 1, ph = st & 1;
          T acc = ZERO;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            acc = PO::fma(w0[ph][t], x[i0 + t], acc);
            acc = PO::fma(w1[ph][t], nx[i0 + t], acc);
          }
          y[p] = PO::sum(acc);
        }
        const T a01 = PO::make(y[0], y[1]), a23 = PO::make(y[2], y[3]);
        const T d01 = PO::sub(PO::mul(a01, PO::fma(a01, a01, M1)), nx[HR / 2]);
        const T d23 = PO::sub(PO::mul(a23, PO::fma(a23, a23, M1)), nx[HR / 2 + 1]);
        PO::store2(sa + q, a01, a23);
        PO::store2(sd + q, d01, d23);
      }
      __syncthreads();
    }
    // outputs on [H, H + lenp)
    {
      T w[2][2][NT];  // ETDRK2: W2 only; otherwise W0 and W1
#pragma unroll
      for (int ph = 0; ph < 2; ++ph)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          w[0][ph][t] = wp[((SCHEME == 2 ? 2 : 0) * 2 + ph) * NT + t];
          w[1][ph][t] = wp[(1 * 2 + ph) * NT + t];
        }
      for (int gi = threadIdx.x; gi < lenp / P; gi += blockDim.x) {
        const int q = H + P * gi;
        T x[WP], nx[WP];
        PO::template load<WP>((SCHEME == 2 ? sd : cur) + q - HR, x);
        if (SCHEME == 1) {
#pragma unroll
          for (int i = 0; i < WP; ++i) nx[i] = PO::mul(x[i], PO::fma(x[i], x[i], M1));
        }
        ST y[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int st = OFF + p, i0 = st >> 1, ph = st & 1;
          T acc = ZERO;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            acc = PO::fma(w[0][ph][t], x[i0 + t], acc);
            if (SCHEME == 1) acc = PO::fma(w[1][ph][t], nx[i0 + t], acc);
          }
          y[p] = PO::sum(acc);
        }
        T o01 = PO::make(y[0], y[1]), o23 = PO::make(y[2], y[3]);
        if (SCHEME == 2) {
          // u+ = a + (W2 / dt) D
          T av[2];
          PO::template load<2>(sa + q, av);
          o01 = PO::fma(o01, INV, av[0]);
          o23 = PO::fma(o23, INV, av[1]);
        }
        chk = PO::fma(o01, ZERO, chk);
        chk = PO::fma(o23, ZERO, chk);
        ST* o = out + g.off + g.t0 + P * gi;
        if (P * gi + P <= g.len) {
          PO::store2(o, o01, o23);
        } else {
          ST v[4];
          PO::split(o01, v[0], v[1]);
          PO::split(o23, v[2], v[3]);
#pragma unroll
          for (int p = 0; p < P; ++p)
            if (P * gi + p < g.len) o[p] = v[p];
        }
      }
    }
    // the edge value loaded during the previous tile belongs to tile k + NS - 2
    // (slot (k + NS - 2) mod NS, not computed before tile k + 1)
    if (pend_q >= 0) buf[int64_t(s >= 2 ? s - 2 : s + NS - 2) * Lmax + pend_q] = pend_v;
    pend_q = eq;
    pend_v = ev;
    fence_proxy_async_smem();
    __syncthreads();  // releases slot s, a and D; makes the stored edge values visible
    tile += gridDim.x;
    if (tile >= a.ntiles) break;
    s = s + 1 == NS ? 0 : s + 1;
  }
  if (s_abort && threadIdx.x == 0) {
    // a bulk copy did not complete in time: report it and give the copies
    // still in flight (this tile and the next NS - 1) a bounded time to land
    atomicOr(flags, 2u);
    for (int d = 0; d < NS; ++d) {
      const int j = (s + d) % NS;
      if (tile + int64_t(d) * gridDim.x < a.ntiles) mbar_wait(&bar[j], (parity >> j) & 1u);
    }
  }
  ST c0, c1;
  PO::split(chk, c0, c1);
  if (!(c0 == ST(0) && c1 == ST(0))) atomicOr(flags, 1u);
}

template <typename ST, int SCHEME>
static const void* pick_fast_n(int n) {
  switch (n) {
    case 3: return (const void*)k_apply_tma<ST, SCHEME, 3>;
    case 5: return (const void*)k_apply_tma<ST, SCHEME, 5>;
    case 7: return (const void*)k_apply_tma<ST, SCHEME, 7>;
    case 9: return (const void*)k_apply_tma<ST, SCHEME, 9>;
    case 11: return (const void*)k_apply_tma<ST, SCHEME, 11>;
    case 13: return (const void*)k_apply_tma<ST, SCHEME, 13>;
    default: return (const void*)k_apply_tma<ST, SCHEME, 15>;
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

// The fast kernels hard-wire the Allen-Cahn nonlinearity for ETD schemes; with
// no nonlinearity every ETD step reduces to u+ = W0 u, the linear kernel (the
// weight stride wq is passed separately and keeps the stored layout).
static int fast_scheme(const ApplyParams& a) { return a.nonlin == 0 ? 0 : a.scheme; }

static const void* kernel_of(const ApplyParams& a, bool mixed) {
  if (a.fast) return mixed ? pick_fast<float>(fast_scheme(a), a.n) : pick_fast<double>(fast_scheme(a), a.n);
  return mixed ? pick<float>(a.scheme, a.nonlin) : pick<double>(a.scheme, a.nonlin);
}

static size_t fast_smem(const ApplyParams& a, bool mixed, int stages) {
  const size_t es = mixed ? 4 : 8;
  return FAST_HEADER + size_t(stages) * size_t(PairTable<15>::STRIDE) * es +
         size_t(stages + (fast_scheme(a) == 2 ? 2 : 0)) * size_t(a.tile + 2 * a.halo) * es;
}

static size_t smem_of(const ApplyParams& a, bool mixed) {
  const size_t es = mixed ? 4 : 8;
  if (a.fast) return fast_smem(a, mixed, a.stages);
  return apply_smem_bytes(a.tile, a.halo, a.scheme, mixed);
}

// Pipeline depth of the fast kernel: as many stage buffers (3..4) as fit
// without lowering the number of CTAs per SM that three buffers allow.
bool apply_configure(ApplyParams& a, bool mixed) {
  a.stages = 0;
  if (!a.fast) return apply_smem_bytes(a.tile, a.halo, a.scheme, mixed) <= size_t(device_info().smem_optin);
  const size_t cap = size_t(device_info().smem_optin);
  const size_t limit = fast_smem(a, mixed, 3) <= cap / 2 ? cap / 2 : cap;
  for (int st = FAST_MAX_STAGES; st >= 3; --st)
    if (fast_smem(a, mixed, st) <= limit) {
      a.stages = st;
      return true;
    }
  return false;
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
