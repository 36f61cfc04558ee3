// lmep_stream.cuh -- building blocks of the streaming apply kernels:
// two-lane arithmetic (packed f32x2 for FP32), mbarrier / bulk-copy
// primitives, tile geometry and the weight-pair tables.
#pragma once
#include <cstdint>

#include "lmep_device.cuh"
#include "lmep_internal.h"

namespace lmep {

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
// Default bound of a wait, in polls (far longer than any bulk copy of a tile).
constexpr int WAIT_POLLS = 1 << 20;
// Wait for the phase with the given parity to complete; gives up after
// `polls` polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int polls = WAIT_POLLS) {
  const unsigned addr = smem_u32(bar);
  for (int it = 0; it < polls; ++it) {
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

}  // namespace lmep
