// lmep_frozen_set.cuh -- records and kernels of the frozen-velocity sets
// (lmep_frozen_set.cu): the lean factorised-row kernel and the fallback for
// the points it rejects.  The fallback is instantiated in its own translation
// units (lmep_set_fb_f32.cu, lmep_set_fb_f64.cu).
#pragma once

#include "lmep_warp_kernel.cuh"

namespace lmep {


// Per-instance record in the workspace.
struct alignas(16) SetInst {
  KParams p;
  int64_t off;       // first state element of the instance
  int64_t list_off;  // first entry of its rejected-point list
  int64_t tab;       // first element of its table (product type): exp(E) rows, stride NP(n), then R_j
  int32_t route;     // 0: factorised rows first; 1: every point through the fallback
};
static_assert(sizeof(SetInst) % 16 == 0, "SetInst is copied as 16-byte vectors");

// Row stride of a table of width n (16-byte vectors of floats, 32 bytes of doubles).
__host__ __device__ constexpr int tab_np(int n) { return (n + 3) / 4 * 4; }
__host__ __device__ constexpr int tab_elems(int n) { return (n + 1) * tab_np(n); }
constexpr int TAB_MAX = (DMAX + 1) * DMAX;

struct SetArgs {
  const SetInst* inst;
  const int2* tiles;  // {instance, first point}
  const void* tab;
  const int32_t* ok;  // per instance: 1 when its exp(E) table is finite
  int32_t* fail_count;
  int32_t* fail_list;
  const void* u;
  void* out;
  unsigned* flags;
};

struct FbArgs {
  const SetInst* inst;
  const WarpJob* jobs;
  int32_t* fail_count;
  const int32_t* fail_list;
  unsigned* done;
  int64_t B;
  const void* u;
  void* out;
  unsigned* flags;
};

template <typename T, int NP>
__device__ __forceinline__ void load_row(const T* src, T (&row)[NP]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int v = 0; v < NP / 4; ++v) {
      const float4 t = reinterpret_cast<const float4*>(src)[v];
      row[4 * v] = t.x;
      row[4 * v + 1] = t.y;
      row[4 * v + 2] = t.z;
      row[4 * v + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int v = 0; v < NP / 2; ++v) {
      const double2 t = reinterpret_cast<const double2*>(src)[v];
      row[2 * v] = t.x;
      row[2 * v + 1] = t.y;
    }
  }
}

// One tile of instance b: points t0 .. t0 + min(block * PPT, N - t0) - 1, thread
// t taking points t0 + t + k * blockDim.x (k < PPT).  The arithmetic of a point
// is that of the factorised stage of frozen_chunk (same operations in the same
// order), so both paths give the same bits.
template <int D, typename PT, int PPT>
__device__ __forceinline__ void set_tile(const SetArgs& a, const SetInst& in, int b, int64_t t0, PT* sT, PT* su,
                                         unsigned& bad) {
  using ST = PT;
  constexpr bool F32 = sizeof(PT) == 4;
  constexpr int H = D - 1;  // a window lies within [i - (n - 1), i + n - 1]
  constexpr int NP = tab_np(D);
  const KParams& p = in.p;
  const int64_t N = p.N;
  const int bc = p.bc;
  const int tp = int(blockDim.x) * PPT;
  const int len = int(N - t0 < int64_t(tp) ? N - t0 : int64_t(tp));
  const ST* u = static_cast<const ST*>(a.u) + in.off;
  ST* out = static_cast<ST*>(a.out) + in.off;
  const ST* tab = static_cast<const ST*>(a.tab) + in.tab;
  for (int e = threadIdx.x; e < tab_elems(D); e += blockDim.x) sT[e] = tab[e];
  for (int q = threadIdx.x; q < len + 2 * H; q += blockDim.x) {
    const int64_t i = t0 - H + q;
    ST v = ST(0);
    if (bc != BC_DIRICHLET || (i >= 0 && i < N)) v = u[grid_index(i, N, bc)];
    su[q] = v;
  }
  __syncthreads();
  const bool fact = in.route == 0 && a.ok[b] != 0;
  PT l[PPT][D];
  int ls[PPT];
  bool take[PPT], live[PPT], vld[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int q = int(threadIdx.x) + k * int(blockDim.x);
    vld[k] = q < len;
    const int64_t i = t0 + (vld[k] ? q : 0);
    const bool wall = bc == BC_DIRICHLET && (i == 0 || i == N - 1);
    live[k] = vld[k] && !wall;
    int64_t st;
    if constexpr (F32) {
      // in FP32 but for the window's integer decision next to a tie (exact FP64 test)
      const float uf = live[k] ? float(su[q + H]) : 0.0f;
      const int kd = p.dep ? departure_shift_f32(uf, p, D) : 0;
      st = window_start(i, N, D, bc, kd);
      const int r = int(i - st);
      const float a1 = p.c1_f - p.fa_f * uf;
      const int kr = int(fmaxf(float(r - (D - 1)), fminf(float(r), floorf(fmaf(-a1, p.dt_h_f, 0.5f)))));
      const float c1f = fmaf(a1, p.dt_h_f, float(kr));
      lagrange_weights<D, float>(float(r - kr) + c1f, l[k]);
    } else {
      const double ui = live[k] ? double(su[q + H]) : 0.0;
      const int kd = p.dep ? departure_shift(ui, p.dt, p.h, D, p.dt_h) : 0;
      st = window_start(i, N, D, bc, kd);
      const int r = int(i - st);
      const double a1 = p.c1 - p.fa * ui;
      const int kr = recentring_shift(a1, p.dt_h, D, r);
      const double c1h = fma(a1, p.dt_h, double(kr));
      lagrange_weights<D, double>(double(r - kr) + c1h, l[k]);
    }
    ls[k] = int(st - (t0 - H));
    PT bound = PT(0);
#pragma unroll
    for (int j = 0; j < D; ++j) bound = fma(abs(l[k][j]), sT[D * NP + j], bound);
    take[k] = live[k] && fact && bound <= PT(SL_TAU);
  }
  // row_m = sum_j l_j exp(E)[j][m]: row j of the table is read once for all PPT points
  PT acc[PPT][D];
#pragma unroll
  for (int k = 0; k < PPT; ++k)
#pragma unroll
    for (int m = 0; m < D; ++m) acc[k][m] = PT(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    PT row[NP];
    load_row<PT, NP>(sT + j * NP, row);
#pragma unroll
    for (int k = 0; k < PPT; ++k)
#pragma unroll
      for (int m = 0; m < D; ++m) acc[k][m] = fma(l[k][j], row[m], acc[k][m]);
  }
  const PT e0 = p.c0dt != 0.0 ? PT(exp(p.c0dt)) : PT(1);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    PT res = PT(0);
#pragma unroll
    for (int m = 0; m < D; ++m) res = fma(acc[k][m] * e0, PT(su[ls[k] + m]), res);
    const int q = int(threadIdx.x) + k * int(blockDim.x);
    const int64_t i = t0 + q;
    if (vld[k] && !live[k]) out[i] = ST(i == 0 ? p.bc_lo : p.bc_hi);
    if (take[k]) {
      out[i] = res;
      bad |= !isfinite(res);
    }
    // rejected points: appended to the instance's list (one atomic per warp)
    const bool rej = live[k] && !take[k];
    const unsigned m = __ballot_sync(FULL, rej);
    if (m) {
      const int lane = threadIdx.x & 31;
      const int lead = __ffs(m) - 1;
      int base = 0;
      if (lane == lead) base = atomicAdd(a.fail_count + b, __popc(m));
      base = __shfl_sync(FULL, base, lead);
      if (rej) a.fail_list[in.list_off + base + __popc(m & ((1u << lane) - 1u))] = int32_t(i);
    }
  }
}

template <typename PT, int PPT>
__global__ void __launch_bounds__(512) k_frozen_set(SetArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) SetInst s_in;
  const int2 td = a.tiles[blockIdx.x];
  const int b = td.x;
  if (threadIdx.x < sizeof(SetInst) / 16)
    reinterpret_cast<int4*>(&s_in)[threadIdx.x] = reinterpret_cast<const int4*>(a.inst + b)[threadIdx.x];
  __syncthreads();
  PT* sT = reinterpret_cast<PT*>(smem);
  PT* su = sT + TAB_MAX;
  unsigned bad = 0;
  const int64_t t0 = td.y;
  switch (s_in.p.n) {
    case 3: set_tile<3, PT, PPT>(a, s_in, b, t0, sT, su, bad); break;
    case 5: set_tile<5, PT, PPT>(a, s_in, b, t0, sT, su, bad); break;
    case 7: set_tile<7, PT, PPT>(a, s_in, b, t0, sT, su, bad); break;
    case 9: set_tile<9, PT, PPT>(a, s_in, b, t0, sT, su, bad); break;
    case 11: set_tile<11, PT, PPT>(a, s_in, b, t0, sT, su, bad); break;
    case 13: set_tile<13, PT, PPT>(a, s_in, b, t0, sT, su, bad); break;
    default: set_tile<15, PT, PPT>(a, s_in, b, t0, sT, su, bad); break;
  }
  if (bad) atomicOr(a.flags, 1u);
}

// The listed points of every instance, 32 per warp, through frozen_chunk's
// finite-series and Pade stages (the jobs carry no factorised table).
template <typename PT>
__global__ void __launch_bounds__(32 * WARPS) k_frozen_set_fallback(FbArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Ws<PT> w(smem + warp * Ws<PT>::BYTES);
  const int64_t gw = int64_t(blockIdx.x) * WARPS + warp, nw = int64_t(gridDim.x) * WARPS;
  unsigned bad = 0;
  for (int64_t b = 0; b < a.B; ++b) {
    const int64_t cnt = a.fail_count[b];
    if (cnt == 0) continue;
    const WarpJob& job = a.jobs[b];
    const SetInst& in = a.inst[b];
    const PT* u = static_cast<const PT*>(a.u) + in.off;
    PT* out = static_cast<PT*>(a.out) + in.off;
    const int32_t* list = a.fail_list + in.list_off;
    const int n = job.p.n;
    for (int64_t c = gw * 32; c < cnt; c += nw * 32) {
      const int64_t e = c + 32 < cnt ? c + 32 : cnt;
      switch (n) {
        case 3: frozen_chunk<3, PT>(job, w, job.dh, job.dhf, c, e, lane, bad, u, out, list); break;
        case 5: frozen_chunk<5, PT>(job, w, job.dh, job.dhf, c, e, lane, bad, u, out, list); break;
        case 7: frozen_chunk<7, PT>(job, w, job.dh, job.dhf, c, e, lane, bad, u, out, list); break;
        case 9: frozen_chunk<9, PT>(job, w, job.dh, job.dhf, c, e, lane, bad, u, out, list); break;
        case 11: frozen_chunk<11, PT>(job, w, job.dh, job.dhf, c, e, lane, bad, u, out, list); break;
        case 13: frozen_chunk<13, PT>(job, w, job.dh, job.dhf, c, e, lane, bad, u, out, list); break;
        default: frozen_chunk<15, PT>(job, w, job.dh, job.dhf, c, e, lane, bad, u, out, list); break;
      }
    }
  }
  if (bad) atomicOr(a.flags, 1u);
  // every CTA has read the counters before it arrives; the last one clears them
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.done, 1u) == gridDim.x - 1) {
      for (int64_t b = 0; b < a.B; ++b) a.fail_count[b] = 0;
      *a.done = 0;
      __threadfence();
    }
  }
}


cudaError_t launch_set_fallback_f32(const FbArgs& a, unsigned grid, cudaStream_t s);
cudaError_t launch_set_fallback_f64(const FbArgs& a, unsigned grid, cudaStream_t s);

}  // namespace lmep
