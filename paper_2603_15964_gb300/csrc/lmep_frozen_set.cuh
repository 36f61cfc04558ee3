// lmep_frozen_set.cuh -- records and kernels of the frozen-velocity sets
// (lmep_frozen_set.cu): the lean factorised-row kernel and the fallback for
// the points it rejects.  The fallback is instantiated in its own translation
// units (lmep_set_fb_f32.cu, lmep_set_fb_f64.cu).
#pragma once

#include "lmep_stream.cuh"
#include "lmep_warp_kernel.cuh"

namespace lmep {


// Per-instance record in the workspace.
struct alignas(16) SetInst {
  KParams p;
  int64_t off;       // first state element of the instance
  int64_t list_off;  // first entry of its rejected-point list
  int64_t tab;       // first element of its table (product type): exp(E) rows, stride NP(n), then R_j
  int32_t route;     // 0: factorised rows first; 1: every point through the fallback
  int32_t ok;        // 1 when the instance's exp(E) table is finite (written by the set-up kernel)
};
static_assert(sizeof(SetInst) % 16 == 0, "SetInst is copied as 16-byte vectors");

// Row stride of a table of width n (16-byte vectors of floats, 32 bytes of doubles).
__host__ __device__ constexpr int tab_np(int n) { return (n + 3) / 4 * 4; }
__host__ __device__ constexpr int tab_elems(int n) { return (n + 1) * tab_np(n); }
constexpr int TAB_MAX = (DMAX + 1) * DMAX;

// Per-tile record: what staging a tile needs before its instance record has
// arrived (the kernel loads these two tiles ahead).
struct alignas(16) SetTile {
  int64_t off;                    // first state element of the instance
  int32_t N, t0, b, n, bc, tab;   // instance size, first point, instance, width, boundary, table offset
};
static_assert(sizeof(SetTile) == 32, "SetTile is 32 bytes");

struct SetArgs {
  const SetInst* inst;
  const SetTile* tiles;   // CTA c's tiles are tiles[starts[c] .. starts[c + 1])
  const int32_t* starts;  // (the API caps a set at 2^31 - 1 tiles)
  const void* tab;
  const int32_t* ok;  // per instance: 1 when its exp(E) table is finite
  int32_t* fail_count;
  int32_t* fail_total;  // rejected points of all instances (the fallback's early exit)
  int32_t* fail_list;
  const void* u;
  void* out;
  unsigned* flags;
};

struct FbArgs {
  const SetInst* inst;
  const WarpJob* jobs;
  int32_t* fail_count;
  int32_t* fail_total;
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

// Programmatic dependent launch (sm_90+): a kernel launched with programmatic
// stream serialization may start while the previous kernel of the stream is
// finishing; griddepcontrol.wait returns once that kernel has completed and
// its memory is visible (at once for an ordinary launch), and
// griddepcontrol.launch_dependents lets the next kernel start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Window start of point i with shift k (window_start in 32-bit integers:
// instances of a set have N < 2^31).
__device__ __forceinline__ int set_window_start(int i, int N, int n, int bc, int k) {
  int s = i - ((n - 1) >> 1) - k;
  if (bc == BC_DIRICHLET) s = s < 0 ? 0 : (s > N - n ? N - n : s);
  return s;
}

// Issue the asynchronous copies that stage tile d in shared memory: its
// instance record, the instance's exp(E) table and the tile's values with
// n - 1 more on each side (one wrap for periodic, N >= n; one reflection for
// Neumann, N >= 2n; Dirichlet windows stay inside [0, N), outside values are 0).
__device__ __forceinline__ unsigned smem_addr(const void* p) { return unsigned(__cvta_generic_to_shared(p)); }
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename PT>
__device__ __forceinline__ void stage_tile(const SetArgs& a, const SetTile& d, SetInst* s_in, PT* sT, PT* su, int tp) {
  constexpr int NI = int(sizeof(SetInst)) / 16;
  for (int e = threadIdx.x; e < NI; e += blockDim.x)
    cp_async<16>(reinterpret_cast<int4*>(s_in) + e, reinterpret_cast<const int4*>(a.inst + d.b) + e);
  constexpr int PER16 = 16 / int(sizeof(PT));
  const PT* tab = static_cast<const PT*>(a.tab) + d.tab;
  const int tel = (d.n + 1) * ((d.n + 3) / 4 * 4);
  for (int e = threadIdx.x; e < tel / PER16; e += blockDim.x) cp_async<16>(sT + e * PER16, tab + e * PER16);
  const int H = d.n - 1;
  const int N = d.N;
  const int len = N - d.t0 < tp ? N - d.t0 : tp;
  const PT* u = static_cast<const PT*>(a.u) + d.off;
  for (int q = threadIdx.x; q < len + 2 * H; q += blockDim.x) {
    int i = d.t0 - H + q;
    bool have = true;
    if (d.bc == BC_PERIODIC) {
      i = i < 0 ? i + N : (i >= N ? i - N : i);
    } else if (d.bc == BC_NEUMANN) {
      i = i < 0 ? -i : i;
      i = i > N - 1 ? 2 * (N - 1) - i : i;
    } else {
      have = i >= 0 && i < N;
    }
    if (have) cp_async<int(sizeof(PT))>(su + q, u + i);
    else su[q] = PT(0);
  }
}

// The points of one staged tile of instance b: points t0 .. t0 + min(block * PPT,
// N - t0) - 1, thread t taking points t0 + t + k * blockDim.x (k < PPT).  The
// arithmetic of a point is that of the factorised stage of frozen_chunk (same
// operations in the same order), so both paths give the same bits.
template <int D, typename PT, int PPT>
__device__ __forceinline__ void set_tile(const SetArgs& a, const SetInst& in, int b, int t0, const PT* sT,
                                         const PT* su, unsigned& bad) {
  using ST = PT;
  constexpr bool F32 = sizeof(PT) == 4;
  constexpr int H = D - 1;  // a window lies within [i - (n - 1), i + n - 1]
  constexpr int NP = tab_np(D);
  const KParams& p = in.p;
  const int N = int(p.N);
  const int bc = p.bc;
  const int tp = int(blockDim.x) * PPT;
  const int len = N - t0 < tp ? N - t0 : tp;
  ST* out = static_cast<ST*>(a.out) + in.off;
  const bool fact = in.route == 0 && in.ok != 0;
  PT l[PPT][D];
  int ls[PPT];
  bool take[PPT], live[PPT], vld[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int q = int(threadIdx.x) + k * int(blockDim.x);
    vld[k] = q < len;
    const int i = t0 + (vld[k] ? q : 0);
    const bool wall = bc == BC_DIRICHLET && (i == 0 || i == N - 1);
    live[k] = vld[k] && !wall;
    int st;
    if constexpr (F32) {
      // in FP32 but for the window's integer decision next to a tie (exact FP64 test)
      const float uf = live[k] ? float(su[q + H]) : 0.0f;
      const int kd = p.dep ? departure_shift_f32(uf, p, D) : 0;
      st = set_window_start(i, N, D, bc, kd);
      const int r = i - st;
      const float a1 = p.c1_f - p.fa_f * uf;
      const int kr = int(fmaxf(float(r - (D - 1)), fminf(float(r), floorf(fmaf(-a1, p.dt_h_f, 0.5f)))));
      const float c1f = fmaf(a1, p.dt_h_f, float(kr));
      lagrange_weights<D, float>(float(r - kr) + c1f, l[k]);
    } else {
      const double ui = live[k] ? double(su[q + H]) : 0.0;
      const int kd = p.dep ? departure_shift(ui, p.dt, p.h, D, p.dt_h) : 0;
      st = set_window_start(i, N, D, bc, kd);
      const int r = i - st;
      const double a1 = p.c1 - p.fa * ui;
      const int kr = recentring_shift(a1, p.dt_h, D, r);
      const double c1h = fma(a1, p.dt_h, double(kr));
      lagrange_weights<D, double>(double(r - kr) + c1h, l[k]);
    }
    ls[k] = st - (t0 - H);
    PT bound = PT(0);
#pragma unroll
    for (int j = 0; j < D; ++j) bound = fma(abs(l[k][j]), sT[D * NP + j], bound);
    take[k] = live[k] && fact && bound <= PT(SL_TAU);
  }
  // row_m = sum_j l_j exp(E)[j][m]: row j of the table is read once for all PPT points.
  // FP32: columns m, m + 1 in one packed f32x2 FMA (each lane an IEEE fma, so
  // the bits are those of the scalar sums); an odd width's last pair carries
  // the table's zero padding in its upper lane, which is never read.
  PT acc[PPT][D];
  if constexpr (F32) {
    using PO = PairOps<float>;
    constexpr int DP = (D + 1) / 2;
    PO::T acc2[PPT][DP];
#pragma unroll
    for (int k = 0; k < PPT; ++k)
#pragma unroll
      for (int m = 0; m < DP; ++m) acc2[k][m] = 0ull;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      PO::T row[NP / 2];
      PO::template load<NP / 2>(sT + j * NP, row);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const PO::T lj = PO::make(l[k][j], l[k][j]);
#pragma unroll
        for (int m = 0; m < DP; ++m) acc2[k][m] = PO::fma(lj, row[m], acc2[k][m]);
      }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k)
#pragma unroll
      for (int m = 0; m < DP; ++m) {
        float lo, hi;
        PO::split(acc2[k][m], lo, hi);
        acc[k][2 * m] = lo;
        if (2 * m + 1 < D) acc[k][2 * m + 1] = hi;
      }
  } else {
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
  }
  // e^{dt c0} of the identity term; a product with exactly 1 changes no bit, so it is skipped
  const bool react = p.c0dt != 0.0;
  const PT e0 = react ? PT(exp(p.c0dt)) : PT(1);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    PT res = PT(0);
    if (react) {
#pragma unroll
      for (int m = 0; m < D; ++m) res = fma(acc[k][m] * e0, PT(su[ls[k] + m]), res);
    } else {
#pragma unroll
      for (int m = 0; m < D; ++m) res = fma(acc[k][m], PT(su[ls[k] + m]), res);
    }
    const int q = int(threadIdx.x) + k * int(blockDim.x);
    const int i = t0 + q;
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
      if (lane == lead) {
        base = atomicAdd(a.fail_count + b, __popc(m));
        atomicAdd(a.fail_total, __popc(m));
      }
      base = __shfl_sync(FULL, base, lead);
      if (rej) a.fail_list[in.list_off + base + __popc(m & ((1u << lane) - 1u))] = int32_t(i);
    }
  }
}

// The tiles tile .. end - 1 of a CTA, staged two buffers deep.  A tile holds
// SEQ sub-tiles of blockDim.x * PPT points, computed in turn (PPT points per
// thread together in registers, SEQ times), so that the per-tile work of the
// CTA (staging, barrier, records) is shared by SEQ * PPT points per thread.
template <typename PT, int PPT, int SEQ>
__device__ __forceinline__ void set_tiles(const SetArgs& a, int tile, const int end, PT* buf, SetInst* s_in,
                                          const int stride, const int tp, unsigned& bad) {
  SetTile cur = a.tiles[tile];
  stage_tile<PT>(a, cur, &s_in[0], buf, buf + TAB_MAX, tp);
  cp_async_commit();
  bool has_nxt = tile + 1 < end;
  SetTile nxt{};
  if (has_nxt) nxt = a.tiles[tile + 1];
  int bi = 0;
  for (;;) {
    cp_async_wait_all();
    __syncthreads();  // tile bi staged; everyone is done with buffer bi ^ 1
    bool has_nn = false;
    SetTile nn{};
    if (has_nxt) {
      PT* o = buf + (bi ^ 1) * stride;
      stage_tile<PT>(a, nxt, &s_in[bi ^ 1], o, o + TAB_MAX, tp);
      has_nn = tile + 2 < end;
      if (has_nn) nn = a.tiles[tile + 2];
    }
    cp_async_commit();
    const PT* sT = buf + bi * stride;
    const PT* su = sT + TAB_MAX;
    const SetInst& in = s_in[bi];
    const int sub = int(blockDim.x) * PPT;
#pragma unroll 1
    for (int q = 0; q < SEQ; ++q) {
      const int t0 = cur.t0 + q * sub;
      if (t0 >= cur.N) break;  // the instance's ragged last tile (uniform over the CTA)
      const PT* suq = su + q * sub;
      switch (cur.n) {
        case 3: set_tile<3, PT, PPT>(a, in, cur.b, t0, sT, suq, bad); break;
        case 5: set_tile<5, PT, PPT>(a, in, cur.b, t0, sT, suq, bad); break;
        case 7: set_tile<7, PT, PPT>(a, in, cur.b, t0, sT, suq, bad); break;
        case 9: set_tile<9, PT, PPT>(a, in, cur.b, t0, sT, suq, bad); break;
        case 11: set_tile<11, PT, PPT>(a, in, cur.b, t0, sT, suq, bad); break;
        case 13: set_tile<13, PT, PPT>(a, in, cur.b, t0, sT, suq, bad); break;
        default: set_tile<15, PT, PPT>(a, in, cur.b, t0, sT, suq, bad); break;
      }
    }
    if (!has_nxt) break;
    cur = nxt;
    nxt = nn;
    has_nxt = has_nn;
    ++tile;
    bi ^= 1;
  }
}

// Persistent: CTA c takes its own run of tiles (balanced on the host).  While
// it computes a tile from one shared-memory buffer, the asynchronous copies of
// its next tile fill the other, and the tile record after that is loaded into
// registers, so the loads of a tile overlap the arithmetic of the previous one.
// One point per thread: at most 64 registers, so that 8 CTAs of 128 threads
// (or 2 of 512) fit on an SM.
template <typename PT, int PPT, int SEQ>
__global__ void __launch_bounds__(512, PPT == 1 ? 2 : 1) k_frozen_set(SetArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) SetInst s_in[2];
  const int tp = int(blockDim.x) * PPT * SEQ;
  const int stride = TAB_MAX + tp + 2 * DMAX;  // elements per buffer (a multiple of 16)
  PT* buf = reinterpret_cast<PT*>(smem);
  // the tile records and instance records are read-only; the state and the
  // counters belong to the previous step's kernels
  pdl_wait();
  pdl_trigger();
  int tile = a.starts[blockIdx.x];
  const int end = a.starts[blockIdx.x + 1];
  unsigned bad = 0;
  if (tile < end) set_tiles<PT, PPT, SEQ>(a, tile, end, buf, s_in, stride, tp, bad);
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
  pdl_wait();     // the lists and the lean kernel's outputs are complete
  pdl_trigger();
  // nothing rejected (the usual case): every CTA leaves after one load, and
  // the counters are all zero already.  The total is cleared only by the last
  // CTA below, after every CTA has read it, so all CTAs take the same branch.
  if (*static_cast<volatile const int32_t*>(a.fail_total) == 0) return;
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
      *a.fail_total = 0;
      *a.done = 0;
      __threadfence();
    }
  }
}


// Launch with programmatic stream serialization (see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_set_fallback_f32(const FbArgs& a, unsigned grid, cudaStream_t s);
cudaError_t launch_set_fallback_f64(const FbArgs& a, unsigned grid, cudaStream_t s);

}  // namespace lmep
