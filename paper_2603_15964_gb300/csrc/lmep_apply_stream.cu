// lmep_apply_stream.cu -- step (a6) for periodic and Neumann tiles with a
// pointwise nonlinearity (none or Allen-Cahn): the warp-streaming apply.
//
// Sec. 3.1 step 3 applies the harvested rows as banded dot products.  Here
// every warp is an independent streaming unit with its own shared-memory
// slots: tiles j+1 .. j+NS-1 of a warp are in flight (one bulk asynchronous
// copy each, counted on the slot's mbarrier, together with the instance's
// weight-pair table) while tile j is computed, so HBM sees a deep queue of
// large reads and no CTA-wide barrier ever stalls the pipeline.  The few
// staged values outside an instance (periodic wrap, Neumann reflection about
// the wall node) and its ragged last elements are read with plain loads one
// tile ahead and stored one tile later.
//
// A round covers 128 staged points, 4 per lane.  Stencils are evaluated on
// aligned pairs with packed f32x2 FMAs against even/odd weight-pair tables;
// N(u) is evaluated once per window pair (as -N, the sign folded into the
// weights).  ETDRK2: each lane computes the first stage a and
// D = N(a) - N(u) on its own 4 points; the second stage takes the
// neighbouring lanes' D through warp shuffles and updates the inner
// 128 - 2 hr points of the round.  The state is read once and written once.
#include <cstdio>

#include "lmep_stream.cuh"

namespace lmep {

namespace {

constexpr int P = 4;  // consecutive points per lane

template <typename ST>
__device__ __forceinline__ typename PairOps<ST>::T shfl_pair(typename PairOps<ST>::T v, int src) {
  if constexpr (sizeof(ST) == 4) {
    return __shfl_sync(0xffffffffu, v, src);
  } else {
    double2 r;
    r.x = __shfl_sync(0xffffffffu, v.x, src);
    r.y = __shfl_sync(0xffffffffu, v.y, src);
    return r;
  }
}

template <typename ST, int SCHEME, int NW>
__global__ void __launch_bounds__(512) k_apply_stream(ApplyParams a, const ST* __restrict__ u, ST* __restrict__ out,
                                                      const ST* __restrict__ W, int wq, unsigned* flags) {
  using PO = PairOps<ST>;
  using T = typename PO::T;
  constexpr int HS = (NW - 1) / 2;
  constexpr int HR = (HS + 3) / 4 * 4;
  constexpr int H = SCHEME == 2 ? 2 * HR : HR;
  constexpr int VW = 16 / int(sizeof(ST));
  constexpr int WIN = P + 2 * HR;  // window of one lane's 4 points (multiple of 4)
  constexpr int WP = WIN / 2;      // pairs per window
  constexpr int OFF = HR - HS;     // stencil start of point 0 inside the window
  constexpr int LH = HR / 4;       // lanes of first-stage halo on each side (ETDRK2)
  constexpr int OUTW = SCHEME == 2 ? 32 * P - 2 * HR : 32 * P;  // points updated per round
  constexpr int NT = PairTable<NW>::NT;
  constexpr int TS = PairTable<NW>::STRIDE;
  constexpr int TE = PairTable<NW>::ENTRIES;
  const int NS = a.stages;
  const int Lmax = a.tile + 2 * H;  // a.tile: points updated per tile (a multiple of OUTW)
  const int lane = threadIdx.x & 31;
  // this warp's shared memory: NS mbarriers, NS tile descriptors, NS
  // weight-pair tables and NS stage buffers
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* ws = smem + size_t(threadIdx.x >> 5) * size_t(a.warp_smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(ws);
  TileDesc* meta = reinterpret_cast<TileDesc*>(ws + 8 * STREAM_MAX_STAGES);
  ST* wtab = reinterpret_cast<ST*>(ws + STREAM_HEADER);
  ST* buf = wtab + NS * TS;
  const ST* ptab = static_cast<const ST*>(a.ptab);
  const T ZERO = PO::make(ST(0), ST(0));
  const T M1 = PO::make(ST(-1), ST(-1));
  const ST inv_dt_s = ST(a.inv_dt);
  const T INV = PO::make(inv_dt_s, inv_dt_s);
  T chk = ZERO;  // fma(out, 0, chk) turns any Inf/NaN output into NaN
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  int64_t tile = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tile >= a.ntiles) return;  // whole warp
  if (lane == 0) {
    for (int j = 0; j < NS; ++j) mbar_init(&bar[j], 1);
    fence_mbar_init();
  }
  __syncwarp();
  // lane 0: bulk copies of a tile (and its pair table) into slot j
  auto issue = [&](const TileDesc& d, const TileGeo& g, int j) {
    meta[j] = d;
    const unsigned bytes = unsigned(g.hi - g.lo) * unsigned(sizeof(ST));
    const unsigned tbytes = ptab ? unsigned(TS * sizeof(ST)) : 0u;
    mbar_expect_tx(&bar[j], bytes + tbytes);
    if (bytes) bulk_g2s(buf + int64_t(j) * Lmax + (g.lo - g.base), u + g.off + g.lo, bytes, &bar[j]);
    if (tbytes) bulk_g2s(wtab + j * TS, ptab + int64_t(g.b) * TS, tbytes, &bar[j]);
  };
  // prologue: the first NS-1 tiles of this warp, edge values stored directly
  for (int j = 0; j < NS - 1; ++j) {
    const int64_t t = tile + int64_t(j) * nwarps;
    if (t >= a.ntiles) break;
    const TileDesc d = load_desc(a, t);
    const TileGeo gj = tile_geo<H, P, VW>(a, d);
    if (lane == 0) issue(d, gj, j);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int64_t src;
      const int q = edge_pos(gj, lane + 32 * e, &src);
      if (q >= 0) buf[int64_t(j) * Lmax + q] = __ldg(u + src);
    }
  }
  if (!ptab)  // one instance: one table, built once
    for (int e = lane; e < TE; e += 32) wtab[e] = pair_table_entry(W, a.w_stride, wq, NW, SCHEME, 0, e);
  TileDesc dnext{};  // descriptor of the next tile to fetch, loaded one tile ahead
  if (tile + int64_t(NS - 1) * nwarps < a.ntiles) dnext = load_desc(a, tile + int64_t(NS - 1) * nwarps);
  int pq[2] = {-1, -1};  // edge values loaded during the previous tile, stored after this one
  ST pv[2] = {ST(0), ST(0)};
  int s = 0;  // slot of the current tile
  unsigned parity = 0;  // parity of each slot's next wait
  bool abort = false;
  for (;;) {
    const int sf = s == 0 ? NS - 1 : s - 1;  // slot of the tile NS - 1 ahead, released when the previous tile ended
    const int64_t ftile = tile + int64_t(NS - 1) * nwarps;
    int eq[2] = {-1, -1};
    ST ev[2] = {ST(0), ST(0)};
    if (ftile < a.ntiles) {
      const TileGeo gf = tile_geo<H, P, VW>(a, dnext);
      if (lane == 0) issue(dnext, gf, sf);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        int64_t src;
        eq[e] = edge_pos(gf, lane + 32 * e, &src);
        if (eq[e] >= 0) ev[e] = __ldg(u + src);
      }
      if (ftile + nwarps < a.ntiles) dnext = load_desc(a, ftile + nwarps);
    }
    int ok = 1;
    if (lane == 0) ok = mbar_wait(&bar[s], (parity >> s) & 1u, a.wait_polls) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) {
      abort = true;
      break;
    }
    parity ^= 1u << s;
    const TileGeo g = tile_geo<H, P, VW>(a, meta[s]);
    const ST* cur = buf + int64_t(s) * Lmax;
    const T* wp = reinterpret_cast<const T*>(wtab + (ptab ? s * TS : 0));  // [k][phase][t]
    const int rounds = (g.len + OUTW - 1) / OUTW;
    ST* const obase = out + g.off + g.t0;
    if (SCHEME == 2) {
      T w0[2][NT], w1[2][NT], w2[2][NT];
#pragma unroll
      for (int ph = 0; ph < 2; ++ph)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          w0[ph][t] = wp[(0 * 2 + ph) * NT + t];
          w1[ph][t] = wp[(1 * 2 + ph) * NT + t];
          w2[ph][t] = wp[(2 * 2 + ph) * NT + t];
        }
      for (int r = 0; r < rounds; ++r) {
        // first stage on this lane's 4 points: a = W0 u + W1 N(u), D = N(a) - N(u)
        const int q = HR + r * OUTW + P * lane;
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
        // D window of the second stage: LH lanes on each side, then this lane
        T dw[WP];
        dw[2 * LH] = PO::sub(PO::mul(a01, PO::fma(a01, a01, M1)), nx[HR / 2]);
        dw[2 * LH + 1] = PO::sub(PO::mul(a23, PO::fma(a23, a23, M1)), nx[HR / 2 + 1]);
#pragma unroll
        for (int h = 1; h <= LH; ++h) {
          const int lo = lane - h < 0 ? lane : lane - h, hi = lane + h > 31 ? lane : lane + h;
          dw[2 * (LH - h)] = shfl_pair<ST>(dw[2 * LH], lo);
          dw[2 * (LH - h) + 1] = shfl_pair<ST>(dw[2 * LH + 1], lo);
          dw[2 * (LH + h)] = shfl_pair<ST>(dw[2 * LH], hi);
          dw[2 * (LH + h) + 1] = shfl_pair<ST>(dw[2 * LH + 1], hi);
        }
        // second stage: u+ = a + (W2 / dt) D on the inner lanes
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int st = OFF + p, i0 = st >> 1, ph = st & 1;
          T acc = ZERO;
#pragma unroll
          for (int t = 0; t < NT; ++t) acc = PO::fma(w2[ph][t], dw[i0 + t], acc);
          y[p] = PO::sum(acc);
        }
        const T o01 = PO::fma(PO::make(y[0], y[1]), INV, a01);
        const T o23 = PO::fma(PO::make(y[2], y[3]), INV, a23);
        const int idx = r * OUTW + P * (lane - LH);  // first updated point of this lane, from t0
        if (lane >= LH && lane < 32 - LH && idx < g.len) {
          if (idx + P <= g.len) {
            PO::store2(obase + idx, o01, o23);
            chk = PO::fma(o01, ZERO, chk);
            chk = PO::fma(o23, ZERO, chk);
          } else {
            ST v[4];
            PO::split(o01, v[0], v[1]);
            PO::split(o23, v[2], v[3]);
#pragma unroll
            for (int p = 0; p < P; ++p)
              if (idx + p < g.len) {
                obase[idx + p] = v[p];
                chk = PO::fma(PO::make(v[p], v[p]), ZERO, chk);
              }
          }
        }
      }
    } else {
      T w0[2][NT], w1[2][NT];
#pragma unroll
      for (int ph = 0; ph < 2; ++ph)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          w0[ph][t] = wp[(0 * 2 + ph) * NT + t];
          w1[ph][t] = SCHEME == 1 ? wp[(1 * 2 + ph) * NT + t] : ZERO;
        }
      for (int r = 0; r < rounds; ++r) {
        const int q = H + r * OUTW + P * lane;
        T x[WP], nx[WP];
        PO::template load<WP>(cur + q - HR, x);
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
            acc = PO::fma(w0[ph][t], x[i0 + t], acc);
            if (SCHEME == 1) acc = PO::fma(w1[ph][t], nx[i0 + t], acc);
          }
          y[p] = PO::sum(acc);
        }
        const T o01 = PO::make(y[0], y[1]), o23 = PO::make(y[2], y[3]);
        const int idx = r * OUTW + P * lane;
        if (idx < g.len) {
          if (idx + P <= g.len) {
            PO::store2(obase + idx, o01, o23);
            chk = PO::fma(o01, ZERO, chk);
            chk = PO::fma(o23, ZERO, chk);
          } else {
#pragma unroll
            for (int p = 0; p < P; ++p)
              if (idx + p < g.len) {
                obase[idx + p] = y[p];
                chk = PO::fma(PO::make(y[p], y[p]), ZERO, chk);
              }
          }
        }
      }
    }
    // the edge values loaded during the previous tile belong to the tile in
    // slot s - 2 (mod NS), which is not computed before the next tile
    const int ps = s >= 2 ? s - 2 : s + NS - 2;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (pq[e] >= 0) buf[int64_t(ps) * Lmax + pq[e]] = pv[e];
      pq[e] = eq[e];
      pv[e] = ev[e];
    }
    fence_proxy_async_smem();
    __syncwarp();  // slot s is free; the stored edge values are visible to the warp
    tile += nwarps;
    if (tile >= a.ntiles) break;
    s = s + 1 == NS ? 0 : s + 1;
  }
  if (abort && lane == 0) {
    // a bulk copy did not complete in time: report it and give the copies
    // still in flight (this tile and the next NS - 1) the default bounded
    // time to land, so that none writes into shared memory after the warp
    // has left
    atomicOr(flags, 2u);
    for (int d = 0; d < NS; ++d) {
      const int j = (s + d) % NS;
      if (tile + int64_t(d) * nwarps < a.ntiles) mbar_wait(&bar[j], (parity >> j) & 1u);
    }
  }
  ST c0, c1;
  PO::split(chk, c0, c1);
  if (!(c0 == ST(0) && c1 == ST(0))) atomicOr(flags, 1u);
}

template <typename ST, int SCHEME>
const void* pick_n(int n) {
  switch (n) {
    case 3: return (const void*)k_apply_stream<ST, SCHEME, 3>;
    case 5: return (const void*)k_apply_stream<ST, SCHEME, 5>;
    case 7: return (const void*)k_apply_stream<ST, SCHEME, 7>;
    case 9: return (const void*)k_apply_stream<ST, SCHEME, 9>;
    case 11: return (const void*)k_apply_stream<ST, SCHEME, 11>;
    case 13: return (const void*)k_apply_stream<ST, SCHEME, 13>;
    default: return (const void*)k_apply_stream<ST, SCHEME, 15>;
  }
}

template <typename ST>
const void* pick_scheme(int scheme, int n) {
  if (scheme == 0) return pick_n<ST, 0>(n);
  if (scheme == 1) return pick_n<ST, 1>(n);
  return pick_n<ST, 2>(n);
}

}  // namespace

const void* stream_kernel(int scheme, int n, bool mixed) {
  return mixed ? pick_scheme<float>(scheme, n) : pick_scheme<double>(scheme, n);
}

size_t stream_warp_smem(const ApplyParams& a, bool mixed, int stages, int scheme) {
  const size_t es = mixed ? 4 : 8;
  const int hr = ((a.n - 1) / 2 + 3) / 4 * 4;
  const int H = scheme == 2 ? 2 * hr : hr;
  const size_t bytes = STREAM_HEADER + size_t(stages) * size_t(pair_table_stride(a.n)) * es +
                       size_t(stages) * size_t(a.tile + 2 * H) * es;
  return (bytes + 127) / 128 * 128;
}

}  // namespace lmep
