// lmep_frozen_set.cu -- several frozen-velocity instances, one launch per step.
//
// Each instance has its own grid (N, h, boundary), stencil width n, operator
// and dt; every point rebuilds its local matrix X = a Dh1 + E at every step
// (Sec. 2.1 steps 1-3, a1-a6 fused).  Its row of exp(X) is taken from the
// factorisation row_r exp(X) = l(r + a)^T exp(E) (Thm. 1 with the General
// Exactness theorem: the derivative matrices of the window commute, and row r
// of exp(a Dh1) is the semi-Lagrangian interpolation at the departure point):
// the Lagrange weights of the window at the departure point times exp(E), which
// is the same for every point of an instance.  One step is two launches:
//
//   k_frozen_set           one CTA per tile of one instance (tiles of the widest
//                          stencils first), the tile's values and the instance's
//                          exp(E) table staged in shared memory, one thread per
//                          point (or two points sharing the table reads); a
//                          point whose error bound sum_j |l_j| R_j (R_j the
//                          absolute row sums of exp(E)) exceeds the bound of the
//                          factorised route is appended to its instance's list;
//   k_frozen_set_fallback  the listed points through the finite series of the
//                          nilpotent local matrix, then Pade scaling and
//                          squaring (one warp per 32 points, as in k_warp); it
//                          exits at once when no point was listed, and its last
//                          CTA clears the lists' counters for the next step.
//
// The lean kernel carries only the factorised route, so it needs no Pade
// workspace and few registers; the lists move the rare rejected points to the
// fallback without a host round trip, so a step can be replayed from a CUDA
// graph.  The exp(E) tables are computed on the device (k_frozen_set_setup,
// FP64 Pade, one warp per instance) with the same arithmetic as the
// single-instance path, so both give the same bits.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <queue>
#include <utility>
#include <vector>

#include "lmep_frozen_set.cuh"

namespace lmep {

namespace {
// exp(E) table of instance blockIdx.x: FP64 Pade (exp_const_warp, the
// arithmetic of the single-instance path) into exps, then in the product type
// its rows (stride NP) and absolute row sums; ok = 0 when exp(E) or Dh2 exp(E)
// is not finite (the instance then takes the fallback for every point).
template <int D, typename PT>
__device__ __forceinline__ void setup_one(const WarpJob& job, const SetInst& in, double* Dh, const Ws<double>& w,
                                          double* e, PT* tab, int32_t* ok, int lane) {
  constexpr int NP = tab_np(D);
  exp_const_warp<D>(job.p, job.dh, Dh, w, e, e + DMAX * DMAX, lane);
  bool finite = true;
  for (int q = lane; q < D * D; q += 32) finite = finite && isfinite(e[q]) && isfinite(e[DMAX * DMAX + q]);
  PT* t = tab + in.tab;
  if (lane < D) {
    double rs = 0.0;
    for (int k = 0; k < NP; ++k) {
      const double v = k < D ? e[lane * D + k] : 0.0;
      t[lane * NP + k] = PT(v);
      if (k < D) rs += fabs(v);
    }
    t[D * NP + lane] = PT(rs);
  } else if (lane < NP) {
    t[D * NP + lane] = PT(0);
  }
  finite = __all_sync(FULL, finite);
  if (lane == 0) ok[blockIdx.x] = finite ? 1 : 0;
}

template <typename PT>
__global__ void __launch_bounds__(32) k_frozen_set_setup(const WarpJob* jobs, SetInst* inst, double* exps,
                                                         void* tab, int32_t* ok) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* Dh = reinterpret_cast<double*>(smem);
  Ws<double> w(smem + DH_BYTES);
  const int b = blockIdx.x, lane = threadIdx.x;
  const WarpJob& job = jobs[b];
  double* e = exps + int64_t(b) * 2 * DMAX * DMAX;
  PT* t = static_cast<PT*>(tab);
  switch (job.p.n) {
    case 3: setup_one<3, PT>(job, inst[b], Dh, w, e, t, ok, lane); break;
    case 5: setup_one<5, PT>(job, inst[b], Dh, w, e, t, ok, lane); break;
    case 7: setup_one<7, PT>(job, inst[b], Dh, w, e, t, ok, lane); break;
    case 9: setup_one<9, PT>(job, inst[b], Dh, w, e, t, ok, lane); break;
    case 11: setup_one<11, PT>(job, inst[b], Dh, w, e, t, ok, lane); break;
    case 13: setup_one<13, PT>(job, inst[b], Dh, w, e, t, ok, lane); break;
    default: setup_one<15, PT>(job, inst[b], Dh, w, e, t, ok, lane); break;
  }
  if (lane == 0) inst[b].ok = ok[b];  // staged with the record by the lean kernel (lane 0 wrote ok[b])
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <typename K>
cudaError_t allow_smem(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}


// The lean kernel of a set and its shared memory: two staging buffers (table, tile and halo).
// points per thread and tile: 1 or 2 together in registers, or 4 / 8 as 1 / 2 together, four times in turn
template <typename PT>
auto set_kernel(int ppt) {
  return ppt == 8 ? k_frozen_set<PT, 2, 4>
                  : (ppt == 4 ? k_frozen_set<PT, 1, 4> : (ppt == 2 ? k_frozen_set<PT, 2, 1> : k_frozen_set<PT, 1, 1>));
}
template <typename PT>
size_t set_smem(const SetLayout& L) {
  return 2 * (size_t(TAB_MAX) + size_t(L.block) * L.ppt + 2 * DMAX) * sizeof(PT);
}
// Persistent grid: every CTA that fits on the device at once (at most one per tile).
template <typename PT>
cudaError_t set_grid(SetLayout& L) {
  auto kern = set_kernel<PT>(L.ppt);
  const size_t smem = set_smem<PT>(L);
  cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L.block, smem)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  L.grid = int(L.ntiles < cap ? L.ntiles : cap);
  return cudaSuccess;
}


}  // namespace

SetLayout frozen_set_layout(int64_t B, const int32_t* n, const int64_t* N, int block, int ppt, bool mixed) {
  SetLayout L{};
  const size_t es = mixed ? 4 : 8;
  const int64_t tp = int64_t(block) * ppt;
  int64_t tiles = 0, points = 0, tabn = 0;
  for (int64_t b = 0; b < B; ++b) {
    tiles += (N[b] + tp - 1) / tp;
    points += N[b];
    tabn += tab_elems(n[b]);
  }
  L.B = B;
  L.ntiles = tiles;
  L.points = points;
  L.block = block;
  L.ppt = ppt;
  L.mixed = mixed;
  L.ctl = 0;
  L.ok = align256(L.ctl + size_t(B + 2) * 4);  // counts, done, total
  L.inst = align256(L.ok + size_t(B) * 4);
  L.jobs = align256(L.inst + size_t(B) * sizeof(SetInst));
  L.tiles = align256(L.jobs + size_t(B) * sizeof(WarpJob));
  L.starts = align256(L.tiles + size_t(tiles) * sizeof(SetTile));
  L.exps = align256(L.starts + size_t(tiles + 1) * 4);  // the grid never exceeds the tile count
  L.tab = align256(L.exps + size_t(B) * 2 * DMAX * DMAX * 8);
  L.lists = align256(L.tab + size_t(tabn) * es);
  L.total = align256(L.lists + size_t(points) * 4);
  return L;
}

cudaError_t frozen_set_prepare(void* ws, SetLayout& L, const KParams* p, const int32_t* route,
                               const int64_t* offsets, cudaStream_t s) {
  cudaError_t e0 = L.mixed ? set_grid<float>(L) : set_grid<double>(L);
  if (e0 != cudaSuccess) return e0;
  char* base = static_cast<char*>(ws);
  std::vector<SetInst> inst(size_t(L.B));
  std::vector<WarpJob> jobs(size_t(L.B));
  std::vector<SetTile> tiles;
  tiles.reserve(size_t(L.ntiles));
  int64_t list_off = 0, tab = 0;
  const int64_t tp = int64_t(L.block) * L.ppt;
  for (int64_t b = 0; b < L.B; ++b) {
    SetInst& in = inst[size_t(b)];
    std::memset(&in, 0, sizeof in);
    in.p = p[b];
    in.off = offsets[b];
    in.list_off = list_off;
    in.tab = tab;
    in.route = route[b];
    list_off += p[b].N;
    tab += tab_elems(p[b].n);
    WarpJob& j = jobs[size_t(b)];
    std::memset(&j, 0, sizeof j);
    j.mode = MODE_FROZEN_STEP;
    j.p = p[b];
    j.items = p[b].N;
    cudaError_t e = fornberg_of(p[b].n, &j.dh, &j.dhf);
    if (e != cudaSuccess) return e;
  }
  // Tiles to CTAs, longest processing time first: tiles in decreasing estimated
  // cost (points x (n^2 + 8n + 40), the row product, weights, bound and apply),
  // each to the CTA with the least work so far; a CTA's tiles are stored
  // together, heaviest first, from starts[c] to starts[c + 1].
  struct Job {
    double cost;
    int64_t b, t0;
  };
  std::vector<Job> work;
  work.reserve(size_t(L.ntiles));
  for (int64_t b = 0; b < L.B; ++b) {
    const double w = double(p[b].n) * p[b].n + 8.0 * p[b].n + 40.0;
    for (int64_t t0 = 0; t0 < p[b].N; t0 += tp) work.push_back({w * double(std::min(tp, p[b].N - t0)), b, t0});
  }
  std::stable_sort(work.begin(), work.end(), [](const Job& x, const Job& y) { return x.cost > y.cost; });
  const int G = L.grid;
  std::vector<std::vector<int64_t>> runs(static_cast<size_t>(G));
  using Load = std::pair<double, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int c = 0; c < G; ++c) heap.push({0.0, c});
  for (size_t q = 0; q < work.size(); ++q) {
    Load top = heap.top();
    heap.pop();
    runs[size_t(top.second)].push_back(int64_t(q));
    top.first += work[q].cost;
    heap.push(top);
  }
  std::vector<int32_t> starts(size_t(G) + 1, 0);
  for (int c = 0; c < G; ++c) {
    starts[size_t(c)] = int32_t(tiles.size());
    for (int64_t q : runs[size_t(c)]) {
      const Job& j = work[size_t(q)];
      SetTile t{};
      t.off = inst[size_t(j.b)].off;
      t.N = int32_t(p[j.b].N);
      t.t0 = int32_t(j.t0);
      t.b = int32_t(j.b);
      t.n = p[j.b].n;
      t.bc = p[j.b].bc;
      t.tab = int32_t(inst[size_t(j.b)].tab);
      tiles.push_back(t);
    }
  }
  starts[size_t(G)] = int32_t(tiles.size());
  cudaError_t e;
  if ((e = cudaMemsetAsync(base + L.ctl, 0, size_t(L.B + 2) * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(base + L.inst, inst.data(), inst.size() * sizeof(SetInst), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(base + L.jobs, jobs.data(), jobs.size() * sizeof(WarpJob), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(base + L.tiles, tiles.data(), tiles.size() * sizeof(SetTile), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(base + L.starts, starts.data(), starts.size() * 4, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = frozen_set_refresh(ws, L, s)) != cudaSuccess) return e;
  // the host copies above read pageable vectors: make sure they are consumed
  return cudaStreamSynchronize(s);
}

cudaError_t frozen_set_refresh(void* ws, const SetLayout& L, cudaStream_t s) {
  char* base = static_cast<char*>(ws);
  const size_t smem = DH_BYTES + Ws<double>::BYTES;
  const WarpJob* jobs = reinterpret_cast<const WarpJob*>(base + L.jobs);
  SetInst* inst = reinterpret_cast<SetInst*>(base + L.inst);
  double* exps = reinterpret_cast<double*>(base + L.exps);
  int32_t* ok = reinterpret_cast<int32_t*>(base + L.ok);
  if (L.mixed) {
    cudaError_t e = allow_smem(k_frozen_set_setup<float>, smem);
    if (e != cudaSuccess) return e;
    k_frozen_set_setup<float><<<unsigned(L.B), 32, smem, s>>>(jobs, inst, exps, base + L.tab, ok);
  } else {
    cudaError_t e = allow_smem(k_frozen_set_setup<double>, smem);
    if (e != cudaSuccess) return e;
    k_frozen_set_setup<double><<<unsigned(L.B), 32, smem, s>>>(jobs, inst, exps, base + L.tab, ok);
  }
  return cudaGetLastError();
}

namespace {
template <typename PT>
cudaError_t set_step(char* base, const SetLayout& L, const void* u_in, void* u_out, unsigned* flags, cudaStream_t s) {
  SetArgs a;
  a.inst = reinterpret_cast<const SetInst*>(base + L.inst);
  a.tiles = reinterpret_cast<const SetTile*>(base + L.tiles);
  a.starts = reinterpret_cast<const int32_t*>(base + L.starts);
  a.tab = base + L.tab;
  a.ok = reinterpret_cast<const int32_t*>(base + L.ok);
  a.fail_count = reinterpret_cast<int32_t*>(base + L.ctl);
  a.fail_total = a.fail_count + L.B + 1;
  a.fail_list = reinterpret_cast<int32_t*>(base + L.lists);
  a.u = u_in;
  a.out = u_out;
  a.flags = flags;
  cudaError_t e;
  if ((e = launch_pdl(set_kernel<PT>(L.ppt), unsigned(L.grid), unsigned(L.block), set_smem<PT>(L), s, a)) !=
      cudaSuccess)
    return e;
  FbArgs f;
  f.inst = a.inst;
  f.jobs = reinterpret_cast<const WarpJob*>(base + L.jobs);
  f.fail_count = a.fail_count;
  f.fail_total = a.fail_total;
  f.fail_list = a.fail_list;
  f.done = reinterpret_cast<unsigned*>(base + L.ctl) + L.B;
  f.B = L.B;
  f.u = u_in;
  f.out = u_out;
  f.flags = flags;
  const unsigned fgrid = unsigned(device_info().sms);
  return sizeof(PT) == 4 ? launch_set_fallback_f32(f, fgrid, s) : launch_set_fallback_f64(f, fgrid, s);
}
}  // namespace

cudaError_t frozen_set_step(void* ws, const SetLayout& L, const void* u_in, void* u_out, unsigned* flags,
                            cudaStream_t s) {
  char* base = static_cast<char*>(ws);
  return L.mixed ? set_step<float>(base, L, u_in, u_out, flags, s) : set_step<double>(base, L, u_in, u_out, flags, s);
}

}  // namespace lmep
