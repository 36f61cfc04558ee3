// lmep_expm.cu -- kernels of steps (a1)-(a5) and the fused frozen-velocity step.
//
// One warp per matrix.  The derivative matrices of the uniform window are
// built once per CTA by Fornberg's recursion (a2) into shared memory; every
// warp then assembles its point's local matrix (a3), exponentiates it (a4)
// and harvests the needed rows (a5).  In the fused frozen-velocity kernel the
// harvested row is applied to the point's window at once (a6), so the weights
// never reach HBM.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "lmep_warp_kernel.cuh"

namespace lmep {

DeviceInfo device_info() {
  static thread_local int dev_cached = -1;
  static thread_local DeviceInfo info{0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != dev_cached) {
    cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&info.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    dev_cached = dev;
  }
  return info;
}

// ------------------------------------------------------------------ (a2) tables
// h^k D^(k) (k = 1..3) of the uniform window depend only on n: they are built
// once per device by Fornberg's recursion into these tables (slot (n - 3) / 2,
// FP64 and an FP32 copy); the expm kernels copy their n's table into shared
// memory instead of rebuilding it in every CTA.
constexpr int FB_SLOTS = (DMAX - 1) / 2;  // n = 3, 5, ..., 15
__device__ double g_fornberg[FB_SLOTS][3 * DMAX * LD];
__device__ float g_fornberg_f[FB_SLOTS][3 * DMAX * LD];

__global__ void k_fornberg_tables() {
  const int n = 3 + 2 * int(blockIdx.x);
  const int t = threadIdx.x;
  if (t < n) {
    double c[4][DMAX];
    fornberg_row(double(t), n, c);
    for (int k = 1; k <= 3; ++k)
      for (int j = 0; j < DMAX; ++j) {
        const double v = j < n ? c[k][j] : 0.0;
        g_fornberg[blockIdx.x][(k - 1) * DMAX * LD + t * LD + j] = v;
        g_fornberg_f[blockIdx.x][(k - 1) * DMAX * LD + t * LD + j] = float(v);
      }
  }
}

namespace {
std::mutex g_fb_mutex;
struct FbState {
  bool ready = false;
  double* d = nullptr;
  float* f = nullptr;
};
FbState g_fb[64];
}  // namespace

cudaError_t fornberg_init() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_fb_mutex);
  FbState& st = g_fb[dev];
  if (st.ready) return cudaSuccess;
  if ((e = cudaGetSymbolAddress(reinterpret_cast<void**>(&st.d), g_fornberg)) != cudaSuccess) return e;
  if ((e = cudaGetSymbolAddress(reinterpret_cast<void**>(&st.f), g_fornberg_f)) != cudaSuccess) return e;
  cudaStream_t s;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
  k_fornberg_tables<<<FB_SLOTS, 32, 0, s>>>();
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e == cudaSuccess) st.ready = true;
  return e;
}

cudaError_t fornberg_of(int n, const double** d, const float** f) {
  cudaError_t e = fornberg_init();
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);
  const int slot = (n - 3) / 2;
  *d = g_fb[dev].d + size_t(slot) * 3 * DMAX * LD;
  *f = g_fb[dev].f + size_t(slot) * 3 * DMAX * LD;
  return cudaSuccess;
}

// ------------------------------------------------------------------ (a1)-(a3)
template <int D>
__global__ void __launch_bounds__(32 * WARPS) k_build_operator(KParams p, const double* __restrict__ u,
                                                               int64_t i0, int64_t count, double* M,
                                                               int32_t* start, int32_t* row) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* Dh = reinterpret_cast<double*>(smem);
  double* X64 = reinterpret_cast<double*>(smem + DH_BYTES) + (threadIdx.x >> 5) * DMAX * LD;
  fornberg_block(Dh, p.n);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t step = int64_t(gridDim.x) * WARPS;
  for (int64_t t = int64_t(blockIdx.x) * WARPS + (threadIdx.x >> 5); t < count; t += step) {
    const int64_t i = i0 + t;
    const double ui = u ? u[i] : 0.0;
    const int k = (p.dep && u) ? departure_shift(ui, p.dt, p.h, p.n, p.dt_h) : 0;
    const int64_t st = window_start(i, p.N, p.n, p.bc, k);
    const int r = int(i - st);
    const double a1 = p.c1 - p.fa * ui;
    assemble<D>(X64, Dh, p.n, p.dt * p.c0, p.dt * a1 / p.h, p.dt * p.c2 / (p.h * p.h),
                p.dt * p.c3 / (p.h * p.h * p.h), lane);
    __syncwarp();
    augment(X64, p.n, p.n_phi, r, p.dt, lane);
    __syncwarp();
    for (int e = lane; e < D * D; e += 32) M[t * D * D + e] = X64[(e / D) * LD + e % D];
    if (lane == 0) {
      start[t] = int32_t(st);
      row[t] = r;
    }
    __syncwarp();
  }
}

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

static int persistent_grid(const void* kernel, int threads, size_t smem, int64_t work_items) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = int64_t(device_info().sms) * per_sm;
  const int64_t need = (work_items + WARPS - 1) / WARPS;
  return int(need < cap ? (need > 0 ? need : 1) : cap);
}

#define LMEP_DISPATCH_D(d, CALL)                 \
  switch (d) {                                   \
    case 3: { constexpr int D = 3; CALL; }       \
    case 4: { constexpr int D = 4; CALL; }       \
    case 5: { constexpr int D = 5; CALL; }       \
    case 6: { constexpr int D = 6; CALL; }       \
    case 7: { constexpr int D = 7; CALL; }       \
    case 8: { constexpr int D = 8; CALL; }       \
    case 9: { constexpr int D = 9; CALL; }       \
    case 10: { constexpr int D = 10; CALL; }     \
    case 11: { constexpr int D = 11; CALL; }     \
    case 12: { constexpr int D = 12; CALL; }     \
    case 13: { constexpr int D = 13; CALL; }     \
    case 14: { constexpr int D = 14; CALL; }     \
    case 15: { constexpr int D = 15; CALL; }     \
    case 16: { constexpr int D = 16; CALL; }     \
    default: return cudaErrorInvalidValue;       \
  }

template <int D>
static cudaError_t run_build(const KParams& p, const double* u, int64_t i0, int64_t count, double* M,
                             int32_t* start, int32_t* row, cudaStream_t s) {
  const size_t smem = DH_BYTES + WARPS * DMAX * LD * 8;
  auto k = k_build_operator<D>;
  cudaError_t e = prep(k, smem);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid((const void*)k, 32 * WARPS, smem, count);
  k<<<grid, 32 * WARPS, smem, s>>>(p, u, i0, count, M, start, row);
  return cudaGetLastError();
}

cudaError_t launch_build_operator(const KParams& p, const double* u, int64_t i0, int64_t count,
                                  double* M, int32_t* start, int32_t* row, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  LMEP_DISPATCH_D(p.n + p.n_phi, return run_build<D>(p, u, i0, count, M, start, row, s));
}

cudaError_t launch_expm(const double* A, int64_t P, int d, double* E, bool mixed, int32_t* ms,
                        cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  WarpJob job{};
  job.mode = MODE_FULL;
  job.items = P;
  job.A = A;
  job.E = E;
  job.ms = ms;
  return mixed ? warp_job_f32(d, job, s) : warp_job_f64(d, job, s);
}

cudaError_t launch_harvest_const(const KParams& p, const double* h_inst, int64_t B, void* W,
                                 bool mixed, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  WarpJob job{};
  job.mode = MODE_CONST;
  job.p = p;
  cudaError_t e = fornberg_of(p.n, &job.dh, &job.dhf);
  if (e != cudaSuccess) return e;
  job.items = B * p.n;
  job.h_inst = h_inst;
  job.out = W;
  return mixed ? warp_job_f32(p.n + p.n_phi, job, s) : warp_job_f64(p.n + p.n_phi, job, s);
}

cudaError_t launch_harvest_nodes(const KParams& p, const double* x, void* W, bool mixed, cudaStream_t s) {
  if (p.N <= 0) return cudaSuccess;
  WarpJob job{};
  job.mode = MODE_NODES;
  job.p = p;
  job.items = p.N;
  job.x = x;
  job.out = W;
  return mixed ? warp_job_f32(p.n + p.n_phi, job, s) : warp_job_f64(p.n + p.n_phi, job, s);
}

// exp(E) of the point-independent part E = c2h Dh2 + c3h Dh3 of a
// frozen-velocity local matrix: one warp, FP64 Pade scaling and squaring,
// row-major D x D into out; then Dh2 exp(E) (D x D) into out2, the direction
// of d exp(E) / d c2h (Dh2 commutes with E).
template <int D>
__global__ void __launch_bounds__(32) k_exp_const(KParams p, const double* dh, double* out, double* out2) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* Dh = reinterpret_cast<double*>(smem);
  Ws<double> w(smem + DH_BYTES);
  exp_const_warp<D>(p, dh, Dh, w, out, out2, threadIdx.x);
}

cudaError_t launch_exp_const(const KParams& p, double* out, double* out2, cudaStream_t s) {
  const double* d;
  const float* f;
  cudaError_t e = fornberg_of(p.n, &d, &f);
  if (e != cudaSuccess) return e;
  const size_t smem = DH_BYTES + Ws<double>::BYTES;
  switch (p.n) {
    case 3: k_exp_const<3><<<1, 32, smem, s>>>(p, d, out, out2); break;
    case 5: k_exp_const<5><<<1, 32, smem, s>>>(p, d, out, out2); break;
    case 7: k_exp_const<7><<<1, 32, smem, s>>>(p, d, out, out2); break;
    case 9: k_exp_const<9><<<1, 32, smem, s>>>(p, d, out, out2); break;
    case 11: k_exp_const<11><<<1, 32, smem, s>>>(p, d, out, out2); break;
    case 13: k_exp_const<13><<<1, 32, smem, s>>>(p, d, out, out2); break;
    case 15: k_exp_const<15><<<1, 32, smem, s>>>(p, d, out, out2); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_frozen(const KParams& p, const void* u, void* out, bool fused, bool mixed,
                          unsigned* flags, cudaStream_t s, int32_t* stats, const double* sl) {
  if (p.n_phi != 0) return cudaErrorInvalidValue;
  WarpJob job{};
  job.mode = fused ? MODE_FROZEN_STEP : MODE_FROZEN_W;
  job.p = p;
  if (sl) {
    job.sl = 1;
    for (int e = 0; e < p.n * p.n + p.n; ++e) {
      if (mixed) job.slt.f[e] = float(sl[e]);
      else job.slt.d[e] = sl[e];
    }
  }
  cudaError_t e = fornberg_of(p.n, &job.dh, &job.dhf);
  if (e != cudaSuccess) return e;
  job.items = p.N * (p.batch > 1 ? p.batch : 1);
  job.u = u;
  job.out = out;
  job.flags = flags;
  job.ms = stats;
  return mixed ? warp_job_f32(p.n, job, s) : warp_job_f64(p.n, job, s);
}

}  // namespace lmep
