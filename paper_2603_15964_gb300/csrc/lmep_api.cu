// lmep_api.cu -- the C ABI of include/lmep.h: argument checks, dispatch,
// status flags and the batch workspace.  All compute runs in the kernels of
// lmep_expm.cu, lmep_apply.cu and lmep_adjoint.cu.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lmep.h"
#include "lmep_internal.h"

using lmep::ApplyParams;
using lmep::Instance;
using lmep::KParams;
using lmep::make_params;

struct BatchPlan {
  ApplyParams ap;
  const void* W;     // per-instance weights inside the workspace
  int64_t points;    // total points of the batch
  int grid, block;
  bool mixed;
  size_t bytes;
};

struct lmep_handle {
  int device;
  unsigned* flags;  // device status word: bit 0 = non-finite output, bit 1 = a bounded wait gave up
  int32_t expm_method = LMEP_EXPM_AUTO;  // frozen-velocity rows (lmep_set_expm_method)
  int32_t wait_polls = 1 << 20;          // bound of the streaming apply's waits (lmep_set_wait_limit)
  // factorised frozen-velocity rows: exp(E) per (n, c2h, c3h) of a frozen operator (FP64, n x n,
  // the n absolute row sums, then Dh2 exp(E) n x n for the adjoint), computed once on the device
  // (sl_scratch) and kept on the host
  double* sl_scratch = nullptr;
  std::mutex sl_mu;
  std::map<std::tuple<int, uint64_t, uint64_t>, std::vector<double>> sl_cache;
  std::map<const void*, BatchPlan> plans;
  std::map<const void*, lmep::SetLayout> sets;  // prepared frozen-velocity sets, by workspace
};

namespace {

thread_local std::string g_last_error;

lmep_status fail(lmep_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
lmep_status cuda_fail(cudaError_t e, const char* where) {
  return fail(LMEP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(call, where)                          \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

// wide: the entry point also takes the wide stencils (odd n = 17 .. 25) of the
// constant-coefficient linear scheme (lmep_wide.cu)
lmep_status check_grid(const lmep_grid* g, int n_phi, bool wide = false) {
  if (!g) return fail(LMEP_ERR_INVALID, "grid is NULL");
  if (wide && n_phi == 0 && lmep::wide_width(g->n)) {
    if (g->N < g->n) return fail(LMEP_ERR_INVALID, "N must be >= n");
    if (g->N > (int64_t(1) << 40)) return fail(LMEP_ERR_INVALID, "N too large");
    if (!(g->h > 0.0)) return fail(LMEP_ERR_INVALID, "h must be positive");
    if (g->bc < 0 || g->bc > 2) return fail(LMEP_ERR_INVALID, "unknown boundary condition");
    if (g->batch > 1) return fail(LMEP_ERR_UNSUPPORTED, "wide stencils take batch <= 1");
    if (g->window_shift < -(g->n - 1) / 2 || g->window_shift > (g->n - 1) / 2)
      return fail(LMEP_ERR_INVALID, "|window_shift| must be <= (n-1)/2");
    if (g->reserved != 0) return fail(LMEP_ERR_INVALID, "lmep_grid.reserved must be 0");
    return LMEP_OK;
  }
  if (lmep::wide_width(g->n))
    return fail(LMEP_ERR_UNSUPPORTED, "n = 17..25 is built for the constant-coefficient linear scheme only");
  if (g->n < 3 || g->n > 15 || (g->n % 2) == 0) return fail(LMEP_ERR_INVALID, "n must be odd, 3..15 (17..25: linear)");
  if (g->N < g->n) return fail(LMEP_ERR_INVALID, "N must be >= n");
  if (g->N > (int64_t(1) << 40)) return fail(LMEP_ERR_INVALID, "N too large");
  if (!(g->h > 0.0)) return fail(LMEP_ERR_INVALID, "h must be positive");
  if (g->bc < 0 || g->bc > 2) return fail(LMEP_ERR_INVALID, "unknown boundary condition");
  if (g->batch < 0) return fail(LMEP_ERR_INVALID, "batch must be >= 0");
  if (g->N * (g->batch > 1 ? g->batch : 1) > (int64_t(1) << 40)) return fail(LMEP_ERR_INVALID, "batch * N too large");
  if (n_phi < 0 || n_phi > 3) return fail(LMEP_ERR_INVALID, "n_phi must be 0, 1, 2 or 3");
  if (g->n + n_phi > 16) return fail(LMEP_ERR_UNSUPPORTED, "n + n_phi must be <= 16");
  if (g->window_shift < -(g->n - 1) / 2 || g->window_shift > (g->n - 1) / 2)
    return fail(LMEP_ERR_INVALID, "|window_shift| must be <= (n-1)/2");
  if (g->reserved != 0) return fail(LMEP_ERR_INVALID, "lmep_grid.reserved must be 0");
  return LMEP_OK;
}

lmep_status no_shift(const lmep_grid* g) {
  if (g->window_shift != 0) return fail(LMEP_ERR_UNSUPPORTED, "window_shift is for constant-coefficient linear steps");
  return LMEP_OK;
}

lmep_status check_prec(int32_t precision) {
  if (precision != LMEP_PREC_FP64 && precision != LMEP_PREC_MIXED)
    return fail(LMEP_ERR_INVALID, "precision must be LMEP_PREC_FP64 or LMEP_PREC_MIXED");
  return LMEP_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

uint64_t bits_of(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
}

// exp(E), E = c2h Dh2 + c3h Dh3, of a frozen operator for the factorised rows (n x n FP64,
// the n absolute row sums, then Dh2 exp(E) n x n), from the handle's cache or computed now:
// one FP64 Pade launch on `stream` and a synchronisation, so only outside a stream
// capture.  *table = nullptr when it is not available (capture, cache full, non-finite);
// the rows then take the finite series.
lmep_status sl_table(lmep_handle* h, const KParams& p, cudaStream_t stream, const double** table) {
  *table = nullptr;
  const auto key = std::make_tuple(p.n, bits_of(p.c2h), bits_of(p.c3h));
  std::lock_guard<std::mutex> lock(h->sl_mu);
  auto it = h->sl_cache.find(key);
  if (it != h->sl_cache.end()) {
    *table = it->second.empty() ? nullptr : it->second.data();
    return LMEP_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(stream, &cs), "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone || h->sl_cache.size() >= 4096) return LMEP_OK;
  if (!h->sl_scratch) CK(cudaMalloc(&h->sl_scratch, sizeof(double) * 2 * 16 * 16), "cudaMalloc(exp table)");
  CK(lmep::launch_exp_const(p, h->sl_scratch, h->sl_scratch + 16 * 16, stream), "exp(E)");
  const int n = p.n;
  std::vector<double> e(size_t(n) * n), d2(size_t(n) * n);
  CK(cudaMemcpyAsync(e.data(), h->sl_scratch, sizeof(double) * n * n, cudaMemcpyDeviceToHost, stream), "read exp(E)");
  CK(cudaMemcpyAsync(d2.data(), h->sl_scratch + 16 * 16, sizeof(double) * n * n, cudaMemcpyDeviceToHost, stream),
     "read D2 exp(E)");
  CK(cudaStreamSynchronize(stream), "exp(E)");
  std::vector<double> t(size_t(n) * n + n + size_t(n) * n);
  bool finite = true;
  for (int j = 0; j < n; ++j) {
    double rs = 0.0;
    for (int k = 0; k < n; ++k) {
      const double v = e[size_t(j) * n + k];
      finite = finite && std::isfinite(v);
      t[size_t(j) * n + k] = v;
      rs += std::fabs(v);
    }
    t[size_t(n) * n + j] = rs;
  }
  for (size_t q = 0; q < size_t(n) * n; ++q) {
    finite = finite && std::isfinite(d2[q]);
    t[size_t(n) * n + n + q] = d2[q];
  }
  if (!finite) t.clear();  // remembered: this operator takes the finite series
  auto ins = h->sl_cache.emplace(key, std::move(t)).first;
  *table = ins->second.empty() ? nullptr : ins->second.data();
  return LMEP_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int default_tile(bool mixed) { return mixed ? 2048 : 1024; }
// staged points per warp tile of the streaming kernel (4 slots per warp fit)
int default_fast_tile(bool mixed) { return mixed ? 1024 : 512; }

}  // namespace

namespace lmep {
KParams make_params(const lmep_grid* g, const lmep_operator* op, double dt, int n_phi) {
  KParams p{};
  p.N = g->N;
  p.batch = g->batch > 1 ? g->batch : 1;
  p.h = g->h;
  p.bc = g->bc;
  p.n = g->n;
  p.dep = g->departure_centring ? 1 : 0;
  p.n_phi = n_phi;
  p.bc_lo = g->bc_lo;
  p.bc_hi = g->bc_hi;
  p.dt = dt;
  p.c0 = op->c0;
  p.c1 = op->c1;
  p.c2 = op->c2;
  p.c3 = op->c3;
  p.fa = op->frozen_adv;
  p.dt_h = dt / g->h;
  p.c0dt = dt * op->c0;
  p.c2h = dt * op->c2 / (g->h * g->h);
  p.c3h = dt * op->c3 / (g->h * g->h * g->h);
  p.c0dt_f = float(p.c0dt);
  p.c2h_f = float(p.c2h);
  p.c3h_f = float(p.c3h);
  p.c1_f = float(p.c1);
  p.fa_f = float(p.fa);
  p.dt_h_f = float(p.dt_h);
  return p;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace lmep

extern "C" {

const char* lmep_version(void) { return "lmep-gb300 0.1 (sm_103a)"; }

const char* lmep_last_error(void) { return g_last_error.c_str(); }

const char* lmep_status_string(lmep_status s) {
  switch (s) {
    case LMEP_OK: return "ok";
    case LMEP_ERR_INVALID: return "invalid argument";
    case LMEP_ERR_CUDA: return "CUDA error";
    case LMEP_ERR_NONFINITE: return "non-finite result";
    case LMEP_ERR_TIMEOUT: return "timeout";
    case LMEP_ERR_UNSUPPORTED: return "unsupported shape";
    case LMEP_ERR_NOMEM: return "workspace too small";
  }
  return "unknown status";
}

lmep_status lmep_create(lmep_handle** out) {
  if (!out) return fail(LMEP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  unsigned* flags = nullptr;
  CK(cudaMalloc(&flags, 256), "cudaMalloc(status)");
  cudaError_t e = cudaMemset(flags, 0, 256);
  if (e != cudaSuccess) {
    cudaFree(flags);
    return cuda_fail(e, "cudaMemset(status)");
  }
  e = lmep::fornberg_init();  // before any stream capture that may use the handle
  if (e != cudaSuccess) {
    cudaFree(flags);
    return cuda_fail(e, "derivative tables");
  }
  lmep_handle* h = new lmep_handle();
  h->device = dev;
  h->flags = flags;
  *out = h;
  return LMEP_OK;
}

lmep_status lmep_destroy(lmep_handle* h) {
  if (!h) return LMEP_OK;
  cudaFree(h->flags);
  if (h->sl_scratch) cudaFree(h->sl_scratch);
  delete h;
  return LMEP_OK;
}

lmep_status lmep_build_operator(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, double dt,
                                int32_t n_phi, const double* u_dev, int64_t i0, int64_t count,
                                double* M_dev, int32_t* start_dev, int32_t* row_dev, void* stream) {
  if (!h || !op) return fail(LMEP_ERR_INVALID, "handle/operator is NULL");
  lmep_status st = check_grid(g, n_phi);
  if (st != LMEP_OK) return st;
  if (g->batch > 1) return fail(LMEP_ERR_UNSUPPORTED, "lmep_build_operator takes batch <= 1");
  if (count < 0 || i0 < 0 || i0 + count > g->N) return fail(LMEP_ERR_INVALID, "point range outside grid");
  if (count == 0) return LMEP_OK;
  if (!M_dev || !start_dev || !row_dev) return fail(LMEP_ERR_INVALID, "output pointer is NULL");
  if (op->frozen_adv != 0.0 && !u_dev) return fail(LMEP_ERR_INVALID, "frozen operator needs u_dev");
  CK(lmep::launch_build_operator(make_params(g, op, dt, n_phi), u_dev, i0, count, M_dev, start_dev,
                                 row_dev, S(stream)),
     "build_operator");
  return LMEP_OK;
}

lmep_status lmep_expm(lmep_handle* h, const double* A_dev, int64_t P, int32_t d, double* E_dev,
                      int32_t precision, int32_t* ms_dev, void* stream) {
  if (!h) return fail(LMEP_ERR_INVALID, "handle is NULL");
  if (d < 3 || d > 16) return fail(LMEP_ERR_UNSUPPORTED, "d must be 3..16");
  if (P < 0) return fail(LMEP_ERR_INVALID, "P < 0");
  lmep_status st = check_prec(precision);
  if (st != LMEP_OK) return st;
  if (P == 0) return LMEP_OK;
  if (!A_dev || !E_dev) return fail(LMEP_ERR_INVALID, "NULL matrix pointer");
  CK(lmep::launch_expm(A_dev, P, d, E_dev, precision == LMEP_PREC_MIXED, ms_dev, S(stream)), "expm");
  return LMEP_OK;
}

lmep_status lmep_harvest_weights(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, double dt,
                                 int32_t n_phi, const void* u_frozen_dev, void* W_dev, int32_t precision,
                                 void* stream) {
  if (!h || !op || !W_dev) return fail(LMEP_ERR_INVALID, "NULL handle/operator/W");
  lmep_status st = check_grid(g, n_phi, true);
  if (st != LMEP_OK) return st;
  st = check_prec(precision);
  if (st != LMEP_OK) return st;
  if (!(dt > 0.0)) return fail(LMEP_ERR_INVALID, "dt must be positive");
  const KParams p = make_params(g, op, dt, n_phi);
  const bool mixed = precision == LMEP_PREC_MIXED;
  if (g->n > 15) {
    // wide stencils: constant coefficients, rows of exp(X) only (factorised form, lmep_wide.cu)
    if (u_frozen_dev || op->frozen_adv != 0.0)
      return fail(LMEP_ERR_UNSUPPORTED, "wide stencils (n > 15) take constant coefficients");
    CK(lmep::launch_harvest_wide(p, W_dev, mixed, S(stream)), "harvest(wide)");
    return LMEP_OK;
  }
  if (u_frozen_dev) {
    if ((st = no_shift(g)) != LMEP_OK) return st;
    if (n_phi != 0) return fail(LMEP_ERR_INVALID, "frozen-velocity weights need n_phi == 0");
    if (g->bc == LMEP_BC_NEUMANN && g->N < 2 * g->n) return fail(LMEP_ERR_UNSUPPORTED, "Neumann frozen weights need N >= 2n");
    KParams pf = p;
    pf.series = h->expm_method != LMEP_EXPM_PADE;
    const double* sl = nullptr;
    if (h->expm_method == LMEP_EXPM_AUTO && (st = sl_table(h, pf, S(stream), &sl)) != LMEP_OK) return st;
    CK(lmep::launch_frozen(pf, u_frozen_dev, W_dev, false, mixed, h->flags, S(stream), nullptr, sl),
       "harvest(frozen)");
    return LMEP_OK;
  }
  if (op->frozen_adv != 0.0) return fail(LMEP_ERR_INVALID, "frozen operator needs u_frozen_dev");
  if (g->batch > 1) return fail(LMEP_ERR_UNSUPPORTED, "constant-coefficient harvest takes batch <= 1");
  CK(lmep::launch_harvest_const(p, nullptr, 1, W_dev, mixed, S(stream)), "harvest(constant)");
  return LMEP_OK;
}

lmep_status lmep_harvest_scheme_weights(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, double dt,
                                        int32_t scheme, void* W_dev, int32_t precision, void* stream) {
  if (!h || !op || !W_dev) return fail(LMEP_ERR_INVALID, "NULL handle/operator/W");
  if (scheme < 0 || scheme > 3) return fail(LMEP_ERR_INVALID, "unknown scheme");
  lmep_status st = check_grid(g, scheme);
  if (st != LMEP_OK) return st;
  if ((st = check_prec(precision)) != LMEP_OK) return st;
  if (!(dt > 0.0)) return fail(LMEP_ERR_INVALID, "dt must be positive");
  if (op->frozen_adv != 0.0) return fail(LMEP_ERR_INVALID, "stored weights need a constant operator");
  if (g->batch > 1) return fail(LMEP_ERR_UNSUPPORTED, "constant-coefficient harvest takes batch <= 1");
  const bool mixed = precision == LMEP_PREC_MIXED;
  if (scheme < 3) {
    CK(lmep::launch_harvest_const(make_params(g, op, dt, scheme), nullptr, 1, W_dev, mixed, S(stream)), "harvest");
    return LMEP_OK;
  }
  // ETDRK4: rows of exp(dt L), dt alpha, dt beta, dt gamma (augmented, p = 3, at dt), then
  // exp(dt L / 2) and (dt/2) phi_1(dt L / 2) (augmented, p = 1, at dt/2): 6 rows per row class
  KParams p = make_params(g, op, dt, 3);
  p.w_rows = 6;
  p.rk4 = 1;
  CK(lmep::launch_harvest_const(p, nullptr, 1, W_dev, mixed, S(stream)), "harvest(etdrk4, dt)");
  KParams q = make_params(g, op, 0.5 * dt, 1);
  q.w_rows = 6;
  q.w_row0 = 4;
  CK(lmep::launch_harvest_const(q, nullptr, 1, W_dev, mixed, S(stream)), "harvest(etdrk4, dt/2)");
  return LMEP_OK;
}

lmep_status lmep_step(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, int32_t scheme,
                      int32_t nonlin, double dt, const void* W_dev, void* u_dev, void* work_dev,
                      int64_t nsteps, int32_t precision, void* stream) {
  if (!h || !op) return fail(LMEP_ERR_INVALID, "NULL handle/operator");
  if (scheme < 0 || scheme > 3) return fail(LMEP_ERR_INVALID, "unknown scheme");
  if (nonlin < 0 || nonlin > 3) return fail(LMEP_ERR_INVALID, "unknown nonlinearity");
  if ((scheme == 0) != (nonlin == 0)) return fail(LMEP_ERR_INVALID, "linear scheme <=> no nonlinearity");
  lmep_status st = check_grid(g, scheme, true);
  if (st != LMEP_OK) return st;
  st = check_prec(precision);
  if (st != LMEP_OK) return st;
  if (nsteps < 0) return fail(LMEP_ERR_INVALID, "nsteps < 0");
  if (!u_dev || !work_dev) return fail(LMEP_ERR_INVALID, "NULL state buffer");
  if (u_dev == work_dev) return fail(LMEP_ERR_INVALID, "u_dev and work_dev must differ");
  if (!(dt > 0.0)) return fail(LMEP_ERR_INVALID, "dt must be positive");
  if (nsteps == 0) return LMEP_OK;
  const bool mixed = precision == LMEP_PREC_MIXED;
  const size_t es = mixed ? 4 : 8;
  void* cur = u_dev;
  void* nxt = work_dev;
  if (g->n > 15) {
    // wide stencils: stored rows of the linear scheme on a periodic grid (lmep_wide.cu)
    if (!W_dev || op->frozen_adv != 0.0) return fail(LMEP_ERR_UNSUPPORTED, "wide stencils (n > 15) take stored rows");
    if (g->bc != LMEP_BC_PERIODIC) return fail(LMEP_ERR_UNSUPPORTED, "wide stencils (n > 15) step periodic grids");
    for (int64_t t = 0; t < nsteps; ++t) {
      CK(lmep::launch_apply_wide(g->N, g->n, g->window_shift, W_dev, cur, nxt, mixed, h->flags, S(stream)),
         "step(wide)");
      std::swap(cur, nxt);
    }
    if (cur != u_dev) CK(cudaMemcpyAsync(u_dev, cur, size_t(g->N) * es, cudaMemcpyDeviceToDevice, S(stream)), "copy");
    return LMEP_OK;
  }
  if (!W_dev) {
    if ((st = no_shift(g)) != LMEP_OK) return st;
    if (scheme != 0) return fail(LMEP_ERR_INVALID, "frozen-velocity stepping uses the linear scheme");
    if (g->bc == LMEP_BC_NEUMANN && g->N < 2 * g->n) return fail(LMEP_ERR_UNSUPPORTED, "Neumann frozen step needs N >= 2n");
    if (op->frozen_adv == 0.0) return fail(LMEP_ERR_INVALID, "W_dev is NULL but the operator is not frozen");
    KParams p = make_params(g, op, dt, 0);
    p.series = h->expm_method != LMEP_EXPM_PADE;
    const double* sl = nullptr;
    if (h->expm_method == LMEP_EXPM_AUTO && (st = sl_table(h, p, S(stream), &sl)) != LMEP_OK) return st;
    for (int64_t t = 0; t < nsteps; ++t) {
      CK(lmep::launch_frozen(p, cur, nxt, true, mixed, h->flags, S(stream), nullptr, sl), "step(frozen)");
      std::swap(cur, nxt);
    }
  } else {
    if (op->frozen_adv != 0.0) return fail(LMEP_ERR_INVALID, "stored weights need a constant operator");
    if (g->batch > 1) return fail(LMEP_ERR_UNSUPPORTED, "stored-weight stepping takes batch <= 1 (use lmep_batch_*)");
    if (scheme != 0 && (st = no_shift(g)) != LMEP_OK) return st;
    if (scheme == 3) {
      // ETDRK4: the CTA-tiled four-stage kernel, every boundary condition and nonlinearity
      const int H = lmep::rk4_halo(g->n, nonlin, g->bc);
      if (g->bc == LMEP_BC_NEUMANN && g->N < 2 * H + 8) return fail(LMEP_ERR_UNSUPPORTED, "N too small for the halo");
      if (g->bc == LMEP_BC_PERIODIC && g->N < H + 8) return fail(LMEP_ERR_UNSUPPORTED, "N too small for the halo");
      for (int64_t t = 0; t < nsteps; ++t) {
        CK(lmep::launch_apply_rk4(g->N, g->h, g->bc, g->n, nonlin, dt, g->bc_lo, g->bc_hi, cur, nxt, W_dev, mixed,
                                  h->flags, S(stream)),
           "step(etdrk4)");
        std::swap(cur, nxt);
      }
      if (cur != u_dev)
        CK(cudaMemcpyAsync(u_dev, cur, size_t(g->N) * es, cudaMemcpyDeviceToDevice, S(stream)), "copy");
      return LMEP_OK;
    }
    if (nonlin >= 2 && g->bc != LMEP_BC_PERIODIC)
      return fail(LMEP_ERR_UNSUPPORTED, "KdV and Burgers terms with ETD1/ETDRK2 need a periodic grid");
    // the pipelined kernel copies 16-byte aligned blocks of the state
    const bool fast = nonlin < 2 && g->bc != LMEP_BC_DIRICHLET && g->window_shift == 0 && aligned16(cur) &&
                      aligned16(nxt);
    const int H = fast ? lmep::apply_fast_halo(g->n, scheme)
                       : lmep::apply_halo(g->n, scheme, nonlin, g->bc) + std::abs(int(g->window_shift));
    if (g->bc == LMEP_BC_NEUMANN && g->N < 2 * H + 8) return fail(LMEP_ERR_UNSUPPORTED, "N too small for the halo");
    if (g->bc == LMEP_BC_PERIODIC && g->N < H + 8) return fail(LMEP_ERR_UNSUPPORTED, "N too small for the halo");
    ApplyParams a{};
    a.halo = H;
    a.shift = g->window_shift;
    a.fast = fast ? 1 : 0;
    a.n = g->n;
    a.scheme = scheme;
    a.nonlin = nonlin;
    a.tile = fast ? lmep::fast_tile_out(default_fast_tile(mixed), g->n, scheme) : default_tile(mixed);
    if (g->bc == LMEP_BC_DIRICHLET && a.tile < 4 * g->n) a.tile = 4 * g->n;
    a.dt = dt;
    a.bc_lo = g->bc_lo;
    a.bc_hi = g->bc_hi;
    a.inst = nullptr;
    a.tiles = nullptr;
    a.desc = nullptr;
    a.ptab = nullptr;
    a.ntiles = (g->N + a.tile - 1) / a.tile;
    a.wq = 1 + scheme;
    a.w_stride = int64_t(g->n) * a.wq * g->n;
    a.N = g->N;
    a.h = g->h;
    a.bc = g->bc;
    const int block = 256;
    if (!lmep::apply_configure(a, mixed, block)) return fail(LMEP_ERR_UNSUPPORTED, "tile does not fit in shared memory");
    const int grid = lmep::apply_grid(a, block, 0, mixed);
    for (int64_t t = 0; t < nsteps; ++t) {
      a.wait_polls = h->wait_polls;
      CK(lmep::launch_apply(a, cur, nxt, W_dev, mixed, block, grid, h->flags, S(stream)), "step(apply)");
      std::swap(cur, nxt);
    }
  }
  const size_t total = size_t(g->N) * size_t(W_dev ? 1 : (g->batch > 1 ? g->batch : 1));
  if (cur != u_dev) CK(cudaMemcpyAsync(u_dev, cur, total * es, cudaMemcpyDeviceToDevice, S(stream)), "copy");
  return LMEP_OK;
}

// ------------------------------------------------------------------ batches
namespace {
struct BatchLayout {
  size_t inst_off, tiles_off, desc_off, h_off, w_off, ptab_off, total;
  int64_t ntiles;
  int tile;  // points updated per tile
};
lmep_status batch_layout(const lmep_batch_desc* d, int32_t precision, BatchLayout* L) {
  if (!d || d->B <= 0 || !d->N_host || !d->h_host || !d->bc_host) return fail(LMEP_ERR_INVALID, "bad batch descriptor");
  if (d->n < 3 || d->n > 15 || d->n % 2 == 0) return fail(LMEP_ERR_INVALID, "n must be odd, 3..15");
  if (d->scheme == 3) return fail(LMEP_ERR_UNSUPPORTED, "ETDRK4 batches are not supported (use lmep_step)");
  if (d->scheme < 0 || d->scheme > 2 || d->n + d->scheme > 16) return fail(LMEP_ERR_INVALID, "bad scheme");
  if (d->nonlin < 0 || d->nonlin > 3) return fail(LMEP_ERR_INVALID, "unknown nonlinearity");
  if (d->nonlin >= 2) return fail(LMEP_ERR_UNSUPPORTED, "KdV and Burgers batches are not supported");
  if ((d->scheme == 0) != (d->nonlin == 0)) return fail(LMEP_ERR_INVALID, "linear scheme <=> no nonlinearity");
  if (d->op.frozen_adv != 0.0) return fail(LMEP_ERR_INVALID, "batches use constant operators");
  lmep_status st = check_prec(precision);
  if (st != LMEP_OK) return st;
  const bool mixed = precision == LMEP_PREC_MIXED;
  int tile = d->tile > 0 ? d->tile : default_fast_tile(mixed);
  if (tile % 128 != 0 || tile > 16384) return fail(LMEP_ERR_INVALID, "tile must be a multiple of 128, <= 16384");
  if (d->block != 0 && d->block != 64 && d->block != 128 && d->block != 256 && d->block != 512)
    return fail(LMEP_ERR_INVALID, "block must be 64, 128, 256 or 512");
  const int H = lmep::apply_fast_halo(d->n, d->scheme);
  const int tile_out = lmep::fast_tile_out(tile, d->n, d->scheme);
  int64_t ntiles = 0;
  for (int64_t b = 0; b < d->B; ++b) {
    const int64_t N = d->N_host[b];
    if (d->bc_host[b] != LMEP_BC_PERIODIC && d->bc_host[b] != LMEP_BC_NEUMANN)
      return fail(LMEP_ERR_INVALID, "batch instances must be periodic or Neumann");
    if (N < 2 * H + 8 || N < d->n) return fail(LMEP_ERR_UNSUPPORTED, "instance too small for the halo");
    if (!(d->h_host[b] > 0.0)) return fail(LMEP_ERR_INVALID, "h must be positive");
    ntiles += (N + tile_out - 1) / tile_out;
  }
  if (ntiles > (int64_t(1) << 31) - 1) return fail(LMEP_ERR_INVALID, "too many tiles");
  const size_t es = mixed ? 4 : 8;
  L->tile = tile_out;
  L->ntiles = ntiles;
  L->inst_off = 256;
  L->tiles_off = align_up(L->inst_off + size_t(d->B) * sizeof(Instance), 256);
  L->desc_off = align_up(L->tiles_off + size_t(ntiles) * sizeof(int2), 256);
  L->h_off = align_up(L->desc_off + size_t(ntiles) * sizeof(lmep::TileDesc), 256);
  L->w_off = align_up(L->h_off + size_t(d->B) * sizeof(double), 256);
  L->ptab_off = align_up(L->w_off + size_t(d->B) * d->n * (1 + d->scheme) * d->n * es, 256);
  L->total = align_up(L->ptab_off + size_t(d->B) * size_t(lmep::pair_table_stride(d->n)) * es, 256);
  return LMEP_OK;
}
}  // namespace

lmep_status lmep_batch_workspace_bytes(const lmep_batch_desc* d, int32_t precision, size_t* bytes_out) {
  if (!bytes_out) return fail(LMEP_ERR_INVALID, "bytes_out is NULL");
  BatchLayout L;
  lmep_status st = batch_layout(d, precision, &L);
  if (st != LMEP_OK) return st;
  *bytes_out = L.total;
  return LMEP_OK;
}

lmep_status lmep_batch_prepare(lmep_handle* h, const lmep_batch_desc* d, void* ws, size_t bytes,
                               int32_t precision, void* stream) {
  if (!h || !ws) return fail(LMEP_ERR_INVALID, "NULL handle/workspace");
  if (!aligned16(ws)) return fail(LMEP_ERR_INVALID, "workspace must be 16-byte aligned");
  BatchLayout L;
  lmep_status st = batch_layout(d, precision, &L);
  if (st != LMEP_OK) return st;
  if (bytes < L.total) return fail(LMEP_ERR_NOMEM, "workspace smaller than lmep_batch_workspace_bytes");
  const bool mixed = precision == LMEP_PREC_MIXED;
  std::vector<Instance> inst(size_t(d->B));
  std::vector<int2> tiles;
  std::vector<lmep::TileDesc> desc;
  tiles.reserve(size_t(L.ntiles));
  desc.reserve(size_t(L.ntiles));
  int64_t off = 0;
  for (int64_t b = 0; b < d->B; ++b) {
    inst[b].off = off;
    inst[b].N = d->N_host[b];
    inst[b].h = d->h_host[b];
    inst[b].bc = d->bc_host[b];
    inst[b].pad = 0;
    for (int64_t t0 = 0; t0 < inst[b].N; t0 += L.tile) {
      tiles.push_back(make_int2(int(b), int(t0)));
      desc.push_back(lmep::TileDesc{off, inst[b].N, t0, int32_t(b), inst[b].bc});
    }
    off += (inst[b].N + 3) / 4 * 4;  // every instance starts on a 16-byte boundary
  }
  char* base = static_cast<char*>(ws);
  CK(cudaMemcpyAsync(base + L.inst_off, inst.data(), inst.size() * sizeof(Instance), cudaMemcpyHostToDevice,
                     S(stream)), "copy(instances)");
  CK(cudaMemcpyAsync(base + L.tiles_off, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice,
                     S(stream)), "copy(tiles)");
  CK(cudaMemcpyAsync(base + L.desc_off, desc.data(), desc.size() * sizeof(lmep::TileDesc), cudaMemcpyHostToDevice,
                     S(stream)), "copy(tile descriptors)");
  CK(cudaMemcpyAsync(base + L.h_off, d->h_host, size_t(d->B) * sizeof(double), cudaMemcpyHostToDevice,
                     S(stream)), "copy(h)");
  // weights of every instance, harvested on the device
  lmep_grid g{};
  g.N = 1 << 20;
  g.h = 1.0;
  g.bc = LMEP_BC_PERIODIC;
  g.n = d->n;
  KParams p = make_params(&g, &d->op, d->dt, d->scheme);
  CK(lmep::launch_harvest_const(p, reinterpret_cast<const double*>(base + L.h_off), d->B, base + L.w_off,
                                mixed, S(stream)), "harvest(batch)");
  CK(lmep::launch_pair_tables(base + L.w_off, int64_t(d->n) * (1 + d->scheme) * d->n, 1 + d->scheme, d->n,
                              d->scheme, d->B, base + L.ptab_off, mixed, S(stream)), "pair tables");
  // the host copies above read pageable vectors: make sure they are consumed
  CK(cudaStreamSynchronize(S(stream)), "sync(prepare)");
  BatchPlan plan{};
  ApplyParams& a = plan.ap;
  a.n = d->n;
  a.scheme = d->scheme;
  a.nonlin = d->nonlin;
  a.halo = lmep::apply_fast_halo(d->n, d->scheme);
  a.fast = 1;
  a.tile = L.tile;
  a.dt = d->dt;
  a.inst = reinterpret_cast<const Instance*>(base + L.inst_off);
  a.tiles = reinterpret_cast<const int2*>(base + L.tiles_off);
  a.desc = reinterpret_cast<const lmep::TileDesc*>(base + L.desc_off);
  a.ptab = base + L.ptab_off;
  a.ntiles = L.ntiles;
  a.wq = 1 + d->scheme;
  a.w_stride = int64_t(d->n) * a.wq * d->n;
  a.N = 0;
  a.h = 1.0;
  a.bc = LMEP_BC_PERIODIC;
  plan.block = d->block > 0 ? d->block : 256;
  if (!lmep::apply_configure(a, mixed, plan.block)) return fail(LMEP_ERR_INVALID, "tile too large for shared memory");
  plan.W = base + L.w_off;
  plan.points = off;
  plan.mixed = mixed;
  plan.grid = lmep::apply_grid(a, plan.block, d->ctas_per_sm, mixed);
  plan.bytes = L.total;
  h->plans[ws] = plan;
  return LMEP_OK;
}

lmep_status lmep_step_batched(lmep_handle* h, const void* ws, void* u_dev, void* work_dev, int64_t nsteps,
                              void* stream) {
  if (!h || !ws || !u_dev || !work_dev) return fail(LMEP_ERR_INVALID, "NULL argument");
  if (u_dev == work_dev) return fail(LMEP_ERR_INVALID, "u_dev and work_dev must differ");
  auto it = h->plans.find(ws);
  if (it == h->plans.end()) return fail(LMEP_ERR_INVALID, "workspace was not prepared with this handle");
  if (nsteps < 0) return fail(LMEP_ERR_INVALID, "nsteps < 0");
  if (!aligned16(u_dev) || !aligned16(work_dev)) return fail(LMEP_ERR_INVALID, "batched states must be 16-byte aligned");
  const BatchPlan& plan = it->second;
  ApplyParams ap = plan.ap;
  ap.wait_polls = h->wait_polls;
  void* cur = u_dev;
  void* nxt = work_dev;
  for (int64_t t = 0; t < nsteps; ++t) {
    CK(lmep::launch_apply(ap, cur, nxt, plan.W, plan.mixed, plan.block, plan.grid, h->flags, S(stream)),
       "step_batched");
    std::swap(cur, nxt);
  }
  const size_t es = plan.mixed ? 4 : 8;
  if (cur != u_dev)
    CK(cudaMemcpyAsync(u_dev, cur, size_t(plan.points) * es, cudaMemcpyDeviceToDevice, S(stream)), "copy");
  return LMEP_OK;
}

lmep_status lmep_step_batched_once(lmep_handle* h, const void* ws, const void* u_in_dev, void* u_out_dev,
                                   void* stream) {
  if (!h || !ws || !u_in_dev || !u_out_dev) return fail(LMEP_ERR_INVALID, "NULL argument");
  if (u_in_dev == u_out_dev) return fail(LMEP_ERR_INVALID, "u_in_dev and u_out_dev must differ");
  auto it = h->plans.find(ws);
  if (it == h->plans.end()) return fail(LMEP_ERR_INVALID, "workspace was not prepared with this handle");
  if (!aligned16(u_in_dev) || !aligned16(u_out_dev))
    return fail(LMEP_ERR_INVALID, "batched states must be 16-byte aligned");
  const BatchPlan& plan = it->second;
  ApplyParams ap = plan.ap;
  ap.wait_polls = h->wait_polls;
  CK(lmep::launch_apply(ap, u_in_dev, u_out_dev, plan.W, plan.mixed, plan.block, plan.grid, h->flags, S(stream)),
     "step_batched_once");
  return LMEP_OK;
}

// ------------------------------------------------------------------ frozen-velocity sets
namespace {
lmep_status set_layout(const lmep_frozen_set_desc* d, int32_t precision, int32_t method, lmep::SetLayout* L,
                       std::vector<KParams>* ps, std::vector<int32_t>* route, std::vector<int64_t>* offs) {
  if (!d || d->B <= 0 || !d->grids_host || !d->ops_host || !d->dt_host)
    return fail(LMEP_ERR_INVALID, "bad frozen-set descriptor");
  if (d->B > (int64_t(1) << 20)) return fail(LMEP_ERR_INVALID, "too many instances");
  lmep_status st = check_prec(precision);
  if (st != LMEP_OK) return st;
  const int block = d->block > 0 ? d->block : 256;
  const int ppt = d->points_per_thread > 0 ? d->points_per_thread : 2;
  if (block != 64 && block != 128 && block != 256 && block != 512)
    return fail(LMEP_ERR_INVALID, "block must be 64, 128, 256 or 512");
  if (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 8) return fail(LMEP_ERR_INVALID, "points_per_thread must be 1, 2, 4 or 8");
  std::vector<int32_t> n(size_t(d->B));
  std::vector<int64_t> N(size_t(d->B));
  int64_t off = 0;
  for (int64_t b = 0; b < d->B; ++b) {
    const lmep_grid* g = d->grids_host + b;
    const lmep_operator* op = d->ops_host + b;
    const double dt = d->dt_host[b];
    if ((st = check_grid(g, 0)) != LMEP_OK) return st;
    if ((st = no_shift(g)) != LMEP_OK) return st;
    if (g->batch > 1) return fail(LMEP_ERR_INVALID, "frozen-set instances take batch <= 1");
    if (op->frozen_adv == 0.0) return fail(LMEP_ERR_INVALID, "frozen-set instances need a frozen operator");
    if (!(dt > 0.0)) return fail(LMEP_ERR_INVALID, "dt must be positive");
    if (g->N >= (int64_t(1) << 31)) return fail(LMEP_ERR_UNSUPPORTED, "frozen-set instances take N < 2^31");
    if (g->bc == LMEP_BC_NEUMANN && g->N < 2 * g->n) return fail(LMEP_ERR_UNSUPPORTED, "Neumann needs N >= 2n");
    KParams p = make_params(g, op, dt, 0);
    p.series = method != LMEP_EXPM_PADE;
    if (ps) ps->push_back(p);
    if (route) route->push_back(method == LMEP_EXPM_AUTO ? 0 : 1);
    if (offs) offs->push_back(off);
    n[size_t(b)] = g->n;
    N[size_t(b)] = g->N;
    off += (g->N + 3) / 4 * 4;
  }
  *L = lmep::frozen_set_layout(d->B, n.data(), N.data(), block, ppt, precision == LMEP_PREC_MIXED);
  if (L->ntiles >= (int64_t(1) << 31)) return fail(LMEP_ERR_UNSUPPORTED, "too many tiles");
  return LMEP_OK;
}
}  // namespace

lmep_status lmep_frozen_set_workspace_bytes(const lmep_frozen_set_desc* d, int32_t precision, size_t* bytes_out) {
  if (!bytes_out) return fail(LMEP_ERR_INVALID, "bytes_out is NULL");
  lmep::SetLayout L;
  lmep_status st = set_layout(d, precision, LMEP_EXPM_AUTO, &L, nullptr, nullptr, nullptr);
  if (st != LMEP_OK) return st;
  *bytes_out = L.total;
  return LMEP_OK;
}

lmep_status lmep_frozen_set_prepare(lmep_handle* h, const lmep_frozen_set_desc* d, void* ws, size_t bytes,
                                    int32_t precision, void* stream) {
  if (!h || !ws) return fail(LMEP_ERR_INVALID, "NULL handle/workspace");
  if (!aligned16(ws)) return fail(LMEP_ERR_INVALID, "workspace must be 16-byte aligned");
  lmep::SetLayout L;
  std::vector<KParams> ps;
  std::vector<int32_t> route;
  std::vector<int64_t> offs;
  lmep_status st = set_layout(d, precision, h->expm_method, &L, &ps, &route, &offs);
  if (st != LMEP_OK) return st;
  if (bytes < L.total) return fail(LMEP_ERR_NOMEM, "workspace smaller than lmep_frozen_set_workspace_bytes");
  h->sets.erase(ws);
  CK(lmep::frozen_set_prepare(ws, L, ps.data(), route.data(), offs.data(), S(stream)), "frozen_set_prepare");
  h->sets[ws] = L;
  return LMEP_OK;
}

lmep_status lmep_frozen_set_refresh(lmep_handle* h, void* ws, void* stream) {
  if (!h || !ws) return fail(LMEP_ERR_INVALID, "NULL argument");
  auto it = h->sets.find(ws);
  if (it == h->sets.end()) return fail(LMEP_ERR_INVALID, "workspace was not prepared with this handle");
  CK(lmep::frozen_set_refresh(ws, it->second, S(stream)), "frozen_set_refresh");
  return LMEP_OK;
}

lmep_status lmep_frozen_set_step_once(lmep_handle* h, const void* ws, const void* u_in_dev, void* u_out_dev,
                                      void* stream) {
  if (!h || !ws || !u_in_dev || !u_out_dev) return fail(LMEP_ERR_INVALID, "NULL argument");
  if (u_in_dev == u_out_dev) return fail(LMEP_ERR_INVALID, "u_in_dev and u_out_dev must differ");
  auto it = h->sets.find(ws);
  if (it == h->sets.end()) return fail(LMEP_ERR_INVALID, "workspace was not prepared with this handle");
  CK(lmep::frozen_set_step(const_cast<void*>(ws), it->second, u_in_dev, u_out_dev, h->flags, S(stream)),
     "frozen_set_step_once");
  return LMEP_OK;
}

lmep_status lmep_adjoint_scratch_bytes(const lmep_grid* g, int32_t precision, size_t* bytes_out) {
  if (!bytes_out) return fail(LMEP_ERR_INVALID, "bytes_out is NULL");
  lmep_status st = check_grid(g, 0);
  if (st != LMEP_OK) return st;
  st = check_prec(precision);
  if (st != LMEP_OK) return st;
  *bytes_out = lmep::adjoint_scratch_bytes(g->N * (g->batch > 1 ? g->batch : 1), g->n, precision == LMEP_PREC_MIXED);
  return LMEP_OK;
}

lmep_status lmep_adjoint_step(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, double dt,
                              const void* u_dev, const void* lam_next_dev, void* lam_dev, double* dnu_dev,
                              void* scratch_dev, size_t scratch_bytes, int32_t precision, void* stream) {
  if (!h || !op) return fail(LMEP_ERR_INVALID, "NULL handle/operator");
  lmep_status st = check_grid(g, 0);
  if (st != LMEP_OK) return st;
  st = check_prec(precision);
  if (st != LMEP_OK) return st;
  if ((st = no_shift(g)) != LMEP_OK) return st;
  if (g->bc == LMEP_BC_NEUMANN) return fail(LMEP_ERR_UNSUPPORTED, "adjoint supports periodic and Dirichlet grids");
  if (g->bc == LMEP_BC_PERIODIC && g->N < 2 * g->n) return fail(LMEP_ERR_UNSUPPORTED, "periodic adjoint needs N >= 2n");
  if (!u_dev || !lam_next_dev || !lam_dev || !dnu_dev || !scratch_dev) return fail(LMEP_ERR_INVALID, "NULL buffer");
  if (lam_dev == lam_next_dev) return fail(LMEP_ERR_INVALID, "lam_dev must differ from lam_next_dev");
  const bool mixed = precision == LMEP_PREC_MIXED;
  if (scratch_bytes < lmep::adjoint_scratch_bytes(g->N * (g->batch > 1 ? g->batch : 1), g->n, mixed))
    return fail(LMEP_ERR_NOMEM, "scratch too small");
  const KParams p = make_params(g, op, dt, 0);
  const double* sl = nullptr;
  if (h->expm_method == LMEP_EXPM_AUTO && (st = sl_table(h, p, S(stream), &sl)) != LMEP_OK) return st;
  CK(lmep::launch_adjoint(p, u_dev, lam_next_dev, lam_dev, dnu_dev, scratch_dev, mixed, h->flags, S(stream), sl),
     "adjoint");
  return LMEP_OK;
}

lmep_status lmep_frozen_stats(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, double dt,
                              const void* u_dev, int32_t* stats_dev, int32_t precision, void* stream) {
  if (!h || !op || !u_dev || !stats_dev) return fail(LMEP_ERR_INVALID, "NULL argument");
  lmep_status st = check_grid(g, 0);
  if (st != LMEP_OK) return st;
  st = check_prec(precision);
  if (st != LMEP_OK) return st;
  if ((st = no_shift(g)) != LMEP_OK) return st;
  if (op->frozen_adv == 0.0) return fail(LMEP_ERR_INVALID, "lmep_frozen_stats needs a frozen operator");
  if (!(dt > 0.0)) return fail(LMEP_ERR_INVALID, "dt must be positive");
  if (g->bc == LMEP_BC_NEUMANN && g->N < 2 * g->n) return fail(LMEP_ERR_UNSUPPORTED, "Neumann needs N >= 2n");
  KParams p = make_params(g, op, dt, 0);
  p.series = h->expm_method != LMEP_EXPM_PADE;
  const bool mixed = precision == LMEP_PREC_MIXED;
  const double* sl = nullptr;
  if (h->expm_method == LMEP_EXPM_AUTO && (st = sl_table(h, p, S(stream), &sl)) != LMEP_OK) return st;
  CK(lmep::launch_frozen(p, u_dev, nullptr, false, mixed, h->flags, S(stream), stats_dev, sl), "frozen_stats");
  return LMEP_OK;
}

lmep_status lmep_set_expm_method(lmep_handle* h, int32_t method) {
  if (!h) return fail(LMEP_ERR_INVALID, "handle is NULL");
  if (method != LMEP_EXPM_AUTO && method != LMEP_EXPM_PADE && method != LMEP_EXPM_SERIES)
    return fail(LMEP_ERR_INVALID, "method must be LMEP_EXPM_AUTO, LMEP_EXPM_PADE or LMEP_EXPM_SERIES");
  h->expm_method = method;
  return LMEP_OK;
}

lmep_status lmep_set_wait_limit(lmep_handle* h, int64_t polls) {
  if (!h) return fail(LMEP_ERR_INVALID, "handle is NULL");
  if (polls > (int64_t(1) << 30)) return fail(LMEP_ERR_INVALID, "polls must be <= 2^30");
  h->wait_polls = polls < 0 ? (1 << 20) : int32_t(polls);
  return LMEP_OK;
}

lmep_status lmep_sync_status(lmep_handle* h, void* stream) {
  if (!h) return fail(LMEP_ERR_INVALID, "handle is NULL");
  CK(cudaStreamSynchronize(S(stream)), "cudaStreamSynchronize");
  unsigned flags = 0;
  CK(cudaMemcpy(&flags, h->flags, sizeof(unsigned), cudaMemcpyDeviceToHost), "read status");
  if (flags) {
    CK(cudaMemset(h->flags, 0, sizeof(unsigned)), "clear status");
    if (flags & 2u) return fail(LMEP_ERR_TIMEOUT, "a kernel gave up waiting for a bulk copy");
    return fail(LMEP_ERR_NONFINITE, "a kernel produced a non-finite value");
  }
  return LMEP_OK;
}

// ------------------------------------------------------------------ non-uniform grids
namespace {
lmep_status check_nodes(int64_t N, int32_t n, int32_t scheme, int32_t precision) {
  if (n < 3 || n > 15 || n % 2 == 0) return fail(LMEP_ERR_INVALID, "n must be odd, 3..15");
  if (N < n) return fail(LMEP_ERR_INVALID, "N must be >= n");
  if (N >= (int64_t(1) << 31)) return fail(LMEP_ERR_UNSUPPORTED, "non-uniform grids take N < 2^31");
  if (scheme < 0 || scheme > 3) return fail(LMEP_ERR_INVALID, "unknown scheme");
  if (n + scheme > 16) return fail(LMEP_ERR_UNSUPPORTED, "n + n_phi must be <= 16");
  return check_prec(precision);
}
}  // namespace

lmep_status lmep_harvest_nodes(lmep_handle* h, int64_t N, const double* x_dev, int32_t n, const lmep_operator* op,
                               double dt, int32_t scheme, void* W_dev, int32_t precision, void* stream) {
  if (!h || !op || !x_dev || !W_dev) return fail(LMEP_ERR_INVALID, "NULL handle/operator/nodes/W");
  lmep_status st = check_nodes(N, n, scheme, precision);
  if (st != LMEP_OK) return st;
  if (!(dt > 0.0)) return fail(LMEP_ERR_INVALID, "dt must be positive");
  if (op->frozen_adv != 0.0) return fail(LMEP_ERR_INVALID, "stored weights need a constant operator");
  lmep_grid g{};
  g.N = N;
  g.h = 1.0;
  g.bc = LMEP_BC_DIRICHLET;
  g.n = n;
  const bool mixed = precision == LMEP_PREC_MIXED;
  const int R = lmep::pw_rows(scheme);
  KParams p = make_params(&g, op, dt, scheme);
  p.w_rows = R;
  p.rk4 = scheme == 3;
  CK(lmep::launch_harvest_nodes(p, x_dev, W_dev, mixed, S(stream)), "harvest_nodes");
  if (scheme == 3) {
    KParams q = make_params(&g, op, 0.5 * dt, 1);
    q.w_rows = R;
    q.w_row0 = 4;
    CK(lmep::launch_harvest_nodes(q, x_dev, W_dev, mixed, S(stream)), "harvest_nodes(dt/2)");
  }
  return LMEP_OK;
}

lmep_status lmep_step_nodes(lmep_handle* h, int64_t N, int32_t n, int32_t scheme, int32_t nonlin, double dt,
                            double bc_lo, double bc_hi, const void* W_dev, void* u_dev, void* work_dev, int64_t nsteps,
                            int32_t precision, void* stream) {
  if (!h || !W_dev || !u_dev || !work_dev) return fail(LMEP_ERR_INVALID, "NULL argument");
  lmep_status st = check_nodes(N, n, scheme, precision);
  if (st != LMEP_OK) return st;
  if (nonlin != LMEP_N_NONE && nonlin != LMEP_N_ALLEN_CAHN)
    return fail(LMEP_ERR_UNSUPPORTED, "non-uniform grids take a pointwise nonlinearity (Allen-Cahn) or none");
  if ((scheme == 0) != (nonlin == 0)) return fail(LMEP_ERR_INVALID, "linear scheme <=> no nonlinearity");
  if (u_dev == work_dev) return fail(LMEP_ERR_INVALID, "u_dev and work_dev must differ");
  if (nsteps < 0) return fail(LMEP_ERR_INVALID, "nsteps < 0");
  if (!(dt > 0.0)) return fail(LMEP_ERR_INVALID, "dt must be positive");
  const bool mixed = precision == LMEP_PREC_MIXED;
  void* cur = u_dev;
  void* nxt = work_dev;
  for (int64_t t = 0; t < nsteps; ++t) {
    CK(lmep::launch_apply_pw(N, n, scheme, nonlin, dt, bc_lo, bc_hi, cur, nxt, W_dev, mixed, h->flags, S(stream)),
       "step_nodes");
    std::swap(cur, nxt);
  }
  if (cur != u_dev)
    CK(cudaMemcpyAsync(u_dev, cur, size_t(N) * (mixed ? 4 : 8), cudaMemcpyDeviceToDevice, S(stream)), "copy");
  return LMEP_OK;
}

lmep_status lmep_amplification(const double* w_dev, int32_t n, int32_t r, const double* theta_dev, int64_t M,
                               double* G_dev, void* stream) {
  if (n < 1 || n > 64) return fail(LMEP_ERR_INVALID, "n must be 1..64");
  if (r < 0 || r >= n) return fail(LMEP_ERR_INVALID, "r must be in [0, n)");
  if (M < 0) return fail(LMEP_ERR_INVALID, "M < 0");
  if (M == 0) return LMEP_OK;
  if (!w_dev || !theta_dev || !G_dev) return fail(LMEP_ERR_INVALID, "NULL buffer");
  CK(lmep::launch_symbol(w_dev, n, r, theta_dev, M, G_dev, S(stream)), "amplification");
  return LMEP_OK;
}

lmep_status lmep_fma_peak(int32_t precision, double* flops_out) {
  if (!flops_out) return fail(LMEP_ERR_INVALID, "flops_out is NULL");
  lmep_status st = check_prec(precision);
  if (st != LMEP_OK) return st;
  CK(lmep::fma_peak(precision == LMEP_PREC_MIXED, flops_out), "fma_peak");
  return LMEP_OK;
}

}  // extern "C"
