// lmep_internal.h -- launcher interface between the C ABI layer and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

struct lmep_grid;
struct lmep_operator;

namespace lmep {

// Problem parameters passed by value to every kernel.
struct KParams {
  int64_t N;
  int64_t batch;  // instances of N points stored back to back (0 or 1: one)
  double h;
  int bc;
  int n;
  int dep;      // departure centring on/off
  int n_phi;
  double bc_lo, bc_hi;
  double dt, c0, c1, c2, c3, fa;
  // derived on the host once per launch: dt/h, dt c0, dt c2/h^2, dt c3/h^3,
  // and their FP32 roundings for the FP32 form
  double dt_h, c0dt, c2h, c3h;
  float c0dt_f, c2h_f, c3h_f;
  float c1_f, fa_f, dt_h_f;  // FP32 roundings of c1, fa and dt/h (FP32-form window setup)
  // frozen-velocity rows: 1 = finite series of the nilpotent local matrix with
  // a Pade scaling-and-squaring fallback (after the factorised rows, when the
  // launch carries exp(E)), 0 = Pade scaling and squaring only
  int series;
  // constant-coefficient harvest output: weight rows stored per row class
  // (0: 1 + n_phi) and the first of them written; rk4 = 1 stores, for
  // n_phi = 3, the rows of exp(X), dt alpha, dt beta, dt gamma of ETDRK4
  // (combinations of the FP64 rows of dt^k phi_k) instead of the raw rows
  int w_rows, w_row0, rk4;
};

// Set the thread-local text returned by lmep_last_error().
void set_last_error(const std::string& msg);

// Kernel parameters of one grid, operator and time step (lmep_api.cu): the
// derived constants dt/h, dt c0, dt c2/h^2, dt c3/h^3 and their FP32
// roundings are formed here once, so every entry point passes identical
// parameters to the kernels.
KParams make_params(const struct ::lmep_grid* g, const struct ::lmep_operator* op, double dt, int n_phi);

// ---- wide stencils (lmep_wide.cu): odd n = 17 .. 25, constant-coefficient linear scheme
bool wide_width(int n);
// Rows W[r][0][j] of every row class r (FP64 arithmetic, stored in the state type).
cudaError_t launch_harvest_wide(const KParams& p, void* W, bool mixed, cudaStream_t s);
// One step u -> out on a periodic grid with the row of class (n - 1) / 2 + shift.
cudaError_t launch_apply_wide(int64_t N, int n, int shift, const void* W, const void* u, void* out, bool mixed,
                              unsigned* flags, cudaStream_t s);

struct DeviceInfo {
  int sms;
  int smem_optin;  // dynamic shared memory a CTA may opt in to (bytes)
};
DeviceInfo device_info();

// ---- expm family (lmep_expm.cu)
// Build the per-n derivative tables on the current device (once; synchronous).
cudaError_t fornberg_init();
// Device addresses of the h^k D^(k) tables (k = 1..3) of width n, FP64 and FP32.
cudaError_t fornberg_of(int n, const double** d, const float** f);
cudaError_t launch_build_operator(const KParams& p, const double* u, int64_t i0, int64_t count,
                                  double* M, int32_t* start, int32_t* row, cudaStream_t s);
cudaError_t launch_expm(const double* A, int64_t P, int d, double* E, bool mixed, int32_t* ms,
                        cudaStream_t s);
// Constant-coefficient weights for B instances (h_inst nullable -> p.h), W[b][n][1+n_phi][n].
cudaError_t launch_harvest_const(const KParams& p, const double* h_inst, int64_t B, void* W,
                                 bool mixed, cudaStream_t s);
// Frozen velocity: fused == false writes W[N][n]; fused == true writes u_out.
// sl (host, nullable): exp(E) of the point-independent part of the local matrix,
// n x n row-major, then its n absolute row sums (factorised rows; rounded to FP32
// for the FP32 form).
cudaError_t launch_frozen(const KParams& p, const void* u, void* out, bool fused, bool mixed,
                          unsigned* flags, cudaStream_t s, int32_t* stats = nullptr, const double* sl = nullptr);
// exp(c2h Dh2 + c3h Dh3) of the window (FP64, n x n row-major) into out and
// Dh2 exp(c2h Dh2 + c3h Dh3) into out2 (device).
cudaError_t launch_exp_const(const KParams& p, double* out, double* out2, cudaStream_t s);

// ---- frozen-velocity sets (lmep_frozen_set.cu): several instances, each with
// its own grid, operator, dt and stencil width, advanced by one launch per
// step (plus a launch that finishes the rare points the first one rejects).
struct SetLayout {
  size_t ctl, ok, inst, jobs, tiles, starts, exps, tab, lists, total;  // byte offsets of the regions, total size
  int64_t B, ntiles, points;
  int block, ppt;
  int grid;  // persistent grid of the lean kernel (set by frozen_set_prepare)
  bool mixed;
};
// Region offsets and sizes of a set of B instances (widths n[b], sizes N[b]) for
// tiles of block * ppt points.
SetLayout frozen_set_layout(int64_t B, const int32_t* n, const int64_t* N, int block, int ppt, bool mixed);
// Fill a workspace: instance records, fallback jobs, tile table (each CTA's
// tiles together, balanced by estimated cost), cleared counters, then the
// exp(E) tables on the device.
// route[b] = 0: factorised rows first; 1: every point through the fallback
// (finite series, then Pade; p.series = 0: Pade only).  Synchronises s.
cudaError_t frozen_set_prepare(void* ws, SetLayout& L, const KParams* p, const int32_t* route,
                               const int64_t* offsets, cudaStream_t s);
// Recompute the exp(E) tables of a prepared workspace (device only).
cudaError_t frozen_set_refresh(void* ws, const SetLayout& L, cudaStream_t s);
// One step of every instance from u_in to u_out.
cudaError_t frozen_set_step(void* ws, const SetLayout& L, const void* u_in, void* u_out, unsigned* flags,
                            cudaStream_t s);

// ---- banded apply (lmep_apply.cu)
struct Instance {
  int64_t off;   // first element of the instance in the concatenated state
  int64_t N;
  double h;
  int bc;
  int pad;
};
// One tile of a batch: instance offset, length and boundary condition, and the
// tile's first point (32 bytes, read as two 16-byte vectors).
struct TileDesc {
  int64_t off;
  int64_t N;
  int64_t t0;
  int32_t b;
  int32_t bc;
};
static_assert(sizeof(TileDesc) == 32, "TileDesc is 32 bytes");
struct ApplyParams {
  int n, scheme, nonlin, tile;
  int halo;          // staged halo per side (apply_halo / apply_fast_halo)
  int shift;         // window shift upstream (lmep_grid.window_shift; CTA-tiled kernel, linear scheme)
  int fast;          // 1: pipelined register-tiled kernel (periodic/Neumann, pointwise nonlinearity)
  int stages;        // fast kernel: stage slots per warp (set by apply_configure)
  int wait_polls;    // fast kernel: bound of a warp's wait for its next tile, in polls (default 2^20)
  int warp_smem;     // fast kernel: shared-memory bytes per warp (set by apply_configure)
  double dt;
  double bc_lo, bc_hi;
  // instance table (device) and tile table (device, int2 = {instance, start})
  const Instance* inst;
  const int2* tiles;
  const TileDesc* desc;  // fast kernel: tile descriptors (nullptr: one instance)
  const void* ptab;      // fast kernel: per-instance weight-pair tables (nullptr: one instance)
  int64_t ntiles;
  int64_t w_stride;  // elements between the weight blocks of consecutive instances
  int wq;            // weight rows stored per row class (1 + n_phi)
  // single-instance fallback when inst == nullptr
  int64_t N;
  double h;
  int bc;
  // set by launch_apply: 1 / dt, 1 / h (one instance) and, for a derivative
  // nonlinearity, the device table of h D^(1) rows of width n (row r at r * LD)
  double inv_dt, inv_h;
  const double* dh;
};
int apply_halo(int n, int scheme, int nonlin, int bc);
int apply_fast_halo(int n, int scheme);
int fast_tile_out(int tile, int n, int scheme);
size_t apply_smem_bytes(int tile, int halo, int scheme, bool mixed);
cudaError_t launch_apply(const ApplyParams& a, const void* u, void* out, const void* W, bool mixed,
                         int block, int grid, unsigned* flags, cudaStream_t s);
int apply_grid(const ApplyParams& a, int block, int ctas_per_sm, bool mixed);
// Choose the fast kernel's pipeline depth for `block` threads per CTA; false
// if the tile does not fit in shared memory.
bool apply_configure(ApplyParams& a, bool mixed, int block);
// ---- non-uniform grids (Sec. 4.3.3): per-node harvest (lmep_expm.cu, the warp
// kernel's MODE_NODES; p.N, p.n, p.n_phi, the coefficients, dt, w_rows, w_row0,
// rk4) into W[N][w_rows][n], and the apply with those stored rows
// (lmep_apply_pw.cu; Dirichlet walls, N(u) pointwise or none).
cudaError_t launch_harvest_nodes(const KParams& p, const double* x, void* W, bool mixed, cudaStream_t s);
int pw_rows(int scheme);
cudaError_t launch_apply_pw(int64_t N, int n, int scheme, int nonlin, double dt, double bc_lo, double bc_hi,
                            const void* u, void* out, const void* W, bool mixed, unsigned* flags, cudaStream_t s);

// ---- ETDRK4 apply (lmep_apply_rk4.cu): one step of one instance with the six
// weight rows per row class of lmep_harvest_scheme_weights (E, dt alpha,
// dt beta, dt gamma, exp(dt L / 2), (dt/2) phi_1(dt L / 2)); nonlin 1 (Allen-Cahn),
// 2 (KdV) or 3 (Burgers).
int rk4_halo(int n, int nonlin, int bc);
cudaError_t launch_apply_rk4(int64_t N, double h, int bc, int n, int nonlin, double dt, double bc_lo, double bc_hi,
                             const void* u, void* out, const void* W, bool mixed, unsigned* flags, cudaStream_t s);
// ---- warp-streaming apply (lmep_apply_stream.cu)
constexpr int STREAM_MAX_STAGES = 4;
constexpr int STREAM_HEADER = 8 * STREAM_MAX_STAGES + 32 * STREAM_MAX_STAGES;  // mbarriers, tile descriptors
const void* stream_kernel(int scheme, int n, bool mixed);
size_t stream_warp_smem(const ApplyParams& a, bool mixed, int stages, int scheme);
// Weight-pair tables of the fast kernel (elements per instance, and the kernel
// that fills B of them from harvested weights).
int pair_table_stride(int n);
cudaError_t launch_pair_tables(const void* W, int64_t w_stride, int wq, int n, int scheme, int64_t B, void* tab,
                               bool mixed, cudaStream_t s);

// ---- adjoint (lmep_adjoint.cu)
size_t adjoint_scratch_bytes(int64_t N, int n, bool mixed);
// sl (host, nullable): the factorised-row table of launch_frozen followed by Dh2 exp(E)
// (n x n); with it every point whose bound allows takes the factorised derivatives.
cudaError_t launch_adjoint(const KParams& p, const void* u, const void* lam_next, void* lam,
                           double* dnu, void* scratch, bool mixed, unsigned* flags, cudaStream_t s,
                           const double* sl = nullptr);

// ---- Fourier symbol of a weight row (lmep_spectral.cu): G[2q], G[2q+1] = Re, Im of
// sum_j w_j e^{i theta_q (j - r)}
cudaError_t launch_symbol(const double* w, int n, int r, const double* theta, int64_t M, double* G, cudaStream_t s);

// ---- peak (lmep_peak.cu)
cudaError_t fma_peak(bool fp32, double* flops);

}  // namespace lmep
