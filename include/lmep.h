/*
 * lmep.h -- C ABI of the GB300 (sm_103a) Local Matrix Exponential Propagator.
 *
 * Method: V. Bayona, "Unifying Finite Differences and Semi-Lagrangian Schemes
 * via Localized Matrix Exponentials".  For every grid point x_i the library
 *   (a1) selects the point's stencil window and harvest row       (Sec. 2.1 steps 1, 3)
 *   (a2) builds the derivative matrices D^(k) on the window        (Sec. 2.1 step 1, Fornberg)
 *   (a3) assembles X_i = dt A_i, A_i = c0 I + c1 D1 + c2 D2 + c3 D3 - frozen_adv u_i D1
 *                                                                    (Thm. 2 proof)
 *   (a4) exponentiates X_i, or the augmented local matrix for the
 *        ETD phi-functions                                           (Sec. 2.1 step 2, Sec. 3.1)
 *   (a5) harvests the weight rows                                    (Sec. 2.1 step 3, Sec. 3.1 step 2)
 *   (a6) applies them as one banded update u <- W u + dt Phi N(u)   (Sec. 3, Sec. 3.1 step 3)
 * and (a7) runs the discrete adjoint of the frozen-velocity step.
 *
 * Conventions (all entry points):
 *  - Every pointer named *_dev is device memory on the current CUDA device,
 *    owned by the caller, contiguous, at least 16-byte aligned.  *_host is
 *    host memory.  The library owns only the handle and its status block.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  No call synchronises except
 *    lmep_sync_status and lmep_fma_peak.
 *  - Invalid arguments return LMEP_ERR_INVALID before anything is launched.
 *    A failed launch returns LMEP_ERR_CUDA.  Non-finite results produced on
 *    the device are flagged and reported by the next lmep_sync_status.
 *  - Nothing throws across the ABI.  A handle is not thread-safe.
 *  - Floating-point layouts: dtype follows `precision`: LMEP_PREC_FP64 uses
 *    double everywhere; LMEP_PREC_MIXED (the batched FP32 form) stores the
 *    state and the weights as float, evaluates the Pade polynomial products
 *    in FP32 with FP32 accumulation, and keeps the Pade denominator solve and
 *    the squaring phase in FP64.
 */
#ifndef LMEP_H
#define LMEP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LMEP_API __attribute__((visibility("default")))
#else
#define LMEP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LMEP_OK = 0,
  LMEP_ERR_INVALID = 1,     /* bad argument; nothing was launched */
  LMEP_ERR_CUDA = 2,        /* a CUDA call failed; see lmep_last_error() */
  LMEP_ERR_NONFINITE = 3,   /* a kernel produced Inf/NaN since the last sync */
  LMEP_ERR_TIMEOUT = 4,     /* a kernel gave up a bounded wait for one of its own bulk copies */
  LMEP_ERR_UNSUPPORTED = 5, /* valid request outside the built shapes (e.g. n + n_phi > 16) */
  LMEP_ERR_NOMEM = 6        /* workspace smaller than required */
} lmep_status;

typedef enum { LMEP_BC_PERIODIC = 0, LMEP_BC_DIRICHLET = 1, LMEP_BC_NEUMANN = 2 } lmep_bc;
typedef enum { LMEP_PREC_FP64 = 0, LMEP_PREC_MIXED = 1 } lmep_precision;
typedef enum { LMEP_SCHEME_LINEAR = 0, LMEP_SCHEME_ETD1 = 1, LMEP_SCHEME_ETDRK2 = 2, LMEP_SCHEME_ETDRK4 = 3 } lmep_scheme;
/* N(u): Allen-Cahn u - u^3; KdV -6 u u_x; Burgers -u u_x (u_x from the row of
 * D^(1) of the point's window, Sec. 4.3.1 and 4.3.2) */
typedef enum { LMEP_N_NONE = 0, LMEP_N_ALLEN_CAHN = 1, LMEP_N_KDV = 2, LMEP_N_BURGERS = 3 } lmep_nonlin;
typedef enum { LMEP_EXPM_AUTO = 0, LMEP_EXPM_PADE = 1, LMEP_EXPM_SERIES = 2 } lmep_expm_method;

/* Uniform 1-D grid and stencil (Sec. 2.1 step 1).
 *  N      number of points.  Periodic: x_j = x0 + j h, j < N.  Dirichlet and
 *         Neumann: both walls are grid points (x_0 and x_{N-1}).
 *  h      spacing.
 *  bc     lmep_bc.  Dirichlet walls keep bc_lo / bc_hi and are never updated;
 *         near a wall the window slides inside the domain (one-sided
 *         stencil, edge row).  Neumann: homogeneous, even reflection about the
 *         wall node.  Periodic: centred window, indices mod N.
 *  n      stencil width, odd, 3 <= n <= 15, n <= N.  Wide stencils, odd
 *         17 <= n <= 25 (the widths of the one-sided study of Sec. 4.1), are
 *         built for the constant-coefficient linear scheme only: the harvest
 *         with n_phi = 0 and the stored-weight step on a periodic grid, any
 *         window_shift; every other call returns LMEP_ERR_UNSUPPORTED for them.
 *  departure_centring  frozen-velocity problems only: shift each window
 *         upstream by k_i = clamp(floor(u_i dt / h + 1/2), -(n-1)/2, (n-1)/2).
 *  batch  number of independent instances of this grid stored back to back
 *         (state arrays hold batch * N values; 0 means 1).  Honoured by the
 *         frozen-velocity step and harvest, lmep_frozen_stats and
 *         lmep_adjoint_step; the other calls require batch <= 1.
 *  window_shift  constant-coefficient stepping with the linear scheme only
 *         (Sec. 4.1's one-sided stencils): every window is shifted upstream
 *         by k = window_shift nodes, |k| <= (n-1)/2, and point i takes row
 *         class (n-1)/2 + k of its window (start i - (n-1)/2 - k; Dirichlet:
 *         clamped into the domain).  k = (n-1)/2 is the fully upwind window
 *         for a positive speed.  0 elsewhere.
 *  reserved  must be 0. */
typedef struct lmep_grid {
  int64_t N;
  double h;
  int32_t bc;
  int32_t n;
  int32_t departure_centring;
  int32_t batch;
  int32_t window_shift;
  int32_t reserved;
  double bc_lo, bc_hi;
} lmep_grid;

/* Linear operator L = c0 + c1 d/dx + c2 d^2/dx^2 + c3 d^3/dx^3 (Thm. 2 proof),
 * plus -frozen_adv * u_i * d/dx at point i with u_i frozen (local Burgers). */
typedef struct lmep_operator {
  double c0, c1, c2, c3;
  double frozen_adv;
} lmep_operator;

typedef struct lmep_handle lmep_handle;

/* Create a handle on the current device.  Allocates the device status block
 * (one cudaMalloc of 256 bytes); *out receives the handle. */
LMEP_API lmep_status lmep_create(lmep_handle** out);
LMEP_API lmep_status lmep_destroy(lmep_handle* h);

/* (a1)-(a3): for points i0 .. i0+count-1 write, on the device,
 *   start_dev[p] window start (global index of window node 0 before any
 *                wrap or reflection), row_dev[p] the harvest row r,
 *   M_dev[p]     the d x d row-major matrix that (a4) exponentiates, d = n + n_phi:
 *                n_phi = 0: X = dt A_i (plain, not re-centred);
 *                n_phi > 0: the transposed row-restricted augmented matrix
 *                [[X, 0], [dt e_r^T, 0], [0, dt, 0]..] whose rows r, n, n+1, ..
 *                (first n columns) are row r of exp(X), dt phi_1(X), dt^2 phi_2(X), ..
 * u_dev: double[N] frozen velocities, required iff op->frozen_adv != 0.
 * Sizes: M_dev double[count][d][d]; start_dev, row_dev int32[count]. */
LMEP_API lmep_status lmep_build_operator(lmep_handle* h, const lmep_grid* g, const lmep_operator* op,
                                double dt, int32_t n_phi, const double* u_dev, int64_t i0,
                                int64_t count, double* M_dev, int32_t* start_dev,
                                int32_t* row_dev, void* stream);

/* (a4) alone: E_p = exp(A_p) for P matrices of size d x d (3 <= d <= 16),
 * row-major double in and out, by Pade scaling and squaring (Higham 2005).
 * precision LMEP_PREC_MIXED evaluates the polynomial products in FP32.
 * ms_dev (nullable) receives int32[P][2] = (Pade degree m, squarings s). */
LMEP_API lmep_status lmep_expm(lmep_handle* h, const double* A_dev, int64_t P, int32_t d, double* E_dev,
                      int32_t precision, int32_t* ms_dev, void* stream);

/* (a1)-(a5): harvest weight rows.
 *  u_frozen_dev == NULL: constant coefficients; W_dev receives [n][1+n_phi][n]
 *      (0 <= n_phi <= 3, n + n_phi <= 16):
 *      W[r][k][:] = row r of dt^k phi_k(dt L) (k = 0: exp(dt L)) for every row class r.
 *      Wide stencils (n = 17..25, n_phi = 0): the rows are formed in FP64 from
 *      the factorisation row r of exp(X) = e^{c0 dt} l(r + a)^T exp(E)
 *      (Thm. 1 and the General Exactness theorem; a = c1 dt / h, E = dt (c2 D2
 *      + c3 D3) nilpotent, its exponential a finite Taylor sum), not by Pade.
 *  u_frozen_dev != NULL: frozen velocity (requires n_phi == 0): W_dev receives
 *      [batch][N][1][n], the weights of point i on its own window (zeros at Dirichlet walls).
 *      u_frozen_dev has the state dtype of `precision`.
 * W dtype: double for LMEP_PREC_FP64, float for LMEP_PREC_MIXED. */
LMEP_API lmep_status lmep_harvest_weights(lmep_handle* h, const lmep_grid* g, const lmep_operator* op,
                                 double dt, int32_t n_phi, const void* u_frozen_dev, void* W_dev,
                                 int32_t precision, void* stream);

/* The weights lmep_step reads for a scheme, harvested once for a
 * constant-coefficient problem (Sec. 2.1 step 3, Sec. 3.1 step 2):
 *  linear, ETD1, ETDRK2: [n][1+s][n] (s = 0, 1, 2), exactly lmep_harvest_weights
 *      with n_phi = s;
 *  ETDRK4 (Sec. 3): [n][6][n], per row class r the rows of exp(dt L), dt alpha,
 *      dt beta, dt gamma (alpha = phi_1 - 3 phi_2 + 4 phi_3, beta = 2 phi_2 -
 *      4 phi_3, gamma = 4 phi_3 - phi_2 at dt L, formed in FP64 from the rows of
 *      the augmented local matrix with p = 3), then exp(dt L / 2) and
 *      (dt/2) phi_1(dt L / 2) (augmented, p = 1, at dt/2).  Requires n <= 13.
 * W dtype: double for LMEP_PREC_FP64, float for LMEP_PREC_MIXED. */
LMEP_API lmep_status lmep_harvest_scheme_weights(lmep_handle* h, const lmep_grid* g, const lmep_operator* op,
                                                 double dt, int32_t scheme, void* W_dev, int32_t precision,
                                                 void* stream);

/* (a6) `nsteps` time steps of u in place (Sec. 3, Sec. 3.1 step 3).
 *  W_dev != NULL: stored constant-coefficient weights from
 *      lmep_harvest_scheme_weights (linear, ETD1, ETDRK2: the same as
 *      lmep_harvest_weights with n_phi = 0, 1, 2).
 *      Linear:  u+ = W0 u.   ETD1: u+ = W0 u + W1 N(u).
 *      ETDRK2:  a = W0 u + W1 N(u);  u+ = a + (W2 / dt)(N(a) - N(u)).
 *      ETDRK4:  a = E2 u + P2 N(u), b = E2 u + P2 N(a), c = E2 a + P2 (2 N(b) - N(u)),
 *               u+ = E u + A N(u) + B (N(a) + N(b)) + G N(c)  (rows as above).
 *      N: lmep_nonlin, with D1 the harvest row of the first-derivative matrix
 *      on the same window.  KdV and Burgers terms with ETD1/ETDRK2 need a
 *      periodic grid; ETDRK4 takes every boundary condition.
 *      Wide stencils (n = 17..25): the linear scheme on a periodic grid, with
 *      the row of class (n-1)/2 + window_shift; other schemes and boundaries
 *      return LMEP_ERR_UNSUPPORTED.
 *  W_dev == NULL: frozen velocity: every point rebuilds and exponentiates its
 *      own operator every step ((a1)-(a6) fused); requires the linear scheme.
 *  u_dev, work_dev: state dtype of `precision`, N elements each (batch * N for
 *  the frozen-velocity step); work_dev is scratch of the same size; the result
 *  is left in u_dev. */
LMEP_API lmep_status lmep_step(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, int32_t scheme,
                      int32_t nonlin, double dt, const void* W_dev, void* u_dev, void* work_dev,
                      int64_t nsteps, int32_t precision, void* stream);

/* Many independent constant-coefficient instances advanced by one persistent
 * launch per step (Allen-Cahn batch).  Instances share n, scheme, nonlin,
 * dt, the operator and precision; each has its own N_b, h_b and bc_b (periodic
 * or Neumann).  The caller allocates a workspace of lmep_batch_workspace_bytes
 * bytes; lmep_batch_prepare fills it (tile table and per-instance weights,
 * harvested on the device) and must run before lmep_step_batched.  State u
 * holds the instances back to back, instance b starting at element
 * o_b = sum_{c<b} round_up(N_c, 4) (every instance 16-byte aligned); the up to
 * three padding elements after an instance are never read or written.  The
 * state arrays therefore hold o_B = sum_b round_up(N_b, 4) elements. */
typedef struct lmep_batch_desc {
  int64_t B;                 /* number of instances */
  const int64_t* N_host;     /* [B] points per instance */
  const double* h_host;      /* [B] spacing per instance */
  const int32_t* bc_host;    /* [B] LMEP_BC_PERIODIC or LMEP_BC_NEUMANN */
  int32_t n;                 /* stencil width (odd, <= 13 for ETDRK2) */
  int32_t scheme;            /* lmep_scheme */
  int32_t nonlin;            /* lmep_nonlin (KdV not supported in batches) */
  int32_t tile;              /* staged points per warp tile: 0 = default; else a multiple
                                of 128 (one round of 128 points per 32 lanes).  A tile
                                updates `tile` points, or for ETDRK2
                                (tile / 128) * (128 - 2 * round_up((n - 1) / 2, 4)):
                                the first stage of a round spans its updated points
                                plus one stencil halo on each side.  A tile too large
                                for 3 slots per warp in shared memory is rejected. */
  int32_t block;             /* threads per CTA: 0 = default; 64, 128, 256 or 512 */
  int32_t ctas_per_sm;       /* persistent CTAs per SM: 0 = default */
  double dt;
  lmep_operator op;          /* shared coefficients (frozen_adv must be 0) */
} lmep_batch_desc;

LMEP_API lmep_status lmep_batch_workspace_bytes(const lmep_batch_desc* d, int32_t precision,
                                       size_t* bytes_out);
LMEP_API lmep_status lmep_batch_prepare(lmep_handle* h, const lmep_batch_desc* d, void* workspace_dev,
                               size_t workspace_bytes, int32_t precision, void* stream);
LMEP_API lmep_status lmep_step_batched(lmep_handle* h, const void* workspace_dev, void* u_dev,
                              void* work_dev, int64_t nsteps, void* stream);

/* One step of a prepared batch from u_in_dev to u_out_dev (distinct buffers,
 * no copy): one persistent launch, suitable for replay in a CUDA graph that
 * alternates the two buffers. */
LMEP_API lmep_status lmep_step_batched_once(lmep_handle* h, const void* workspace_dev, const void* u_in_dev,
                                            void* u_out_dev, void* stream);

/* Several frozen-velocity problems advanced together, one persistent
 * launch per step (Sec. 2.1 steps 1-3 fused with the banded update of
 * Sec. 3.1 step 3; every point rebuilds and exponentiates its local operator
 * at every step).  Instance b has its own grid (N, h, boundary, stencil width
 * n, departure centring), frozen operator and time step.  The row of exp(X)
 * of a point is l(r + a)^T exp(E) (see lmep_set_expm_method: Thm. 1 with the
 * General Exactness theorem), exp(E) computed once per instance on the device
 * by lmep_frozen_set_prepare (or again by lmep_frozen_set_refresh); a point
 * whose error bound is too large for that form is finished, within the same
 * call, by the finite series or Pade scaling and squaring, exactly as
 * lmep_step does for one instance.  The route follows the handle's
 * lmep_set_expm_method at prepare time (AUTO: factorised rows first; SERIES
 * or PADE: every point through those stages).
 *
 * State layout (u_in, u_out, state dtype of `precision`): the instances back
 * to back, instance b at element o_b = sum_{c<b} round_up(N_c, 4); the
 * padding elements are neither read nor written.  Results equal those of
 * lmep_step with a NULL weight array on each instance, bit for bit. */
typedef struct lmep_frozen_set_desc {
  int64_t B;                         /* instances, 1 .. 2^20 */
  const lmep_grid* grids_host;       /* [B]: odd n 3..15, batch <= 1, N < 2^31 (Neumann: N >= 2n) */
  const lmep_operator* ops_host;     /* [B]: frozen_adv != 0 */
  const double* dt_host;             /* [B]: > 0 */
  int32_t block;                     /* threads per CTA: 0 (default 256), 64, 128, 256 or 512 */
  int32_t points_per_thread;         /* 0 (default 2), 1, 2, 4 or 8; a CTA updates block * this points per
                                        tile: 1 or 2 points per thread together, 4 / 8 as 1 / 2 four times */
} lmep_frozen_set_desc;

/* Bytes of the workspace of a set (instance records, tile table, exp(E)
 * tables, one int32 per point for the rejected-point lists). */
LMEP_API lmep_status lmep_frozen_set_workspace_bytes(const lmep_frozen_set_desc* d, int32_t precision,
                                                     size_t* bytes_out);
/* Fill a caller-allocated workspace (16-byte aligned, at least
 * lmep_frozen_set_workspace_bytes bytes) and compute every instance's exp(E)
 * on the device.  Copies host tables and synchronises `stream`, so it is not
 * for stream capture.  The workspace then belongs to handle h until it is
 * prepared again. */
LMEP_API lmep_status lmep_frozen_set_prepare(lmep_handle* h, const lmep_frozen_set_desc* d, void* workspace_dev,
                                             size_t workspace_bytes, int32_t precision, void* stream);
/* Recompute the exp(E) tables of a prepared workspace on the device (one
 * launch, no host memory touched; the per-run setup cost of the set). */
LMEP_API lmep_status lmep_frozen_set_refresh(lmep_handle* h, void* workspace_dev, void* stream);
/* One step of every instance from u_in_dev to u_out_dev (distinct,
 * non-overlapping buffers): two launches (the lean kernel, then the fallback
 * for the points it rejected, which returns at once when there are none), no
 * host synchronisation, suitable for replay in a CUDA graph that alternates
 * the two buffers.  Calls that share a workspace must not overlap on the GPU.
 * u_in_dev and u_out_dev may also be page-locked host memory (cudaHostAlloc /
 * cudaMallocHost) on a system with unified addressing: the kernels then read
 * the input and write the output across the host link themselves, with no
 * separate copy (same results, bit for bit). */
LMEP_API lmep_status lmep_frozen_set_step_once(lmep_handle* h, const void* workspace_dev, const void* u_in_dev,
                                               void* u_out_dev, void* stream);

/* (a7) one reverse step of the frozen-velocity linear scheme (Dirichlet or
 * periodic), given the forward state u^n:
 *   lam_dev[k]  = sum_i lam_next[i] dF_i/du_k,
 *   *dnu_dev   += sum_i lam_next[i] dF_i/dnu   (double accumulator, nu = c2),
 * with dF_i/du_i containing the row of the Frechet derivative of the local
 * exponential in the direction dX/du_i = -dt frozen_adv D1, and dF_i/dnu the
 * one in the direction dX/dnu = dt D2 (Higham, Functions of Matrices, Thm 3.6).
 * Where the factorised form holds (the default route) these rows are closed
 * forms of l(z)^T exp(E); the FP32 form evaluates them in FP32 on the window's
 * values minus their linear interpolant (formed in FP64, its contribution
 * added exactly) and sums dnu in FP64; the Pade Frechet rows run in FP64.
 * scratch_dev: at least lmep_adjoint_scratch_bytes(g, precision) bytes.
 * u_dev, lam_next_dev, lam_dev: state dtype; dnu_dev: double[1]. */
LMEP_API lmep_status lmep_adjoint_scratch_bytes(const lmep_grid* g, int32_t precision, size_t* bytes_out);
LMEP_API lmep_status lmep_adjoint_step(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, double dt,
                              const void* u_dev, const void* lam_next_dev, void* lam_dev,
                              double* dnu_dev, void* scratch_dev, size_t scratch_bytes,
                              int32_t precision, void* stream);

/* The same reverse step as lmep_adjoint_step, for callers that cannot
 * allocate device memory: a plug-in whose host application's allocator owns
 * the whole device, a latency-critical loop that must not enter the driver's
 * allocator, a sandbox with a device budget fixed before the library loads.
 * This entry point allocates nothing and takes no handle: its scratch is a
 * file-scope static __device__ array of 8 MiB inside the library, held by
 * every GPU that loads the library until the process exits.  The paper has
 * no counterpart; this is an interface for such callers only.
 *  - Limit: grids needing more than 8 MiB of scratch (N (n + 1) elements of
 *    the state dtype + 4 N + 256 bytes, e.g. N <= 63548 at n = 15 in FP64,
 *    N <= 123358 at n = 15 in the FP32 form) are rejected with
 *    LMEP_ERR_INVALID and a message; use lmep_adjoint_step.
 *  - Route: without a handle there is no cached exp(E) table, so every point
 *    takes the Pade Frechet derivatives (the route lmep_adjoint_step takes
 *    under LMEP_EXPM_PADE); on the Burgers benchmark grids that is about two
 *    orders of magnitude slower than the default route of lmep_adjoint_step,
 *    with the same parity tolerances.
 *  - The first call on each device, with that device current, looks up the
 *    array's device address (cudaGetSymbolAddress) and caches it; later
 *    calls check the cached address against the current context (after a
 *    cudaDeviceReset it is looked up again).  Make the first call on a
 *    device, and the first after a reset, before any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents;
 *    every scratch element a call reads is written earlier in the same call.
 *    Calls that overlap on the GPU (other streams, other threads) race on it.
 *  - Non-finite results are not reported by this entry point (there is no
 *    handle); check the outputs.
 *  - One instance per call: grids with batch > 1 are rejected.
 * Arguments and dnu_dev accumulation are those of lmep_adjoint_step. */
LMEP_API lmep_status lmep_adjoint_step_noalloc(const lmep_grid* g, const lmep_operator* op, double dt,
                                               const void* u_dev, const void* lam_next_dev, void* lam_dev,
                                               double* dnu_dev, int32_t precision, void* stream);

/* Diagnostics of the frozen-velocity path: for every point i write
 * stats_dev[3 i .. 3 i + 2] = (Pade degree m, squarings s, full squarings a)
 * exactly as the fused step chooses them for state u_dev (the remaining
 * 2^(s-a) - 1 squaring factors act on the harvested row only); (0, 0, 0)
 * marks a row taken from the finite series in the precision's product type,
 * (1, 0, 0) one taken from the finite series in FP64 (FP32 form only) and
 * (2, 0, 0) one taken from the factorised form (see lmep_set_expm_method).
 * Runs the
 * frozen-velocity kernel without writing weights.  Dirichlet wall points are
 * left untouched.  u_dev: state dtype of `precision`; stats_dev: int32[N][3]. */
LMEP_API lmep_status lmep_frozen_stats(lmep_handle* h, const lmep_grid* g, const lmep_operator* op, double dt,
                                       const void* u_dev, int32_t* stats_dev, int32_t precision, void* stream);

/* How the frozen-velocity launches of handle h (lmep_step and
 * lmep_harvest_weights with a frozen operator, lmep_frozen_stats) evaluate a
 * row of exp(X) (Sec. 2.1 step 4).  Without its identity term the local
 * matrix X = a Dh1 + E, E = c2h Dh2 + c3h Dh3, is a polynomial without
 * constant term in the window's differentiation matrix: it is nilpotent
 * (X^n = 0 on n nodes), so a row of its exponential is the finite Taylor sum
 * of n terms, and its parts commute, so row r of exp(X) is l(r + a)^T exp(E)
 * with l the Lagrange weights of the window (Thm. 1) and exp(E) the same for
 * every point.
 *  LMEP_EXPM_SERIES: the finite sum, with an a-posteriori error bound per
 *         point, beta = sum_k |row of |X|^k|_1 / k! (the computed row is
 *         within about 2 u beta of the exact one, u the unit roundoff).  The
 *         FP32 form sums in FP32 while beta <= 16, else in FP64 while
 *         beta <= 2^20; the FP64 path in FP64 while beta <= 64; a point with
 *         a larger bound takes the PADE route.
 *  LMEP_EXPM_AUTO (the default): first the factorised row l(r + a)^T exp(E)
 *         in the precision's product type, where its bound
 *         sum_j |l_j| |row j of exp(E)|_1 is at most 16, the rest as SERIES;
 *         exp(E) is computed once per (n, dt c2 / h^2, dt c3 / h^3) in FP64
 *         (Pade) and kept in the handle (the first call for an operator
 *         synchronises `stream` once; inside a stream capture an operator not
 *         seen before takes SERIES).  The factorised row avoids the rounding
 *         of the assembled X: on the Burgers rows it is within a few 1e-16 of
 *         the exact rational rows, where exp of the rounded FP64 X (SERIES,
 *         PADE) can be off by ~2e-12.
 *  LMEP_EXPM_PADE: Pade scaling and squaring (Higham 2005; Al-Mohy and
 *         Higham 2009) for every point.
 * All routes meet the same parity tolerances.  Other calls are unaffected.
 * Returns LMEP_ERR_INVALID for a NULL handle or an unknown method. */
LMEP_API lmep_status lmep_set_expm_method(lmep_handle* h, int32_t method);

/* Bound of the waits of the streaming apply kernels of handle h (lmep_step
 * with stored weights on periodic and Neumann grids, lmep_step_batched and
 * lmep_step_batched_once): a warp waits at most `polls` polls of its tile's
 * mbarrier for the bulk copies of its next tile; if they have not all landed
 * it gives up, sets the timeout flag (reported as LMEP_ERR_TIMEOUT by
 * lmep_sync_status), waits with the default bound for its copies still in
 * flight and leaves its remaining tiles not computed.  Default (and polls < 0):
 * 2^20 polls, far longer than any copy; 0 makes every such wait give up at
 * once -- for tests of the timeout path, which leaves the context usable.
 * polls > 2^30 is rejected. */
LMEP_API lmep_status lmep_set_wait_limit(lmep_handle* h, int64_t polls);

/* Synchronise `stream`, read and clear the device status flags.
 * Returns LMEP_ERR_TIMEOUT if a kernel gave up a bounded wait for one of its
 * own bulk copies (its outputs are then incomplete), else LMEP_ERR_NONFINITE
 * if any kernel produced Inf/NaN since the last call. */
LMEP_API lmep_status lmep_sync_status(lmep_handle* h, void* stream);

/* Non-uniform grids (Sec. 4.3.3, e.g. Chebyshev nodes): every node has its
 * own local differentiation matrices, so its weights are harvested once per
 * node and stored.  Nodes x_dev: double[N], strictly increasing, both ends
 * Dirichlet walls (kept at bc_lo / bc_hi and never updated).  Point i uses
 * the window of nodes start_i .. start_i + n - 1, start_i = clamp(i - (n-1)/2,
 * 0, N - n), harvest row i - start_i (one-sided next to the walls).  Its
 * derivative matrices come from Fornberg's recursion on the window's nodes (in
 * local coordinates scaled by the window's mean spacing), X_i = dt (c0 + c1 D1
 * + c2 D2 + c3 D3), and the rows are those of lmep_harvest_scheme_weights for
 * the scheme (1, 2, 3 or 6 rows per point), stored W_dev[N][rows][n] in the
 * state dtype.  3 <= n <= 15 odd, n + n_phi(scheme) <= 16, N < 2^31;
 * op->frozen_adv must be 0. */
LMEP_API lmep_status lmep_harvest_nodes(lmep_handle* h, int64_t N, const double* x_dev, int32_t n,
                                        const lmep_operator* op, double dt, int32_t scheme, void* W_dev,
                                        int32_t precision, void* stream);
/* `nsteps` steps of u in place with the stored per-node rows of
 * lmep_harvest_nodes (same N, n, scheme, dt): linear, ETD1, ETDRK2 or ETDRK4
 * (formulas of lmep_step), N(u) = u - u^3 (LMEP_N_ALLEN_CAHN) or none
 * (linear scheme).  work_dev: scratch of N state values. */
LMEP_API lmep_status lmep_step_nodes(lmep_handle* h, int64_t N, int32_t n, int32_t scheme, int32_t nonlin,
                                     double dt, double bc_lo, double bc_hi, const void* W_dev, void* u_dev,
                                     void* work_dev, int64_t nsteps, int32_t precision, void* stream);

/* Fourier symbol of one harvested row (Sec. 4.1's spectral footprint, the
 * amplification factor of a constant-coefficient periodic step):
 *   G(theta_q) = sum_j w_j e^{i theta_q (j - r)},  q < M,
 * w_dev: double[n] (e.g. row r of exp(dt L) from lmep_harvest_weights in
 * FP64), theta_dev: double[M], G_dev: double[M][2] (real, imaginary part).
 * |G| > 1 for some theta means the mode grows.  1 <= n <= 64, 0 <= r < n. */
LMEP_API lmep_status lmep_amplification(const double* w_dev, int32_t n, int32_t r, const double* theta_dev,
                                        int64_t M, double* G_dev, void* stream);

/* FMA-chain microbenchmark (all SMs): *flops_out receives achieved FLOP/s
 * (2 per FMA) of FP64 (precision 0) or FP32 (precision 1) FMAs.  Synchronous. */
LMEP_API lmep_status lmep_fma_peak(int32_t precision, double* flops_out);

LMEP_API const char* lmep_status_string(lmep_status s);
/* Thread-local text of the last error raised on this thread ("" if none). */
LMEP_API const char* lmep_last_error(void);
/* Library version string. */
LMEP_API const char* lmep_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LMEP_H */
