/*
 * phicomb -- GB300-native (sm_103a) solver for linear combinations of phi-function actions
 *
 *     w_i = sum_{j=0}^{p} alpha_i^j phi_j(t_i A) v_j,   i = 1..r,
 *
 * with phi_0(z) = e^z and phi_j(z) = sum_k z^k/(k+j)!  (Al-Mohy, "Computing Linear Combinations of
 * phi-Function Actions for Exponential Integrators", arXiv 2509.26475, eqs. (1.2)-(1.3)).
 *
 * Two calls carry the method:
 *   phic_select_params  -- Algorithm 1 (Section 3): the spectral shift xi* and the scaling s from a
 *                          guarded power basis of A, the objective f(xi) and Brent's minimiser.
 *   phic_solve          -- Algorithm 3 (Section 4): the block scaling-and-recovering truncated Taylor
 *                          method for all r combinations at once (Algorithm 2 is its r = 1 case).
 * The parameters from phic_select_params depend on A only and are meant to be reused across calls
 * (Section 6), so they stay in device memory and phic_solve reads them from there.
 *
 * Conventions
 *   - Every pointer documented "device" must point to memory of the current CUDA device; "host"
 *     pointers are read before the call returns.  Nothing is retained after a call returns.
 *   - Ownership: the caller owns every device buffer, including the workspace.  The library allocates
 *     no device memory, keeps no state between calls other than cached launch configurations and the
 *     host-side batch handles it returns, and never synchronises the stream (except the batch set-up
 *     and autotuning calls, which say so).  All work is enqueued on `stream` (0 = legacy default stream).
 *   - Device-side outcomes (non-finite norms, the term cap, a timed-out grid barrier, a bad column
 *     index) are written as a phic_status into phic_params.status / phic_stats.status in device
 *     memory; the return value of a call only reports what the host could check before enqueuing
 *     (arguments, workspace size, launch errors).  Read the device status after the stream has
 *     reached the call.
 *   - Indices are int32: n and nnz must be below 2^31.
 *   - Real arithmetic only (the paper allows complex A; that is not supported).
 *   - All functions are thread-safe; concurrent calls must use distinct workspaces.
 */
#ifndef PHICOMB_H
#define PHICOMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* phic_stream_t; /* identical to cudaStream_t */

typedef enum {
  PHIC_OK = 0,
  PHIC_INVALID_ARG = 1,        /* bad argument or malformed CSR (found on the host or on the device) */
  PHIC_NONFINITE = 2,          /* a norm became Inf or NaN */
  PHIC_TERM_CAP = 3,           /* a Taylor loop reached max_terms without passing the truncation test */
  PHIC_TIMEOUT = 4,            /* a grid barrier wait exceeded the spin limit; the kernel returned */
  PHIC_CUDA_ERROR = 5,         /* a CUDA runtime call failed (launch, memset, attribute query) */
  PHIC_WORKSPACE_TOO_SMALL = 6 /* ws_bytes below the size reported by the *_workspace_size query */
} phic_status;

typedef enum { PHIC_F64 = 0, PHIC_F32 = 1 } phic_prec;

/* Sparse operator A in CSR form (device arrays).  rowptr[n+1] (rowptr[0] = 0, non-decreasing,
 * rowptr[n] = nnz), colidx[nnz] in [0, n), values[nnz] of type `prec`.  Columns inside a row may come
 * in any order; duplicates are summed.  The arrays are checked on the device before use: a malformed
 * rowptr or a column index out of range sets PHIC_INVALID_ARG and no out-of-range address is read. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* colidx;
  const void* values;
  int32_t prec; /* phic_prec of values */
} phic_csr;

/* Options of Algorithm 1 (defaults from Section 3: m = 61, tol = 2^-53, delta = 0.8). */
typedef struct {
  int32_t m;              /* degree of the power basis, 1 <= m <= 128 (default 61) */
  double tol;             /* target tolerance used in s = s0 f(xi*) / (tol m!)^(1/m) */
  double delta;           /* guard factor: g_max = delta log(realmax), g_min = delta log(realmin) */
  uint64_t seed;          /* seed of the splitmix64 unit vector when v is NULL */
  int32_t max_evals;      /* objective evaluations allowed to Brent's method (default 200) */
  double spin_limit_ms;   /* bound on one grid-barrier wait (default 2000 ms) */
} phic_select_opts;

/* Parameters produced by phic_select_params (device memory), consumed by phic_solve. */
typedef struct {
  double xi;       /* optimal shift xi* (the paper's xi; mu = e^{t xi / s} is derived in phic_solve) */
  double s;        /* scaling parameter s > 0 (before multiplication by max|t_i|) */
  double s0;       /* preliminary scale: geometric mean of the last accepted growth factors */
  double f_star;   /* objective value f(xi*) */
  int32_t r;       /* last accepted power index of the guarded basis */
  int32_t evals;   /* objective evaluations used by Brent's method */
  int32_t status;  /* phic_status of the device-side run */
  int32_t pad;
} phic_params;

/* Per-solve record written by phic_solve (device memory). */
typedef struct {
  int32_t status;          /* phic_status of the device-side run */
  int32_t s_int;           /* scaling count ceil(s max|t_i|) (at least 1) */
  int32_t series_terms;    /* k when the block series loop stopped */
  int32_t max_inner_terms; /* largest term count of one recovery step */
  int64_t recovery_terms;  /* total Taylor terms over the s_int - 1 recovery steps */
  int64_t spmm_count;      /* sparse block products performed */
  double xi;               /* shift used */
  double s;                /* scaling parameter used */
  int32_t op_format;       /* copy of B = (A - xi I) 2^-eA the products read: PHIC_OP_* */
  int32_t op_slots;        /* its diagonals (DIA) or entries per row (ELL); 0 otherwise */
} phic_stats;

/* phic_stats.op_format.  For stored operators the setup picks DIA (the values of at most 16 diagonals, row-aligned) when
 * the stored diagonals are that few and fill the rows well, else ELL (a fixed number of slots per row,
 * at most 64) when n times the longest row fits the copy's room, else the entries in CSR order. */
#define PHIC_OP_CSR 0
#define PHIC_OP_ELL 1
#define PHIC_OP_DIA 2
#define PHIC_OP_LOWRANK 3
#define PHIC_OP_FUNCTION 4 /* a phic_fn_op: products by the caller's function */

/* Flags of phic_solve */
#define PHIC_NO_V0 1u /* V holds v_1..v_p only (p rows); the result is sum_{j>=1} alpha_i^j phi_j(t_i A) v_j
                         (the output option of Section 4 for an omitted v_0) */
#define PHIC_PHASE_SERIES 0x10u  /* enqueue only the block-series kernel (setup and the S loop) */
#define PHIC_PHASE_RECOVER 0x20u /* enqueue only the recovery kernel; the workspace must hold the state left
                                    by a PHIC_PHASE_SERIES call with the same arguments, earlier on the stream.
                                    Neither phase flag: both kernels, in order. */

/* Limits */
#define PHIC_MAX_R 16   /* combinations per call */
#define PHIC_MAX_P 15   /* highest phi index */
#define PHIC_MAX_WIDTH 128 /* (p+1) r, the column count of the block series */

/* Fills `opts` with the defaults of Algorithm 1. */
void phic_select_opts_default(phic_select_opts* opts);

/* Workspace bytes needed by phic_select_params for an n-row operator and degree m:
 * the basis V_0..V_m (n (m+1) doubles), one scratch vector and a control block. */
phic_status phic_select_workspace_size(int64_t n, int32_t m, size_t* bytes);

/* Algorithm 1 (Section 3).  Builds the guarded power basis V_k = A V_{k-1} from the unit vector v
 * (device, n doubles, normalised internally; NULL draws components 2u-1 from splitmix64(seed, i)),
 * stops at the first k whose log-norm would break the overflow/underflow guard, sets s0 from the
 * last five growth factors, normalises and extends the basis to degree m, minimises
 * f(xi) = ||sum_k binom(m,k) (-xi/s0)^(m-k) V_k||_2^(1/m) over [-sqrt(n) s0, sqrt(n) s0] with Brent's
 * method, and writes xi*, s = s0 f(xi*) / (tol m!)^(1/m) and diagnostics to params_dev (device).
 * All arithmetic is FP64 whatever the precision of A's values.  ws (device, 256-byte aligned) must
 * hold phic_select_workspace_size(n, m) bytes. */
phic_status phic_select_params(const phic_csr* A, const phic_select_opts* opts, const double* v, void* ws,
                               size_t ws_bytes, phic_params* params_dev, phic_stream_t stream);

/* Writes user-chosen xi and s into params_dev (device) on `stream`, for callers that skip Algorithm 1. */
phic_status phic_params_set(phic_params* params_dev, double xi, double s, phic_stream_t stream);

/* Workspace bytes needed by phic_solve for n rows, nnz stored entries, p, r and the storage precision:
 * a copy of the values holding A_1 = A - xi I, the block tiles V, D (two each), S, F (two), E, and
 * control blocks. */
phic_status phic_solve_workspace_size(int64_t n, int64_t nnz, int32_t p, int32_t r, int32_t prec, size_t* bytes);

/* The lane layout the solve kernels give a row-major block tile of w columns (a host query; no device
 * work).  Algorithm 3's series carries the (p+1) r columns of its block series, the recovery the 2r (r when
 * p = 0) columns of F.  Each row is handled by L lanes of cw columns, grouped into Lp2 (the next power of
 * two >= L) consecutive lanes; idle lanes of a group cost their warp's instructions all the same.  odd_cw != 0
 * allows 3 or 5 columns a lane where that leaves fewer lane slots (Lp2 cw) than the power-of-two widths,
 * as phic_solve does for its series tile.
 *   w       columns, 1 .. PHIC_MAX_WIDTH
 *   prec    PHIC_F64 or PHIC_F32
 *   out     host int32[5]: {w, the tile's row stride ws (elements), cw, L, Lp2}
 * Returns PHIC_INVALID_ARG for any other w or prec, or a null out. */
phic_status phic_tile_layout(int32_t w, int32_t prec, int32_t odd_cw, int32_t* out);

/* Algorithm 3 (Section 4): w_i = sum_j alpha_i^j phi_j(t_i A) v_j for i = 1..r.
 *   A       CSR operator; A->prec must equal `prec`.
 *   p, r    0 <= p <= PHIC_MAX_P, 1 <= r <= PHIC_MAX_R, (p+1) r <= PHIC_MAX_WIDTH.
 *   V       device, (p+1) x n row-major in `prec`: v_j starts at V + j n (with PHIC_NO_V0: p x n, v_1..v_p).
 *   t       host, r abscissae t_i (any real values; t_i = 0 allowed).
 *   alpha   host, r weights alpha_i (the combination uses alpha_i^j).
 *   tol     truncation tolerance of every Taylor loop (2^-53 for FP64 accuracy, 2^-24 for FP32).
 *   params_dev  device phic_params (xi and s are read; typically from phic_select_params).
 *   W       device, r x n row-major in `prec`: w_i at W + i n.  May not alias V.
 *   ws      device workspace, 256-byte aligned, phic_solve_workspace_size(...) bytes.
 *   stats_dev   device phic_stats or NULL.
 *   max_terms   cap on the terms of one Taylor loop (<= 0 selects 610); reaching it sets PHIC_TERM_CAP.
 * prec = PHIC_F32 keeps A, V, the Taylor terms and W in FP32 with FP32 accumulation (compensated sums in
 * the sparse products); the scalar parameters (s, xi, mu, the nilpotent factors, the norms' comparison)
 * stay FP64.  When params_dev comes from Algorithm 1 (s0 and f_star positive), an FP32 solve raises s to
 * at least s0 f_star / (ln(2^24) / 2), so that no step's Taylor terms grow beyond about e^8.3 before they
 * cancel: their FP32 rounding, not the truncation tolerance, bounds an FP32 result.  phic_stats.s reports
 * the s used. */
phic_status phic_solve(const phic_csr* A, int32_t p, int32_t r, const void* V, const double* t, const double* alpha,
                       double tol, const phic_params* params_dev, uint32_t flags, int32_t max_terms, void* W, void* ws,
                       size_t ws_bytes, phic_stats* stats_dev, int32_t prec, phic_stream_t stream);

/* Size of the static scratch array used by phic_solve_noalloc (32 MiB per device). */
#define PHIC_NOALLOC_MAX_BYTES (32u << 20)

/* phic_solve without a caller-supplied workspace (the paper has no counterpart: this is an interface for
 * callers that cannot allocate device memory).  Some callers may not call cudaMalloc at all: a plug-in
 * running inside a host application that owns every device allocation, a latency-critical loop that
 * cannot afford cudaMalloc's device-wide synchronisation, or a system allowed to allocate only at
 * start-up.  This entry point takes the same arguments as phic_solve minus ws / ws_bytes and keeps its
 * scratch in a file-scope static device array of PHIC_NOALLOC_MAX_BYTES that every GPU loading the
 * library holds until the process exits.  It allocates nothing itself.
 *   - Size limit: when phic_solve_workspace_size(n, nnz, p, r, prec) exceeds PHIC_NOALLOC_MAX_BYTES the
 *     call returns PHIC_WORKSPACE_TOO_SMALL and enqueues nothing (e.g. FP64, p = 3, r = 2 and a 7-point
 *     stencil fit up to about 60,000 rows: the solve workspace takes about 557 bytes a row there).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current and caches it; make that first call before any stream capture.  The cached address
 *     belongs to the device's primary context: after cudaDeviceReset on a device, the library's module is
 *     loaded again and the array may move, so do not call phic_solve_noalloc on that device again in the
 *     same process.
 *   - Every call shares the one array, which keeps the previous call's contents (the call clears the
 *     parts that must start at zero).  Calls whose work overlaps on the GPU -- on different streams, or
 *     from different host threads -- race on the array and give undefined results: serialise them.
 *   - flags may be 0 or PHIC_NO_V0; A, V, t, alpha, params_dev, W, stats_dev, prec and stream are as in
 *     phic_solve. */
phic_status phic_solve_noalloc(const phic_csr* A, int32_t p, int32_t r, const void* V, const double* t,
                               const double* alpha, double tol, const phic_params* params_dev, uint32_t flags,
                               int32_t max_terms, void* W, phic_stats* stats_dev, int32_t prec, phic_stream_t stream);

/* ---- Matrix-free low-rank operators ----------------------------------------------------------------
 * A = U W^T with U and W n x k (k <= PHIC_MAX_RANK), applied as x -> U (W^T x) with O(n k) work and no
 * n x n matrix: the family of large test operators of the paper's third experiment (Section 6), where
 * sum_j phi_j(tA) v_j has the closed form sum_j v_j / j! + U (t sum_j phi_{j+1}(tM) (W^T v_j)) for
 * W = U M^T.  Algorithms 1 and 3 run as for CSR operators; each product with A takes one team-wide
 * reduction Z = W^T X (k x width, summed in FP64) before its row pass, and A - xi I is applied with the
 * shift on every row.  The bound on ||A - xi I||_inf that scales the Taylor terms is
 * max_i sum_q |U_iq| sum_j |W_jq| + |xi|. */
#define PHIC_MAX_RANK 8

typedef struct {
  int64_t n;
  int32_t k;        /* rank, 1 <= k <= PHIC_MAX_RANK */
  int32_t prec;     /* PHIC_F64 or PHIC_F32: the type of U and W */
  const void* U;    /* device, n x k row-major: U(i, q) at U[i k + q] */
  const void* W;    /* device, n x k row-major */
} phic_lowrank;

/* Workspace of phic_lowrank_select_params: that of phic_select_params plus the partial sums of W^T x. */
phic_status phic_lowrank_select_workspace_size(int64_t n, int32_t k, int32_t m, size_t* bytes);

/* Algorithm 1 for A = U W^T (FP64 arithmetic whatever A->prec); as phic_select_params otherwise. */
phic_status phic_lowrank_select_params(const phic_lowrank* A, const phic_select_opts* opts, const double* v, void* ws,
                                       size_t ws_bytes, phic_params* params_dev, phic_stream_t stream);

/* Workspace of phic_lowrank_solve; requires (p+1) r k <= 256. */
phic_status phic_lowrank_solve_workspace_size(int64_t n, int32_t k, int32_t p, int32_t r, int32_t prec, size_t* bytes);

/* Algorithm 3 for A = U W^T; arguments as phic_solve (A->prec must equal prec; (p+1) r k <= 256). */
phic_status phic_lowrank_solve(const phic_lowrank* A, int32_t p, int32_t r, const void* V, const double* t,
                               const double* alpha, double tol, const phic_params* params_dev, uint32_t flags,
                               int32_t max_terms, void* W, void* ws, size_t ws_bytes, phic_stats* stats_dev,
                               int32_t prec, phic_stream_t stream);

/* ---- Operators given as functions ------------------------------------------------------------------
 * Algorithms 1 and 3 need A only through products A X (Sections 3 and 4); here the caller supplies that
 * product as a function, for operators that are not stored as a matrix (a stencil applied on the fly, a
 * convolution, a composition of factors).  The function enqueues Y = A X on the stream it is given and
 * returns; it must not synchronise or allocate.
 *
 * phic_fn_solve runs Algorithm 3 as one CUDA graph: the library records the caller's product into the
 * graph once for each place it occurs (the series term, the first-block recovery, the recovery term), by
 * stream capture, and every data-dependent loop of the method (the series' terms, the recovery's steps and
 * each step's terms) is a conditional WHILE node whose condition the library's kernels set on the device,
 * so that no Taylor term returns to the host.  The function is therefore called during the call to
 * phic_fn_solve, on a capturing stream, and its work must be capturable (kernel launches, memsets and
 * device-to-device copies on that stream only).
 *
 * phic_fn_select_params runs Algorithm 1 with the products enqueued directly on `stream` (in FP64), one
 * per basis vector, and synchronises `stream` after each (the guard and Brent's method are evaluated on
 * the host between device passes). */

/* Y = A X for the columns 0..w-1 of an n-row block, on `stream`.  X and Y are device arrays of type prec
 * (PHIC_F64 or PHIC_F32), row-major: X(i, c) at X[i ldx + c], Y(i, c) at Y[i ldy + c]; ldx, ldy >= w (in
 * elements).  X and Y do not overlap.  Return 0 on success, non-zero to make the calling entry point fail
 * with PHIC_CUDA_ERROR.  phic_fn_select_params calls it with prec = PHIC_F64 whatever the operator's
 * precision. */
typedef int32_t (*phic_apply_fn)(void* ctx, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t w,
                                 int32_t prec, phic_stream_t stream);

typedef struct {
  int64_t n;
  int32_t prec;          /* precision of the solve's tiles (PHIC_F64 or PHIC_F32) */
  int32_t pad;
  phic_apply_fn apply;
  void* ctx;             /* passed to apply */
  double norm_bound;     /* an upper bound of ||A||_inf (> 0): scales the Taylor terms so that
                            ||(A - xi I) 2^-eA||_inf < 1, as the stored operators' own norms do */
} phic_fn_op;

/* Workspace bytes of phic_fn_select_params: the basis V_0..V_m (n (m+1) doubles) and per-chunk partials. */
phic_status phic_fn_select_workspace_size(int64_t n, int32_t m, size_t* bytes);

/* Algorithm 1 (Section 3) for a function operator: as phic_select_params, with the products of the
 * power basis and its extension by A->apply (FP64).  Synchronises `stream` once per basis vector and once
 * per objective evaluation; writes params_dev (device) on `stream` before returning. */
phic_status phic_fn_select_params(const phic_fn_op* A, const phic_select_opts* opts, const double* v, void* ws,
                                  size_t ws_bytes, phic_params* params_dev, phic_stream_t stream);

/* Workspace bytes of phic_fn_solve: the tiles V, D, S and the product Y ((p+1) r columns each), G and E
 * (2r columns; r when p = 0) and a control block. */
phic_status phic_fn_solve_workspace_size(int64_t n, int32_t p, int32_t r, int32_t prec, size_t* bytes);

/* Algorithm 3 (Section 4) for a function operator; arguments as phic_solve (prec must equal A->prec;
 * flags 0 or PHIC_NO_V0).  Builds, instantiates and launches one CUDA graph on `stream` and releases it
 * (the launch completes asynchronously; the graph is not kept).  The caller's apply is called three times
 * during the call, on a capturing stream.  Returns PHIC_CUDA_ERROR when apply fails or its work cannot be
 * captured. */
phic_status phic_fn_solve(const phic_fn_op* A, int32_t p, int32_t r, const void* V, const double* t,
                          const double* alpha, double tol, const phic_params* params_dev, uint32_t flags,
                          int32_t max_terms, void* W, void* ws, size_t ws_bytes, phic_stats* stats_dev,
                          int32_t prec, phic_stream_t stream);

/* A CSR product in the form of phic_apply_fn (ctx: a const phic_csr* whose arrays are device memory and
 * whose prec matches the call's prec for FP32 calls; FP64 calls on an FP32 CSR read its values as FP32 and
 * compute in FP64).  An example of the interface, and the product the tests compare the function path with. */
int32_t phic_csr_apply(void* ctx, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t w, int32_t prec,
                       phic_stream_t stream);

/* ---- Batched solves -------------------------------------------------------------------------------
 * Many independent instances (each its own A, p, r, t, alpha, tol and precision) in ONE persistent
 * cooperative launch.  The paper solves one instance per call; this interface serves workloads of many
 * uneven problems (an integrator over many operators, a request stream).  Each instance is run by a
 * team of CTAs with the same kernels' code as phic_select_params / phic_solve, synchronised by a
 * bounded barrier of its own; a host planner sizes the teams from n (phic_batch_config.rows_per_cta)
 * and orders the work longest first over the launch's CTAs.  A solve's result does not depend on its
 * team size or on the other instances in the launch (the truncation tests use infinity norms, which are
 * maxima); Algorithm 1's sums of squares are rounded per team, so with PHIC_BATCH_SELECT the selected
 * s and xi can differ in the last bits from phic_select_params.
 * The handle (phic_batch) lives in host memory allocated by the library; every device buffer,
 * including the workspace, is the caller's. */

#define PHIC_BATCH_SELECT 0x100u   /* run Algorithm 1 for the instance first, writing *params (its tol is the
                                      item's tol; m, delta, seed and max_evals come from the options) */
#define PHIC_BATCH_NO_SOLVE 0x200u /* run Algorithm 1 only (requires PHIC_BATCH_SELECT) */

/* One instance of a batch. */
typedef struct {
  phic_csr A;              /* operator (device arrays, checked on the device as in phic_solve) */
  int32_t p, r;            /* as in phic_solve */
  uint32_t flags;          /* PHIC_NO_V0, PHIC_BATCH_SELECT, PHIC_BATCH_NO_SOLVE */
  int32_t max_terms;       /* as in phic_solve (<= 0 selects 610) */
  const void* V;           /* device, as in phic_solve */
  void* W;                 /* device, as in phic_solve (may be NULL with PHIC_BATCH_NO_SOLVE) */
  phic_params* params;     /* device: read by the solve; written first when PHIC_BATCH_SELECT is set */
  phic_stats* stats;       /* device or NULL, as in phic_solve */
  const double* v_select;  /* device unit vector for Algorithm 1, or NULL (splitmix64 of the options' seed) */
  double tol;              /* truncation tolerance, as in phic_solve */
  double s_hint;           /* estimate of s for the planner's cost model only; <= 0: see phic_batch_create */
  double t[PHIC_MAX_R];    /* abscissae t_1..t_r (host copy) */
  double alpha[PHIC_MAX_R];/* weights alpha_1..alpha_r (host copy) */
} phic_batch_item;

/* Launch shape of a batch (the autotuner's search space). */
typedef struct {
  int32_t rows_per_cta;   /* an instance of n rows gets ceil(n / rows_per_cta) CTAs, at most the grid
                             (<= 0 selects 4096; at least 256) */
  int32_t blocks_per_sm;  /* resident CTAs per SM: 2 or 3 (<= 0 selects 2) */
  int32_t max_steps;      /* recovery outer steps per instance per launch (<= 0: run to the end).  With a
                             bound, a launch may stop an instance between outer steps; launching the
                             same batch again (phic_batch_resume) continues it. */
  int32_t reserved;
} phic_batch_config;

/* Planner output. */
typedef struct {
  int32_t grid;            /* CTAs of the launch (SMs x blocks_per_sm) */
  int32_t blocks_per_sm;
  int32_t count;           /* instances */
  int32_t max_team;        /* largest team */
  int64_t entries;         /* schedule entries (sum of team sizes) */
  double est_makespan_us;  /* cost-model estimate of the launch */
  double est_busy_frac;    /* estimated busy CTA time / (grid x makespan) */
} phic_batch_info;

typedef struct phic_batch phic_batch;

/* Device workspace bytes of a batch: per instance the workspaces of phic_select_params (with
 * PHIC_BATCH_SELECT) and phic_solve (unless PHIC_BATCH_NO_SOLVE), plus the control blocks, the
 * instance table and the schedule.  opts may be NULL (defaults). */
phic_status phic_batch_workspace_size(const phic_batch_item* items, int32_t count, const phic_select_opts* opts,
                                      size_t* bytes);

/* Checks the items (host side, as phic_solve does), lays out ws (device, 256-byte aligned), plans the
 * teams and the schedule for cfg (NULL: defaults) and copies the instance table and the schedule into
 * ws on `stream`, synchronising `stream` before returning (set-up call, not for capture).  items is
 * read before the call returns.  *out receives the handle.
 * An item with PHIC_BATCH_SELECT and a solve but no s_hint (<= 0) is planned with the hint
 * ||A||_inf / (2 (tol m!)^(1/m)), m = opts->m: Algorithm 1's s = s0 f* / (tol m!)^(1/m) with s0 f*
 * taken as ||A - xi I|| ~ ||A||_inf / 2.  The norms are computed on `stream` first, in ws.
 * phic_batch_plan_host, which reads no device memory, uses s_hint as given (<= 0: one scaling step). */
phic_status phic_batch_create(const phic_batch_item* items, int32_t count, const phic_select_opts* opts,
                              const phic_batch_config* cfg, void* ws, size_t ws_bytes, phic_stream_t stream,
                              phic_batch** out);

/* Enqueues the batch: a memset of the instances' control blocks and one cooperative launch.  No host
 * synchronisation, no allocation: the pair can be captured into a CUDA graph and replayed; each launch
 * recomputes every instance from V (and, with PHIC_BATCH_SELECT, from A). */
phic_status phic_batch_launch(phic_batch* b, phic_stream_t stream);

/* For a batch created with max_steps > 0: enqueues the next slice, in which every instance continues its
 * recovery from where the previous launch stopped (instances already finished do no work).  Call it after
 * one phic_batch_launch until phic_stats.status of every instance is final (the host reads
 * phic_stats.recovery_terms / the state to know; see phic_batch_pending). */
phic_status phic_batch_resume(phic_batch* b, phic_stream_t stream);

/* Number of instances not finished after the work enqueued so far: enqueues a small kernel on `stream`
 * that counts them into *pending_dev (device int32). */
phic_status phic_batch_pending(const phic_batch* b, int32_t* pending_dev, phic_stream_t stream);

phic_status phic_batch_info_get(const phic_batch* b, phic_batch_info* info);

/* Releases the handle (host memory only). */
void phic_batch_destroy(phic_batch* b);

/* The planner alone, on the host (no CUDA call; the items' device pointers are not dereferenced): the
 * team size of each instance (team[count]) and the schedule of a launch of `grid` CTAs as
 * sched_ptr[grid + 1] and (instance, rank) pairs sched[2 * entries], as phic_batch_create would build
 * them for cfg.  Returns PHIC_WORKSPACE_TOO_SMALL (with *entries set) when sched_cap pairs do not fit. */
phic_status phic_batch_plan_host(const phic_batch_item* items, int32_t count, const phic_select_opts* opts,
                                 const phic_batch_config* cfg, int32_t grid, int32_t* team, int32_t* sched_ptr,
                                 int32_t* sched, int64_t sched_cap, int64_t* entries, double* makespan_us);

/* Autotuner: plans and launches the batch with each candidate configuration (all on `stream`, with
 * CUDA events around `reps` launches after one warm-up launch), keeps the fastest by median time and
 * writes it to *best and its median milliseconds to *best_ms.  candidates NULL (or ncand <= 0) searches
 * rows_per_cta in {512, 1024, 2048, 4096, 8192, 16384} x blocks_per_sm in {2, 3}.  The batch's outputs
 * are written by every trial launch.  Synchronises `stream`. */
phic_status phic_batch_autotune(const phic_batch_item* items, int32_t count, const phic_select_opts* opts, void* ws,
                                size_t ws_bytes, const phic_batch_config* candidates, int32_t ncand, int32_t reps,
                                phic_stream_t stream, phic_batch_config* best, double* best_ms);

/* ---- Serving loop ----------------------------------------------------------------------------------
 * A request loop with continuous batching (an extension; the paper has no counterpart).  A worker thread
 * owned by the server admits submitted solves in arrival order while their device footprint (operator,
 * vectors, result, Algorithm 1's basis and Algorithm 3's workspace) fits in the arena, copies their
 * inputs to the device on a copy stream, and runs every loaded request together in slices: each slice
 * is one batched launch in which new requests run Algorithm 1, the series and up to max_steps recovery
 * steps, and requests already running continue their recovery by up to max_steps steps.  Requests that
 * arrive while a slice runs are admitted and loaded meanwhile and join the next slice; finished results
 * are copied back on the copy stream while the next slice runs, and their memory is released.
 * Operators and Taylor state stay on the device for a request's whole life.  A request's result does
 * not depend on the other requests or on how its work was sliced (see the batched launch above).
 * Thread-safe: submit / query / wait may be called from any host thread. */

typedef struct {
  void* arena;               /* device memory managed by the server (caller-owned, 256-byte aligned) */
  size_t arena_bytes;
  int32_t rows_per_cta;      /* team sizing of the slices (<= 0 selects 4096) */
  int32_t blocks_per_sm;     /* 2 or 3 (<= 0 selects 2) */
  int32_t max_steps;         /* recovery outer steps per request per slice (<= 0 selects 4) */
  int32_t max_active;        /* requests per slice (<= 0 selects 1024) */
  int32_t device;            /* CUDA device of the worker thread */
  int32_t m;                 /* Algorithm 1's degree (<= 0 selects 61); delta 0.8, seed 0x5EED, 200 evaluations */
  double slice_us;           /* time budget of a slice by the planner's cost model: requests already running
                                always join; new ones join in arrival order while the budget lasts (at least
                                one per slice).  The budget is scaled by the backlog (waiting requests / 16,
                                between 1 and 16).  <= 0 selects 20000 us */
} phic_server_config;

/* An operator registered with the server: uploaded once, Algorithm 1 run once, then shared by every
 * request that names it (the paper reuses (s, xi) across calls with the same A, Section 6).  HOST arrays,
 * read until the operator is ready. */
typedef struct {
  int64_t n, nnz;
  const int32_t* rowptr;
  const int32_t* colidx;
  const void* values;
  int32_t prec;
  int32_t pad;
} phic_operator;

/* One solve request; every array is in HOST memory and must stay valid (W unread) until the request is
 * reported done.  Page-locked memory lets the copies overlap with the kernels.  With op != 0 the request
 * uses that registered operator (n and prec must match; rowptr, colidx, values and nnz are ignored) and
 * its Algorithm 1 result, with s = s0 f* / (tol m!)^(1/m) for the request's tol; otherwise it brings its
 * own operator and Algorithm 1 runs in its first slice. */
typedef struct {
  int64_t n, nnz;
  const int32_t* rowptr;     /* n + 1 */
  const int32_t* colidx;     /* nnz */
  const void* values;        /* nnz of prec */
  const void* V;             /* (p+1) x n of prec, as in phic_solve (p x n with PHIC_NO_V0) */
  void* W;                   /* r x n of prec: the result, written before the request is reported done */
  int32_t prec, p, r;
  uint32_t flags;            /* PHIC_NO_V0 */
  double tol;                /* truncation tolerance (and Algorithm 1's) */
  int32_t max_terms;         /* as in phic_solve (<= 0 selects 610) */
  int32_t pad;
  int64_t op;                /* registered operator, or 0 */
  double t[PHIC_MAX_R];
  double alpha[PHIC_MAX_R];
} phic_request;

typedef enum {
  PHIC_REQ_QUEUED = 0,   /* waiting for device memory */
  PHIC_REQ_LOADING = 1,  /* inputs being copied in */
  PHIC_REQ_RUNNING = 2,  /* taking part in slices */
  PHIC_REQ_COPYING = 3,  /* result being copied out */
  PHIC_REQ_DONE = 4      /* W holds the result (or status reports the failure) */
} phic_request_state;

typedef struct {
  int32_t state;            /* phic_request_state */
  int32_t status;           /* phic_status of the request (valid when done) */
  int64_t submit_ns;        /* steady-clock times: submission, admission (memory granted), done */
  int64_t admit_ns;
  int64_t done_ns;
  int32_t slices;           /* slices the request took part in */
  int32_t pad;
  phic_params params;       /* Algorithm 1's output (valid when done) */
  phic_stats stats;         /* Algorithm 3's record (valid when done) */
} phic_request_info;

typedef struct {
  int64_t submitted, admitted, completed, failed;
  int64_t slices;           /* batched launches */
  int64_t max_slice_requests;
  int64_t arena_in_use, arena_peak;
  double gpu_busy_ms;       /* sum of the slices' device durations */
} phic_server_counters;

typedef struct phic_server phic_server;

/* Starts the worker thread.  The arena must outlive the server. */
phic_status phic_server_create(const phic_server_config* cfg, phic_server** out);

/* Queues a request (host arguments checked as in phic_solve); *id identifies it.  PHIC_WORKSPACE_TOO_SMALL:
 * the request can never fit in the arena. */
phic_status phic_server_submit(phic_server* srv, const phic_request* req, int64_t* id);

/* Registers an operator (copied in and run through Algorithm 1 as the server's memory allows); *op_id
 * names it in requests.  Requests may name it at once: they wait until it is ready. */
phic_status phic_server_add_operator(phic_server* srv, const phic_operator* op, int64_t* op_id);

/* Algorithm 1's result for a registered operator (status PHIC_OK once ready; *ready 0 before). */
phic_status phic_server_operator_params(phic_server* srv, int64_t op_id, int32_t* ready, phic_params* params);

/* Releases a registered operator once no admitted or queued request uses it. */
phic_status phic_server_remove_operator(phic_server* srv, int64_t op_id);

/* Current state of a request. */
phic_status phic_server_query(phic_server* srv, int64_t id, phic_request_info* info);

/* Waits until the request is done (timeout_ms < 0: no limit); PHIC_TIMEOUT when the limit passed first. */
phic_status phic_server_wait(phic_server* srv, int64_t id, double timeout_ms, phic_request_info* info);

phic_status phic_server_counters_get(phic_server* srv, phic_server_counters* out);

/* Stops the worker after the slice in flight, waits for the device, and releases the server (requests not
 * done are dropped: their W is not written). */
void phic_server_destroy(phic_server* srv);

/* Bound on one grid-barrier wait of phic_solve in milliseconds (default 2000).  Applies to later calls. */
void phic_set_spin_limit_ms(double ms);

/* Upper bound on resident blocks per SM of the persistent kernels (0 restores the default, 4).  Applies
 * to later calls; results do not depend on it. */
void phic_set_blocks_per_sm(int32_t blocks);

/* Test hook for the timeout path: with mode 1 the next phic_solve runs with block 0 of its series
 * kernel leaving before the first grid barrier (when the grid has more than one block), so that the
 * other blocks' bounded waits expire and the solve reports PHIC_TIMEOUT.  Consumed by that call. */
void phic_set_test_fault(int32_t mode);

/* FP64 throughput probe (a diagnostic; the paper has no counterpart).  Enqueues on `stream` one launch of
 * 4 blocks of 256 threads per SM in which every thread runs 8 independent chains of `iters` dependent FP64
 * fused multiply-adds, with no memory traffic; *fmas receives the launch's total count of FMAs
 * (grid x 256 x 8 x iters), so that FMAs / (CUDA-event duration) is the device's FP64 FMA rate, the roof of
 * the FP64-bound sparse products.  sink_dev: device, one double (written only in a case that never
 * occurs).  PHIC_INVALID_ARG for iters < 1 or a NULL pointer. */
phic_status phic_probe_fp64_fma(int32_t iters, double* sink_dev, int64_t* fmas, phic_stream_t stream);

/* Test hook of Algorithm 1 (Section 3): the coefficients of the objective
 * f(xi) = ||sum_k binom(m,k) z^(m-k) V_k||_2^(1/m), z = -xi/s0, exactly as phic_select_params forms them.
 * Writes 3 (m+1) doubles to out_dev (device) on `stream`: out[k] = binom(m,k) z^(m-k) as used, out[m+1+k]
 * = z^(m-k) (double-double square and multiply, rounded once) and out[2(m+1)+k] = binom(m,k) (128-bit
 * integers, rounded once), k = 0..m.  1 <= m <= 128; z finite. */
phic_status phic_test_objective_coeffs(int32_t m, double z, double* out_dev, phic_stream_t stream);

/* Text of a status code (static storage). */
const char* phic_status_string(int32_t status);

/* Number of kernels this library has launched in this process (all threads); for accounting. */
uint64_t phic_launch_count(void);

/* Library version as 10000*major + 100*minor + patch. */
int32_t phic_version(void);

/* Sizes in bytes of the public structs, so that a binding can check its layouts: out[i] for i < n (in
 * this order: phic_csr, phic_select_opts, phic_params, phic_stats, phic_lowrank, phic_batch_item,
 * phic_batch_config, phic_batch_info, phic_server_config, phic_operator, phic_request,
 * phic_request_info, phic_server_counters, phic_fn_op).  Returns how many there are (14), whatever n is;
 * out may be NULL when n is 0. */
int32_t phic_struct_sizes(size_t* out, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* PHICOMB_H */
