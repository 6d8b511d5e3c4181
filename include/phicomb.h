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
 *   - Ownership: the caller owns every buffer, including the workspace.  The library allocates no
 *     memory, keeps no state between calls other than cached launch configurations, and never
 *     synchronises the stream.  All work is enqueued on `stream` (0 = legacy default stream).
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
} phic_stats;

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
 * prec = PHIC_F32 keeps A, V, the Taylor terms and W in FP32 with FP32 accumulation; the scalar
 * parameters (s, xi, mu, the nilpotent factors, the norms' comparison) stay FP64. */
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
 *     stencil fit up to about 70,000 rows).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current and caches it; make that first call before any stream capture.
 *   - Every call shares the one array, which keeps the previous call's contents (the call clears the
 *     parts that must start at zero).  Calls whose work overlaps on the GPU -- on different streams, or
 *     from different host threads -- race on the array and give undefined results: serialise them.
 *   - flags may be 0 or PHIC_NO_V0; A, V, t, alpha, params_dev, W, stats_dev, prec and stream are as in
 *     phic_solve. */
phic_status phic_solve_noalloc(const phic_csr* A, int32_t p, int32_t r, const void* V, const double* t,
                               const double* alpha, double tol, const phic_params* params_dev, uint32_t flags,
                               int32_t max_terms, void* W, phic_stats* stats_dev, int32_t prec, phic_stream_t stream);

/* Bound on one grid-barrier wait of phic_solve in milliseconds (default 2000).  Applies to later calls. */
void phic_set_spin_limit_ms(double ms);

/* Upper bound on resident blocks per SM of the persistent kernels (0 restores the default, 4).  Applies
 * to later calls; results do not depend on it. */
void phic_set_blocks_per_sm(int32_t blocks);

/* Test hook for the timeout path: with mode 1 the next phic_solve runs with block 0 of its series
 * kernel leaving before the first grid barrier (when the grid has more than one block), so that the
 * other blocks' bounded waits expire and the solve reports PHIC_TIMEOUT.  Consumed by that call. */
void phic_set_test_fault(int32_t mode);

/* Text of a status code (static storage). */
const char* phic_status_string(int32_t status);

/* Number of kernels this library has launched in this process (all threads); for accounting. */
uint64_t phic_launch_count(void);

/* Library version as 10000*major + 100*minor + patch. */
int32_t phic_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PHICOMB_H */
