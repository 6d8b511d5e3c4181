// Launch interfaces between the C ABI (capi.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "phicomb.h"

namespace phic {

struct Ctl;

// Row-group layout of a block tile: w columns stored with row stride ws; each row is handled by
// L lanes (CW columns each), grouped into Lp2 = next power of two >= L consecutive lanes.
struct TileLayout {
  int w, ws, cw, L, Lp2;
};
// odd_cw: tiles may also take 3 or 5 columns a lane where that leaves fewer idle lanes (only for series
// kernels built for those widths; see solve_layout).
TileLayout pick_layout(int w, int elem_bytes, bool odd_cw = false);

// Per-solve loop state in device memory.  The series writes the first block; the recovery reads it and,
// when it stops between outer steps (a bounded slice of a batched launch), records where to resume.
struct SolveState {
  int s_int;
  int series_terms;
  int eA;      // B = A_1 2^-eA has infinity norm below 1
  int nodiag;  // some row stores no diagonal entry (its shift is applied explicitly)
  double xi;
  double s;
  int status;     // outcome of the series (PHIC_OK: the recovery may run)
  int rec_init;   // 1 once the first block F has been formed
  int j_done;     // recovery outer steps completed
  int cur;        // Ft buffer that holds F
  double cF;      // ||F||_inf after the last refresh
  long long rec_terms;
  int max_inner;
  int done;       // 1 once the output has been written
  int ell;        // copy of B: ELL with this many slots per row, or 0 for CSR order
  int ndia;       // copy of B: DIA with these diagonals (ndia > 0; takes precedence over ell)
  int dia_off[16];
  // product of the undo factors applied so far, per combination: (pm_h + pm_l) 2^pe (see recover_body)
  double pm_h[PHIC_MAX_R];
  double pm_l[PHIC_MAX_R];
  int pe[PHIC_MAX_R];
  int coef_k;  // terms k = 1..coef_k of the recovery's coefficient table are filled
};

// The recovery's Taylor coefficients c_k = (t_i 2^eA / s)^k / k!, the same in every recovery step, filled
// for k <= kCoefTab the first time a step reaches k: the double-double value and its two neighbours in the
// tile type with the probability of rounding up (thr / 2^32), so that later steps round it without bias
// using integer operations only (see recover_body).
constexpr int kCoefTab = 128;
template <typename T>
struct CoefEntry {
  double ch, cl;  // c_k = ch + cl
  T base, alt;    // c_k's nearest value in T and its neighbour on the side of the remainder
  unsigned thr;   // alt is taken when a 32-bit uniform number is below thr
  float fcoef;    // c_k in FP32, for the norm of the term
};

// Entry of the solve's copy of A_1 = A - xi I, scaled by 2^-eA: column and value in one aligned load.
template <typename T>
struct alignas(2 * sizeof(T)) CsrEnt {
  int col;
  int pad_for_double;
  T v;
};
template <>
struct alignas(8) CsrEnt<float> {
  int col;
  float v;
};

struct SolveArgs {
  int n, nnz;
  const int* rowptr;
  const int* colidx;
  const void* vals;
  void* A1;               // CsrEnt<T>[a1_cap]: columns and values of B = (A - xi I) 2^-eA (CSR or ELL order)
  long long a1_cap;       // entries A1 can hold (ELL is used when n times the longest row fits)
  unsigned char* rowflag; // [n] 1 where the row stores no diagonal entry
  const void* Vin;
  void* W;
  int p, r, no_v0;
  TileLayout S_lay, F_lay;
  double t[PHIC_MAX_R];
  double alpha[PHIC_MAX_R];
  double tol;
  int max_terms;
  const phic_params* params;
  void* Vt[2];
  void* Dt[2];
  void* S;
  void* Ft[2];
  void* E;
  Ctl* ctlS;
  Ctl* ctlR;
  SolveState* state;
  void* coeftab;          // CoefEntry<T>[kCoefTab][PHIC_MAX_R]
  phic_stats* stats;
  unsigned long long spin_ns;
  int fault;
  // low-rank operator A = U W^T (lr_k > 0; the CSR fields are unused then)
  int lr_k;
  const void* lrU;
  const void* lrW;
  double* lr_part;  // [team size][k w] partial sums of W^T X
};

// Rows per chunk of Algorithm 1's sums of squares (each chunk's partial is one 16-byte record).
constexpr int kSelectChunk = 1024;
inline size_t select_partials_bytes(long long n) {
  return (size_t)2 * (size_t)((n + kSelectChunk - 1) / kSelectChunk) * 16;
}

struct SelectArgs {
  int n, nnz;
  const int* rowptr;
  const int* colidx;
  const void* vals;
  int vals_f32;
  const double* v;
  unsigned long long seed;
  int m;
  double tol, delta;
  int max_evals;
  double* Vb;    // basis V_0..V_m, pair-interleaved: V_k[row] at ((k/2) n + row) 2 + k%2
  void* part;    // 2 x ceil(n / kSelectChunk) scaled sums of squares
  Ctl* ctl;
  phic_params* out;
  unsigned long long spin_ns;
  int lr_k;           // low-rank operator A = U W^T (the CSR fields are unused then)
  const void* lrU;
  const void* lrW;
  double* lr_part;
};

// One instance of a batched launch: its solve and selection arguments (both pointing at the instance's
// control block for this launch) and the phases to run.
constexpr int kPhaseSelect = 1, kPhaseSeries = 2, kPhaseRecover = 4;
struct alignas(16) BatchInst {
  SolveArgs sa;
  SelectArgs sel;
  int phases;     // kPhase* bits
  int team;       // CTAs that run this instance together
  int prec;       // PHIC_F64 or PHIC_F32
  int max_steps;  // recovery outer steps in this launch (a slice); INT_MAX: to the end
};

// Schedule entry: the instance a CTA works on next and its rank in that instance's team.  Every CTA's
// entries follow one global order of the instances, so with all CTAs resident no team waits on a CTA
// that waits on it.
struct SchedEntry {
  int inst;
  int rank;
};

struct BatchArgs {
  const BatchInst* inst;
  const int* sched_ptr;     // [grid + 1]: entries of CTA b are sched[sched_ptr[b] .. sched_ptr[b+1])
  const SchedEntry* sched;
  unsigned long long spin_ns;
};

// Each returns a cudaError_t of the cooperative launch (or of the attribute queries).
cudaError_t launch_series(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out);
cudaError_t launch_recover(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out);
cudaError_t launch_select(const SelectArgs& a, cudaStream_t st, int* grid_out);
cudaError_t launch_params_set(phic_params* p, double xi, double s, cudaStream_t st);
// Low-rank operators: the same kernels' bodies with A applied as U (W^T x).
cudaError_t launch_lr_series(const SolveArgs& a, int prec, cudaStream_t st);
cudaError_t launch_lr_recover(const SolveArgs& a, int prec, cudaStream_t st);
cudaError_t launch_lr_select(const SelectArgs& a, cudaStream_t st);
int max_select_grid();
void count_launch();
int blocks_per_sm(int elem_bytes);
// Bound on one barrier wait (ns) set by phic_set_spin_limit_ms.
unsigned long long spin_limit_ns();
// Enqueues a one-block kernel that writes the number of unfinished solves of the batch to *out.
cudaError_t launch_batch_pending(const BatchInst* inst, int count, int* out, cudaStream_t st);
// Infinity norms of a batch's operators, for the planner's estimate of Algorithm 1's s: chunk c covers
// rows [r0, r0 + rows_per_chunk) of its item; out_bits[item] (zeroed by the caller) receives the bits of
// max_i sum_j |a_ij| (a nonnegative double, so its bits order like the value).  Rows whose bounds are
// not in [0, nnz] are skipped.  One block per chunk.
struct NormItem {
  const int* rowptr;
  const void* vals;
  long long nnz;
  int n, f32, rows_per_chunk, pad;
};
struct NormChunk {
  int item;
  int r0;
};
cudaError_t launch_batch_norms(const NormItem* items, const NormChunk* chunks, int nchunks,
                               unsigned long long* out_bits, cudaStream_t st);
// Enqueues a kernel that copies, for each instance of a slice, its done flag, phic_stats and
// phic_params into contiguous device arrays (for one small read-back).
cudaError_t launch_batch_collect(const BatchInst* inst, int count, int* done, phic_stats* stats, phic_params* params,
                                 cudaStream_t st);
// Batched launch with `grid` CTAs of the kernel built for `minb` (2 or 3) resident blocks per SM.
cudaError_t launch_batch(const BatchArgs& b, int grid, int minb, cudaStream_t st);
// Resident blocks per SM of the batched kernel built for minb (0 on error).
int batch_occupancy(int minb);

}  // namespace phic
