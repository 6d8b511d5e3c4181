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
TileLayout pick_layout(int w, int elem_bytes);

struct SolveState {
  int s_int;
  int series_terms;
  int eA;      // B = A_1 2^-eA has infinity norm below 1
  int nodiag;  // some row stores no diagonal entry (its shift is applied explicitly)
  double xi;
  double s;
  double pad2[4];
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
  void* A1;               // CsrEnt<T>[nnz]: columns and values of B = (A - xi I) 2^-eA
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
  phic_stats* stats;
  unsigned long long spin_ns;
  int fault;
};

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
  void* part;    // 2 x grid scaled sums of squares
  Ctl* ctl;
  phic_params* out;
  unsigned long long spin_ns;
};

// Each returns a cudaError_t of the cooperative launch (or of the attribute queries).
cudaError_t launch_series(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out);
cudaError_t launch_recover(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out);
cudaError_t launch_select(const SelectArgs& a, cudaStream_t st, int* grid_out);
cudaError_t launch_params_set(phic_params* p, double xi, double s, cudaStream_t st);
int max_select_grid();
void count_launch();
int blocks_per_sm(int elem_bytes);

}  // namespace phic
