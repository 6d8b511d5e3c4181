// Host-side helpers shared by the C ABI translation units: argument checks, workspace layouts and the
// filling of the kernels' argument blocks.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "phicomb.h"

namespace phic {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

inline bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) % kAlign) == 0; }

inline bool csr_ok(const phic_csr* A) {
  if (!A) return false;
  if (A->n < 1 || A->n >= (int64_t)INT32_MAX || A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX) return false;
  if (!A->rowptr) return false;
  if (A->nnz > 0 && (!A->colidx || !A->values)) return false;
  if (A->prec != PHIC_F64 && A->prec != PHIC_F32) return false;
  return true;
}

struct SelectLayout {
  size_t ctl, part, basis, total;
};
inline SelectLayout select_layout(int64_t n, int m) {
  SelectLayout L;
  L.ctl = 0;
  L.part = align_up(sizeof(Ctl));
  L.basis = L.part + align_up(select_partials_bytes(n));
  L.total = L.basis + align_up((size_t)n * (size_t)((m + 2) / 2 * 2) * sizeof(double));  // pairs of vectors
  return L;
}

// Entries of the solve's copy of B: room for an ELL layout with up to a quarter of padding.
inline long long a1_capacity(long long nnz) { return (nnz > 0 ? nnz : 1) + nnz / 4 + 64; }

struct SolveLayout {
  size_t ctlS, ctlR, state, A1, rowflag, coef, Vt[2], Dt[2], S, Ft[2], E, total;
  long long a1_cap;
  TileLayout sl, fl;
};
// odd_cw: the series tile may take 3 or 5 columns a lane (pick_layout); the single-instance series is built
// for those widths, the batched and the low-rank ones for FP64 tiles only.
inline SolveLayout solve_layout(int64_t n, int64_t nnz, int p, int r, int prec, bool odd_cw = false) {
  SolveLayout L;
  const size_t es = prec == PHIC_F32 ? 4 : 8;
  L.sl = pick_layout((p + 1) * r, (int)es, odd_cw);
  L.fl = pick_layout(p == 0 ? r : 2 * r, (int)es);
  const size_t tileS = align_up((size_t)n * L.sl.ws * es);
  const size_t tileF = align_up((size_t)n * L.fl.ws * es);
  size_t off = 0;
  L.ctlS = off; off += align_up(sizeof(Ctl));
  L.ctlR = off; off += align_up(sizeof(Ctl));
  L.state = off; off += align_up(sizeof(SolveState));
  const size_t head = off;  // control blocks and state: zeroed before each solve
  L.a1_cap = a1_capacity(nnz);
  L.A1 = off; off += align_up((size_t)L.a1_cap * 2 * es);  // (column, value) entries, CSR or ELL order
  L.rowflag = off; off += align_up((size_t)n);
  L.coef = off; off += align_up((size_t)kCoefTab * PHIC_MAX_R * sizeof(CoefEntry<double>));
  for (int q = 0; q < 2; ++q) { L.Vt[q] = off; off += tileS; }
  for (int q = 0; q < 2; ++q) { L.Dt[q] = off; off += tileS; }
  L.S = off; off += tileS;
  for (int q = 0; q < 2; ++q) { L.Ft[q] = off; off += tileF; }
  L.E = off; off += tileF;
  L.total = off;
  (void)head;
  return L;
}

// Checks of the problem arguments that phic_solve and the batched calls share.
inline bool solve_args_ok(const phic_csr* A, int p, int r, const void* V, const double* t, const double* alpha,
                          double tol, uint32_t flags, uint32_t allowed_flags, int prec) {
  if (!csr_ok(A) || A->prec != prec || !V || !t || !alpha) return false;
  if (p < 0 || p > PHIC_MAX_P || r < 1 || r > PHIC_MAX_R || (p + 1) * r > PHIC_MAX_WIDTH) return false;
  if (!(tol > 0.0) || !std::isfinite(tol)) return false;
  if ((flags & ~allowed_flags) != 0 || ((flags & PHIC_NO_V0) && p == 0)) return false;
  for (int i = 0; i < r; ++i)
    if (!std::isfinite(t[i]) || !std::isfinite(alpha[i])) return false;
  return true;
}

// The solve kernels' arguments for one problem whose workspace starts at base with layout L.
inline void fill_solve_args(SolveArgs& a, const phic_csr* A, int p, int r, const void* V, const double* t,
                            const double* alpha, double tol, const phic_params* params_dev, uint32_t flags,
                            int max_terms, void* W, char* base, const SolveLayout& L, phic_stats* stats_dev,
                            unsigned long long spin_ns) {
  std::memset(&a, 0, sizeof(a));
  a.n = (int)A->n;
  a.nnz = (int)A->nnz;
  a.rowptr = A->rowptr;
  a.colidx = A->colidx;
  a.vals = A->values;
  a.A1 = base + L.A1;
  a.a1_cap = L.a1_cap;
  a.rowflag = reinterpret_cast<unsigned char*>(base + L.rowflag);
  a.Vin = V;
  a.W = W;
  a.p = p;
  a.r = r;
  a.no_v0 = (flags & PHIC_NO_V0) ? 1 : 0;
  a.S_lay = L.sl;
  a.F_lay = L.fl;
  for (int i = 0; i < r; ++i) {
    a.t[i] = t[i];
    a.alpha[i] = alpha[i];
  }
  a.tol = tol;
  a.max_terms = max_terms > 0 ? max_terms : 610;
  a.params = params_dev;
  for (int q = 0; q < 2; ++q) {
    a.Vt[q] = base + L.Vt[q];
    a.Dt[q] = base + L.Dt[q];
    a.Ft[q] = base + L.Ft[q];
  }
  a.S = base + L.S;
  a.E = base + L.E;
  a.ctlS = reinterpret_cast<Ctl*>(base + L.ctlS);
  a.ctlR = reinterpret_cast<Ctl*>(base + L.ctlR);
  a.state = reinterpret_cast<SolveState*>(base + L.state);
  a.coeftab = base + L.coef;
  a.stats = stats_dev;
  a.spin_ns = spin_ns;
  a.fault = 0;
}

// Algorithm 1's arguments for one problem whose workspace starts at base with layout L.
inline void fill_select_args(SelectArgs& a, const phic_csr* A, const phic_select_opts& o, const double* v, char* base,
                             const SelectLayout& L, phic_params* params_dev) {
  std::memset(&a, 0, sizeof(a));
  a.n = (int)A->n;
  a.nnz = (int)A->nnz;
  a.rowptr = A->rowptr;
  a.colidx = A->colidx;
  a.vals = A->values;
  a.vals_f32 = A->prec == PHIC_F32;
  a.v = v;
  a.seed = o.seed;
  a.m = o.m;
  a.tol = o.tol;
  a.delta = o.delta;
  a.max_evals = o.max_evals;
  a.Vb = reinterpret_cast<double*>(base + L.basis);
  a.part = base + L.part;
  a.ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  a.out = params_dev;
  a.spin_ns = (unsigned long long)(o.spin_limit_ms * 1e6);
}

inline bool select_opts_ok(const phic_select_opts& o) {
  return !(o.m < 1 || o.m > 128 || !(o.tol > 0.0) || !std::isfinite(o.tol) || !(o.delta > 0.0) || !(o.delta <= 1.0) ||
           o.max_evals < 1 || !(o.spin_limit_ms > 0.0));
}

}  // namespace phic
