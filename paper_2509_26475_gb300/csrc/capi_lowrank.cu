// C ABI for matrix-free low-rank operators A = U W^T (phic_lowrank_*): argument checks, workspace
// layouts (the CSR solve's layout without an operator copy, plus the per-CTA partial sums of W^T X) and
// the launches.
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "layout.h"
#include "lowrank.cuh"
#include "phicomb.h"

namespace phic {
namespace {

size_t lr_part_bytes(int k, int w) { return align_up((size_t)kLowRankMaxGrid * (size_t)k * (size_t)w * sizeof(double)); }

bool lowrank_ok(const phic_lowrank* A) {
  return A && A->n >= 1 && A->n < (int64_t)INT32_MAX && A->k >= 1 && A->k <= PHIC_MAX_RANK && A->U && A->W &&
         (A->prec == PHIC_F64 || A->prec == PHIC_F32);
}

// a phic_csr stand-in carrying n and the precision (no arrays: the low-rank bodies do not read them)
phic_csr csr_shape(const phic_lowrank* A) {
  phic_csr c;
  std::memset(&c, 0, sizeof(c));
  c.n = A->n;
  c.prec = A->prec;
  return c;
}

}  // namespace
}  // namespace phic

using namespace phic;

extern "C" {

phic_status phic_lowrank_select_workspace_size(int64_t n, int32_t k, int32_t m, size_t* bytes) {
  if (!bytes || n < 1 || n >= (int64_t)INT32_MAX || k < 1 || k > PHIC_MAX_RANK || m < 1 || m > 128)
    return PHIC_INVALID_ARG;
  *bytes = select_layout(n, m).total + lr_part_bytes(k, 1);
  return PHIC_OK;
}

phic_status phic_lowrank_select_params(const phic_lowrank* A, const phic_select_opts* opts, const double* v, void* ws,
                                       size_t ws_bytes, phic_params* params_dev, phic_stream_t stream) {
  phic_select_opts o;
  if (opts) o = *opts; else phic_select_opts_default(&o);
  if (!lowrank_ok(A) || !params_dev || !ws || !aligned(ws) || !select_opts_ok(o)) return PHIC_INVALID_ARG;
  const SelectLayout L = select_layout(A->n, o.m);
  if (ws_bytes < L.total + lr_part_bytes(A->k, 1)) return PHIC_WORKSPACE_TOO_SMALL;
  char* base = static_cast<char*>(ws);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(base + L.ctl, 0, sizeof(Ctl), st) != cudaSuccess) return PHIC_CUDA_ERROR;
  const phic_csr c = csr_shape(A);
  SelectArgs a;
  fill_select_args(a, &c, o, v, base, L, params_dev);
  a.lr_k = A->k;
  a.lrU = A->U;
  a.lrW = A->W;
  a.lr_part = reinterpret_cast<double*>(base + L.total);
  return launch_lr_select(a, st) == cudaSuccess ? PHIC_OK : PHIC_CUDA_ERROR;
}

phic_status phic_lowrank_solve_workspace_size(int64_t n, int32_t k, int32_t p, int32_t r, int32_t prec, size_t* bytes) {
  if (!bytes || n < 1 || n >= (int64_t)INT32_MAX || k < 1 || k > PHIC_MAX_RANK || p < 0 || p > PHIC_MAX_P || r < 1 ||
      r > PHIC_MAX_R || (p + 1) * r * k > kLowRankMaxE || (prec != PHIC_F64 && prec != PHIC_F32))
    return PHIC_INVALID_ARG;
  *bytes = solve_layout(n, 0, p, r, prec, prec == PHIC_F64).total + lr_part_bytes(k, (p + 1) * r);
  return PHIC_OK;
}

phic_status phic_lowrank_solve(const phic_lowrank* A, int32_t p, int32_t r, const void* V, const double* t,
                               const double* alpha, double tol, const phic_params* params_dev, uint32_t flags,
                               int32_t max_terms, void* W, void* ws, size_t ws_bytes, phic_stats* stats_dev,
                               int32_t prec, phic_stream_t stream) {
  if (!lowrank_ok(A) || A->prec != prec) return PHIC_INVALID_ARG;
  const phic_csr c = csr_shape(A);
  phic_csr c_chk = c;
  c_chk.rowptr = reinterpret_cast<const int32_t*>(A->U);  // non-null stand-in for the shared checks
  if (!solve_args_ok(&c_chk, p, r, V, t, alpha, tol, flags, PHIC_NO_V0, prec) || !W || !params_dev || !ws ||
      !aligned(ws) || (p + 1) * r * A->k > kLowRankMaxE)
    return PHIC_INVALID_ARG;
  const SolveLayout L = solve_layout(A->n, 0, p, r, prec, prec == PHIC_F64);
  if (ws_bytes < L.total + lr_part_bytes(A->k, (p + 1) * r)) return PHIC_WORKSPACE_TOO_SMALL;
  char* base = static_cast<char*>(ws);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(base, 0, L.A1, st) != cudaSuccess) return PHIC_CUDA_ERROR;  // control blocks + state
  SolveArgs a;
  fill_solve_args(a, &c, p, r, V, t, alpha, tol, params_dev, flags, max_terms, W, base, L, stats_dev, spin_limit_ns());
  a.lr_k = A->k;
  a.lrU = A->U;
  a.lrW = A->W;
  a.lr_part = reinterpret_cast<double*>(base + L.total);
  if (launch_lr_series(a, prec, st) != cudaSuccess) return PHIC_CUDA_ERROR;
  if (launch_lr_recover(a, prec, st) != cudaSuccess) return PHIC_CUDA_ERROR;
  return PHIC_OK;
}

}  // extern "C"
