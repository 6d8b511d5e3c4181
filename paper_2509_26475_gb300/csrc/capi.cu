// C ABI of the phicomb library: argument checks, workspace layout and kernel launches.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "layout.h"
#include "phicomb.h"

namespace phic {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<long long> g_spin_ns{2000000000LL};
std::atomic<int> g_blocks_per_sm{0};
std::atomic<int> g_fault{0};

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

unsigned long long spin_limit_ns() { return (unsigned long long)g_spin_ns.load(); }

int blocks_per_sm(int elem_bytes) {
  (void)elem_bytes;
  const int b = g_blocks_per_sm.load();
  return b > 0 ? b : 4;
}

}  // namespace phic

using namespace phic;

extern "C" {

void phic_select_opts_default(phic_select_opts* o) {
  if (!o) return;
  o->m = 61;
  o->tol = std::ldexp(1.0, -53);
  o->delta = 0.8;
  o->seed = 0x5EEDull;
  o->max_evals = 200;
  o->spin_limit_ms = 2000.0;
}

phic_status phic_select_workspace_size(int64_t n, int32_t m, size_t* bytes) {
  if (!bytes || n < 1 || n >= (int64_t)INT32_MAX || m < 1 || m > 128) return PHIC_INVALID_ARG;
  *bytes = select_layout(n, m).total;
  return PHIC_OK;
}

phic_status phic_select_params(const phic_csr* A, const phic_select_opts* opts, const double* v, void* ws,
                               size_t ws_bytes, phic_params* params_dev, phic_stream_t stream) {
  phic_select_opts o;
  if (opts) o = *opts; else phic_select_opts_default(&o);
  if (!csr_ok(A) || !params_dev || !ws || !aligned(ws)) return PHIC_INVALID_ARG;
  if (!select_opts_ok(o)) return PHIC_INVALID_ARG;
  const SelectLayout L = select_layout(A->n, o.m);
  if (ws_bytes < L.total) return PHIC_WORKSPACE_TOO_SMALL;
  char* base = static_cast<char*>(ws);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(base + L.ctl, 0, sizeof(Ctl), st) != cudaSuccess) return PHIC_CUDA_ERROR;
  SelectArgs a;
  fill_select_args(a, A, o, v, base, L, params_dev);
  return launch_select(a, st, nullptr) == cudaSuccess ? PHIC_OK : PHIC_CUDA_ERROR;
}

phic_status phic_params_set(phic_params* params_dev, double xi, double s, phic_stream_t stream) {
  if (!params_dev || !std::isfinite(xi) || !(s >= 0.0) || !std::isfinite(s)) return PHIC_INVALID_ARG;
  return launch_params_set(params_dev, xi, s, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PHIC_OK : PHIC_CUDA_ERROR;
}

phic_status phic_solve_workspace_size(int64_t n, int64_t nnz, int32_t p, int32_t r, int32_t prec, size_t* bytes) {
  if (!bytes || n < 1 || n >= (int64_t)INT32_MAX || nnz < 0 || nnz >= (int64_t)INT32_MAX || p < 0 ||
      p > PHIC_MAX_P || r < 1 || r > PHIC_MAX_R || (p + 1) * r > PHIC_MAX_WIDTH || (prec != PHIC_F64 && prec != PHIC_F32))
    return PHIC_INVALID_ARG;
  *bytes = solve_layout(n, nnz, p, r, prec, true).total;
  return PHIC_OK;
}

phic_status phic_tile_layout(int32_t w, int32_t prec, int32_t odd_cw, int32_t* out) {
  if (!out || w < 1 || w > PHIC_MAX_WIDTH || (prec != PHIC_F64 && prec != PHIC_F32)) return PHIC_INVALID_ARG;
  const TileLayout t = pick_layout(w, prec == PHIC_F32 ? 4 : 8, odd_cw != 0);
  out[0] = t.w;
  out[1] = t.ws;
  out[2] = t.cw;
  out[3] = t.L;
  out[4] = t.Lp2;
  return PHIC_OK;
}

phic_status phic_solve(const phic_csr* A, int32_t p, int32_t r, const void* V, const double* t, const double* alpha,
                       double tol, const phic_params* params_dev, uint32_t flags, int32_t max_terms, void* W, void* ws,
                       size_t ws_bytes, phic_stats* stats_dev, int32_t prec, phic_stream_t stream) {
  if (!solve_args_ok(A, p, r, V, t, alpha, tol, flags, PHIC_NO_V0 | PHIC_PHASE_SERIES | PHIC_PHASE_RECOVER, prec) ||
      !W || !params_dev || !ws || !aligned(ws))
    return PHIC_INVALID_ARG;
  bool run_series = true, run_recover = true;
  if (flags & (PHIC_PHASE_SERIES | PHIC_PHASE_RECOVER)) {
    run_series = (flags & PHIC_PHASE_SERIES) != 0;
    run_recover = (flags & PHIC_PHASE_RECOVER) != 0;
  }
  const SolveLayout L = solve_layout(A->n, A->nnz, p, r, prec, true);
  if (ws_bytes < L.total) return PHIC_WORKSPACE_TOO_SMALL;
  char* base = static_cast<char*>(ws);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (run_series && cudaMemsetAsync(base, 0, L.A1, st) != cudaSuccess) return PHIC_CUDA_ERROR;  // control + state
  SolveArgs a;
  fill_solve_args(a, A, p, r, V, t, alpha, tol, params_dev, flags, max_terms, W, base, L, stats_dev,
                  (unsigned long long)g_spin_ns.load());
  a.fault = g_fault.exchange(0);
  if (run_series && launch_series(a, prec, st, nullptr) != cudaSuccess) return PHIC_CUDA_ERROR;
  if (run_recover && launch_recover(a, prec, st, nullptr) != cudaSuccess) return PHIC_CUDA_ERROR;
  return PHIC_OK;
}

void phic_set_spin_limit_ms(double ms) {
  if (ms > 0.0 && std::isfinite(ms)) g_spin_ns.store((long long)(ms * 1e6));
}

void phic_set_blocks_per_sm(int32_t blocks) { g_blocks_per_sm.store(blocks > 0 ? blocks : 0); }

void phic_set_test_fault(int32_t mode) { g_fault.store(mode == 1 ? 1 : 0); }

const char* phic_status_string(int32_t s) {
  switch (s) {
    case PHIC_OK: return "ok";
    case PHIC_INVALID_ARG: return "invalid argument";
    case PHIC_NONFINITE: return "non-finite norm";
    case PHIC_TERM_CAP: return "Taylor term cap reached";
    case PHIC_TIMEOUT: return "grid barrier wait timed out";
    case PHIC_CUDA_ERROR: return "CUDA runtime error";
    case PHIC_WORKSPACE_TOO_SMALL: return "workspace too small";
    default: return "unknown status";
  }
}

uint64_t phic_launch_count(void) { return g_launches.load(); }

int32_t phic_version(void) { return 101; }

int32_t phic_struct_sizes(size_t* out, int32_t n) {
  const size_t sizes[] = {sizeof(phic_csr),           sizeof(phic_select_opts),  sizeof(phic_params),
                          sizeof(phic_stats),         sizeof(phic_lowrank),      sizeof(phic_batch_item),
                          sizeof(phic_batch_config),  sizeof(phic_batch_info),   sizeof(phic_server_config),
                          sizeof(phic_operator),      sizeof(phic_request),      sizeof(phic_request_info),
                          sizeof(phic_server_counters), sizeof(phic_fn_op)};
  const int32_t count = (int32_t)(sizeof(sizes) / sizeof(sizes[0]));
  for (int32_t i = 0; out && i < n && i < count; ++i) out[i] = sizes[i];
  return count;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------------
// phic_solve_noalloc: the solve kernels with their scratch in a static device array instead of a
// caller-supplied workspace, for callers that cannot allocate device memory.
// ---------------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[PHIC_NOALLOC_MAX_BYTES];

namespace {
constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per device.  In host code
// the array's name is only a host-side stand-in, so the kernels must be given this address.
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" phic_status phic_solve_noalloc(const phic_csr* A, int32_t p, int32_t r, const void* V, const double* t,
                                          const double* alpha, double tol, const phic_params* params_dev,
                                          uint32_t flags, int32_t max_terms, void* W, phic_stats* stats_dev,
                                          int32_t prec, phic_stream_t stream) {
  if (!solve_args_ok(A, p, r, V, t, alpha, tol, flags, PHIC_NO_V0, prec) || !W || !params_dev) return PHIC_INVALID_ARG;
  const SolveLayout L = solve_layout(A->n, A->nnz, p, r, prec, true);
  if (L.total > (size_t)PHIC_NOALLOC_MAX_BYTES) return PHIC_WORKSPACE_TOO_SMALL;
  void* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return PHIC_CUDA_ERROR;
  char* base = static_cast<char*>(scratch);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // control blocks and loop state must start at zero; the tiles are written before they are read
  if (cudaMemsetAsync(base, 0, L.A1, st) != cudaSuccess) return PHIC_CUDA_ERROR;
  SolveArgs a;
  fill_solve_args(a, A, p, r, V, t, alpha, tol, params_dev, flags, max_terms, W, base, L, stats_dev,
                  (unsigned long long)g_spin_ns.load());
  if (launch_series(a, prec, st, nullptr) != cudaSuccess) return PHIC_CUDA_ERROR;
  if (launch_recover(a, prec, st, nullptr) != cudaSuccess) return PHIC_CUDA_ERROR;
  return PHIC_OK;
}
