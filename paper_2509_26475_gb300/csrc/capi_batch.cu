// C ABI of the batched launch: argument checks, workspace layout, planning (batch_plan.h) and the
// autotuner over launch shapes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "batch_plan.h"
#include "kernels.h"
#include "layout.h"
#include "phicomb.h"

namespace phic {
namespace {

constexpr int kMaxBlocksPerSm = 3;
constexpr int kDefaultRowsPerCta = 4096;
constexpr int kMinRowsPerCta = 256;

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

struct ItemLayout {
  size_t sel_off, sel_basis, solve_off;
  SolveLayout sl;
  bool do_select, do_solve;
};

struct BatchLayout {
  size_t ctl, inst, sched_ptr, sched, items_begin, total;
  int gmax;
  size_t max_entries;
  std::vector<ItemLayout> item;
};

bool item_ok(const phic_batch_item& it) {
  const bool sel = (it.flags & PHIC_BATCH_SELECT) != 0;
  const bool solve = (it.flags & PHIC_BATCH_NO_SOLVE) == 0;
  if ((it.flags & ~(PHIC_NO_V0 | PHIC_BATCH_SELECT | PHIC_BATCH_NO_SOLVE)) != 0) return false;
  if (!sel && !solve) return false;
  if (!it.params || !csr_ok(&it.A)) return false;
  if (solve) {
    if (!solve_args_ok(&it.A, it.p, it.r, it.V, it.t, it.alpha, it.tol, it.flags & PHIC_NO_V0, PHIC_NO_V0,
                       it.A.prec) ||
        !it.W)
      return false;
  } else if (!(it.tol > 0.0) || !std::isfinite(it.tol)) {
    return false;
  }
  return std::isfinite(it.s_hint);
}

bool make_layout(const phic_batch_item* items, int count, const phic_select_opts& o, int sms, BatchLayout& L) {
  L.gmax = sms * kMaxBlocksPerSm;
  size_t off = 0;
  L.ctl = off; off += align_up((size_t)count * sizeof(Ctl));
  L.inst = off; off += align_up((size_t)count * sizeof(BatchInst));
  L.sched_ptr = off; off += align_up((size_t)(L.gmax + 1) * sizeof(int));
  L.max_entries = 0;
  for (int i = 0; i < count; ++i) {
    const long long teams = (items[i].A.n + kMinRowsPerCta - 1) / kMinRowsPerCta;
    L.max_entries += (size_t)std::min<long long>(teams, L.gmax);
  }
  L.sched = off; off += align_up(L.max_entries * sizeof(SchedEntry));
  L.items_begin = off;
  L.item.resize(count);
  for (int i = 0; i < count; ++i) {
    const phic_batch_item& it = items[i];
    ItemLayout& il = L.item[i];
    il.do_select = (it.flags & PHIC_BATCH_SELECT) != 0;
    il.do_solve = (it.flags & PHIC_BATCH_NO_SOLVE) == 0;
    il.sel_off = off;
    if (il.do_select) {
      const size_t part = align_up(select_partials_bytes(it.A.n));
      il.sel_basis = off + part;
      off = il.sel_basis + align_up((size_t)it.A.n * (size_t)((o.m + 2) / 2 * 2) * sizeof(double));
    }
    il.solve_off = off;
    if (il.do_solve) {
      il.sl = solve_layout(it.A.n, it.A.nnz, it.p, it.r, it.A.prec, it.A.prec == PHIC_F64);
      off += il.sl.total;
    }
  }
  L.total = off;
  return true;
}

}  // namespace
}  // namespace phic

// The handle: host copies of the instance table and schedule, and where they live in the workspace.
struct phic_batch {
  std::vector<phic::BatchInst> inst;
  phic::Schedule plan;
  char* ws;
  phic::BatchLayout L;
  int count, grid, minb, max_steps;
  bool first_loaded;  // the device table holds the first-launch phases (else the resume phases)
  std::vector<phic_batch_item> items;
  phic_select_opts opts;
};

namespace phic {
namespace {

void fill_instances(phic_batch& b, bool first_launch) {
  const int count = b.count;
  b.inst.resize(count);
  Ctl* ctl = reinterpret_cast<Ctl*>(b.ws + b.L.ctl);
  for (int i = 0; i < count; ++i) {
    const phic_batch_item& it = b.items[i];
    const ItemLayout& il = b.L.item[i];
    BatchInst& bi = b.inst[i];
    std::memset(&bi, 0, sizeof(bi));
    if (il.do_solve) {
      fill_solve_args(bi.sa, &it.A, it.p, it.r, it.V, it.t, it.alpha, it.tol, it.params, it.flags & PHIC_NO_V0,
                      it.max_terms, it.W, b.ws + il.solve_off, il.sl, it.stats, spin_limit_ns());
      bi.sa.ctlS = ctl + i;
      bi.sa.ctlR = ctl + i;
    } else {
      bi.sa.ctlS = ctl + i;
      bi.sa.ctlR = ctl + i;
    }
    if (il.do_select) {
      SelectLayout sl;
      sl.ctl = 0;
      sl.part = il.sel_off - il.sel_off;
      sl.basis = il.sel_basis - il.sel_off;
      sl.total = 0;
      phic_select_opts o = b.opts;
      o.tol = it.tol;
      fill_select_args(bi.sel, &it.A, o, it.v_select, b.ws + il.sel_off, sl, it.params);
      bi.sel.ctl = ctl + i;
    }
    bi.phases = 0;
    if (first_launch) {
      if (il.do_select) bi.phases |= kPhaseSelect;
      if (il.do_solve) bi.phases |= kPhaseSeries | kPhaseRecover;
    } else if (il.do_solve) {
      bi.phases = kPhaseRecover;
    }
    bi.team = b.plan.team[i];
    bi.prec = it.A.prec;
    bi.max_steps = b.max_steps > 0 ? b.max_steps : 0x7fffffff;
  }
}

phic_status upload(phic_batch& b, cudaStream_t st) {
  if (cudaMemcpyAsync(b.ws + b.L.inst, b.inst.data(), b.inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(b.ws + b.L.sched_ptr, b.plan.sched_ptr.data(), b.plan.sched_ptr.size() * sizeof(int),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PHIC_CUDA_ERROR;
  if (!b.plan.sched.empty() &&
      cudaMemcpyAsync(b.ws + b.L.sched, b.plan.sched.data(), b.plan.sched.size() * sizeof(SchedEntry),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PHIC_CUDA_ERROR;
  return cudaStreamSynchronize(st) == cudaSuccess ? PHIC_OK : PHIC_CUDA_ERROR;
}

// Items that run Algorithm 1 in the launch and carry no s_hint get one from ||A||_inf.  Algorithm 1
// returns s = s0 f* / (tol m!)^(1/m), and s0 f* is of the order of ||A - xi I|| ~ ||A||_inf / 2, so the
// hint ||A||_inf / (2 (tol m!)^(1/m)) orders the instances' costs for the planner (on the batching
// workload the selected s measured 1.31 to 1.36 times it).  The norms are taken on the device; the
// scratch lies in workspace regions that upload() and enqueue() rewrite afterwards (descriptors in the
// instance table, chunks in the schedule, results in the control blocks).  Returns without hints if the
// scratch does not fit.
phic_status fill_norm_hints(phic_batch& b, cudaStream_t st) {
  std::vector<NormItem> ni((size_t)b.count);
  std::vector<NormChunk> ch;
  bool any = false;
  for (int i = 0; i < b.count; ++i) {
    const phic_batch_item& it = b.items[(size_t)i];
    if (!(it.flags & PHIC_BATCH_SELECT) || (it.flags & PHIC_BATCH_NO_SOLVE) || it.s_hint > 0.0) continue;
    NormItem& x = ni[(size_t)i];
    x.rowptr = it.A.rowptr;
    x.vals = it.A.values;
    x.nnz = it.A.nnz;
    x.n = (int)it.A.n;
    x.f32 = it.A.prec == PHIC_F32;
    x.rows_per_chunk = (int)std::max<long long>(4096, (it.A.n + b.L.gmax - 1) / b.L.gmax);
    for (long long r = 0; r < it.A.n; r += x.rows_per_chunk) ch.push_back(NormChunk{i, (int)r});
    any = true;
  }
  if (!any) return PHIC_OK;
  if (ni.size() * sizeof(NormItem) > (size_t)b.count * sizeof(BatchInst) ||
      ch.size() * sizeof(NormChunk) > b.L.max_entries * sizeof(SchedEntry) ||
      (size_t)b.count * sizeof(unsigned long long) > (size_t)b.count * sizeof(Ctl))
    return PHIC_OK;
  NormItem* d_items = reinterpret_cast<NormItem*>(b.ws + b.L.inst);
  NormChunk* d_chunks = reinterpret_cast<NormChunk*>(b.ws + b.L.sched);
  unsigned long long* d_out = reinterpret_cast<unsigned long long*>(b.ws + b.L.ctl);
  std::vector<unsigned long long> bits((size_t)b.count, 0ull);
  if (cudaMemcpyAsync(d_items, ni.data(), ni.size() * sizeof(NormItem), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_chunks, ch.data(), ch.size() * sizeof(NormChunk), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(d_out, 0, bits.size() * sizeof(unsigned long long), st) != cudaSuccess ||
      launch_batch_norms(d_items, d_chunks, (int)ch.size(), d_out, st) != cudaSuccess ||
      cudaMemcpyAsync(bits.data(), d_out, bits.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PHIC_CUDA_ERROR;
  const int m = b.opts.m;
  for (int i = 0; i < b.count; ++i) {
    phic_batch_item& it = b.items[(size_t)i];
    if (!ni[(size_t)i].rowptr) continue;
    double nrm;
    std::memcpy(&nrm, &bits[(size_t)i], sizeof(double));
    const double theta = std::exp((std::log(it.tol) + std::lgamma(m + 1.0)) / m);
    const double h = nrm / (2.0 * theta);
    if (std::isfinite(h) && h > 0.0) it.s_hint = h;
  }
  return PHIC_OK;
}

phic_status enqueue(phic_batch& b, cudaStream_t st) {
  if (cudaMemsetAsync(b.ws + b.L.ctl, 0, (size_t)b.count * sizeof(Ctl), st) != cudaSuccess) return PHIC_CUDA_ERROR;
  BatchArgs a;
  a.inst = reinterpret_cast<const BatchInst*>(b.ws + b.L.inst);
  a.sched_ptr = reinterpret_cast<const int*>(b.ws + b.L.sched_ptr);
  a.sched = reinterpret_cast<const SchedEntry*>(b.ws + b.L.sched);
  a.spin_ns = spin_limit_ns();
  return launch_batch(a, b.grid, b.minb, st) == cudaSuccess ? PHIC_OK : PHIC_CUDA_ERROR;
}

phic_status check_items(const phic_batch_item* items, int32_t count, const phic_select_opts* opts,
                        phic_select_opts& o) {
  if (!items || count < 1) return PHIC_INVALID_ARG;
  if (opts) o = *opts; else phic_select_opts_default(&o);
  if (!select_opts_ok(o)) return PHIC_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!item_ok(items[i])) return PHIC_INVALID_ARG;
  return PHIC_OK;
}

}  // namespace
}  // namespace phic

using namespace phic;

extern "C" {

phic_status phic_batch_workspace_size(const phic_batch_item* items, int32_t count, const phic_select_opts* opts,
                                      size_t* bytes) {
  phic_select_opts o;
  if (!bytes) return PHIC_INVALID_ARG;
  const phic_status s = check_items(items, count, opts, o);
  if (s != PHIC_OK) return s;
  const int sms = device_sms();
  if (sms < 1) return PHIC_CUDA_ERROR;
  BatchLayout L;
  make_layout(items, count, o, sms, L);
  *bytes = L.total;
  return PHIC_OK;
}

phic_status phic_batch_create(const phic_batch_item* items, int32_t count, const phic_select_opts* opts,
                              const phic_batch_config* cfg, void* ws, size_t ws_bytes, phic_stream_t stream,
                              phic_batch** out) {
  if (!out || !ws || !aligned(ws)) return PHIC_INVALID_ARG;
  *out = nullptr;
  phic_select_opts o;
  phic_status s = check_items(items, count, opts, o);
  if (s != PHIC_OK) return s;
  phic_batch_config c{};
  if (cfg) c = *cfg;
  if (c.rows_per_cta <= 0) c.rows_per_cta = kDefaultRowsPerCta;
  if (c.rows_per_cta < kMinRowsPerCta) return PHIC_INVALID_ARG;
  if (c.blocks_per_sm <= 0) c.blocks_per_sm = 2;
  if (c.blocks_per_sm > kMaxBlocksPerSm) return PHIC_INVALID_ARG;
  const int sms = device_sms();
  if (sms < 1) return PHIC_CUDA_ERROR;
  phic_batch* b = new (std::nothrow) phic_batch();
  if (!b) return PHIC_CUDA_ERROR;
  b->items.assign(items, items + count);
  b->opts = o;
  b->count = count;
  b->ws = static_cast<char*>(ws);
  make_layout(items, count, o, sms, b->L);
  if (ws_bytes < b->L.total) {
    delete b;
    return PHIC_WORKSPACE_TOO_SMALL;
  }
  b->minb = c.blocks_per_sm >= 3 ? 3 : 2;
  const int occ = batch_occupancy(b->minb);
  if (occ < 1) {
    delete b;
    return PHIC_CUDA_ERROR;
  }
  b->grid = sms * std::min(c.blocks_per_sm, occ);
  b->max_steps = c.max_steps;
  s = fill_norm_hints(*b, reinterpret_cast<cudaStream_t>(stream));
  if (s != PHIC_OK) {
    delete b;
    return s;
  }
  plan_core(b->items.data(), count, o, b->grid, c.rows_per_cta, true, b->plan);
  fill_instances(*b, true);
  b->first_loaded = true;
  s = upload(*b, reinterpret_cast<cudaStream_t>(stream));
  if (s != PHIC_OK) {
    delete b;
    return s;
  }
  *out = b;
  return PHIC_OK;
}

phic_status phic_batch_launch(phic_batch* b, phic_stream_t stream) {
  if (!b) return PHIC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!b->first_loaded) {  // a resume table is loaded: restore the first-launch table
    fill_instances(*b, true);
    b->first_loaded = true;
    if (cudaMemcpyAsync(b->ws + b->L.inst, b->inst.data(), b->inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return PHIC_CUDA_ERROR;
  }
  return enqueue(*b, st);
}

phic_status phic_batch_resume(phic_batch* b, phic_stream_t stream) {
  if (!b) return PHIC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (b->first_loaded) {
    fill_instances(*b, false);
    b->first_loaded = false;
    if (cudaMemcpyAsync(b->ws + b->L.inst, b->inst.data(), b->inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return PHIC_CUDA_ERROR;
  }
  return enqueue(*b, st);
}

phic_status phic_batch_pending(const phic_batch* b, int32_t* pending_dev, phic_stream_t stream) {
  if (!b || !pending_dev) return PHIC_INVALID_ARG;
  return launch_batch_pending(reinterpret_cast<const BatchInst*>(b->ws + b->L.inst), b->count, pending_dev,
                              reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PHIC_OK : PHIC_CUDA_ERROR;
}

phic_status phic_batch_info_get(const phic_batch* b, phic_batch_info* info) {
  if (!b || !info) return PHIC_INVALID_ARG;
  info->grid = b->grid;
  info->blocks_per_sm = b->grid / std::max(1, device_sms());
  info->count = b->count;
  info->max_team = b->plan.team.empty() ? 0 : *std::max_element(b->plan.team.begin(), b->plan.team.end());
  info->entries = (int64_t)b->plan.sched.size();
  info->est_makespan_us = b->plan.makespan;
  info->est_busy_frac = b->plan.busy;
  return PHIC_OK;
}

void phic_batch_destroy(phic_batch* b) { delete b; }

phic_status phic_batch_plan_host(const phic_batch_item* items, int32_t count, const phic_select_opts* opts,
                                 const phic_batch_config* cfg, int32_t grid, int32_t* team, int32_t* sched_ptr,
                                 int32_t* sched, int64_t sched_cap, int64_t* entries, double* makespan_us) {
  phic_select_opts o;
  phic_status s = check_items(items, count, opts, o);
  if (s != PHIC_OK) return s;
  if (grid < 1 || !team || !sched_ptr || !sched || !entries) return PHIC_INVALID_ARG;
  const int rows = cfg && cfg->rows_per_cta > 0 ? cfg->rows_per_cta : kDefaultRowsPerCta;
  if (rows < kMinRowsPerCta) return PHIC_INVALID_ARG;
  Schedule plan;
  plan_core(items, count, o, grid, rows, true, plan);
  *entries = (int64_t)plan.sched.size();
  if (makespan_us) *makespan_us = plan.makespan;
  if ((int64_t)plan.sched.size() > sched_cap) return PHIC_WORKSPACE_TOO_SMALL;
  for (int i = 0; i < count; ++i) team[i] = plan.team[i];
  for (int g = 0; g <= grid; ++g) sched_ptr[g] = plan.sched_ptr[g];
  for (size_t e = 0; e < plan.sched.size(); ++e) {
    sched[2 * e] = plan.sched[e].inst;
    sched[2 * e + 1] = plan.sched[e].rank;
  }
  return PHIC_OK;
}

phic_status phic_batch_autotune(const phic_batch_item* items, int32_t count, const phic_select_opts* opts, void* ws,
                                size_t ws_bytes, const phic_batch_config* candidates, int32_t ncand, int32_t reps,
                                phic_stream_t stream, phic_batch_config* best, double* best_ms) {
  if (!best || reps < 1) return PHIC_INVALID_ARG;
  std::vector<phic_batch_config> cands;
  if (candidates && ncand > 0) {
    cands.assign(candidates, candidates + ncand);
  } else {
    for (int bps : {2, 3})
      for (int rows : {512, 1024, 2048, 4096, 8192, 16384}) cands.push_back(phic_batch_config{rows, bps, 0, 0});
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PHIC_CUDA_ERROR;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PHIC_CUDA_ERROR;
  }
  double best_t = INFINITY;
  phic_status result = PHIC_OK;
  for (const phic_batch_config& c : cands) {
    phic_batch* b = nullptr;
    phic_status s = phic_batch_create(items, count, opts, &c, ws, ws_bytes, stream, &b);
    if (s != PHIC_OK) {
      result = s;
      break;
    }
    std::vector<double> t;
    s = phic_batch_launch(b, stream);  // warm-up
    for (int q = 0; q < reps && s == PHIC_OK; ++q) {
      if (cudaEventRecord(e0, st) != cudaSuccess) s = PHIC_CUDA_ERROR;
      if (s == PHIC_OK) s = phic_batch_launch(b, stream);
      if (s == PHIC_OK && cudaEventRecord(e1, st) != cudaSuccess) s = PHIC_CUDA_ERROR;
      float ms = 0.f;
      if (s == PHIC_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        s = PHIC_CUDA_ERROR;
      t.push_back(ms);
    }
    phic_batch_destroy(b);
    if (s != PHIC_OK) {
      result = s;
      break;
    }
    std::sort(t.begin(), t.end());
    const double med = t[t.size() / 2];
    if (med < best_t) {
      best_t = med;
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result == PHIC_OK && best_ms) *best_ms = best_t;
  return result;
}

}  // extern "C"
