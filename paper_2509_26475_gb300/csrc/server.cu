// Serving loop with continuous batching (phic_server_*).
//
// One worker thread per server drives two streams: a copy stream for the requests' inputs and results and
// a compute stream for the slices.  The device arena is split into a fixed head (control blocks, the
// slice's instance table and schedule, the collected done flags / records) and a pool from which each
// job takes blocks, first-fit.  A solve request takes its resident state (its operator unless it names a
// registered one, V, W, parameters, record and the solve workspace) and, when it brings its own operator,
// Algorithm 1's basis, returned after its first slice.  A registered operator takes its CSR arrays and
// parameters for its lifetime and Algorithm 1's basis until its selection slice is over.
//
// Worker loop: retire results whose copy-out finished (releasing their memory); admit queued requests in
// arrival order while their blocks fit (copy-in enqueued at once); move requests whose copy-in finished
// to the running set; when no slice is in flight, plan one over the running set (batch_plan.h), upload
// its tables, launch it, and collect each instance's done flag and records into page-locked memory.
// While a slice runs the worker keeps admitting and loading, so arrivals overlap with the device work
// and join the next slice.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_plan.h"
#include "common.cuh"
#include "kernels.h"
#include "layout.h"
#include "phicomb.h"

namespace phic {
namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator of byte ranges (multiples of 256) with coalescing of neighbours on release.
class ArenaAlloc {
 public:
  void init(size_t total) {
    free_.clear();
    if (total) free_[0] = total;
    in_use_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, next = it->first + bytes;
      free_.erase(it);
      if (rest) free_[next] = rest;
      in_use_ += bytes;
      peak_ = std::max(peak_, in_use_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    in_use_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t in_use() const { return in_use_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t in_use_ = 0, peak_ = 0;
};

struct Req {
  int64_t id = 0;
  bool is_op = false;      // a registered operator (Algorithm 1 only) rather than a solve
  Req* op = nullptr;       // solves: the registered operator used, if any
  int op_refs = 0;         // operators: requests admitted or queued that use it
  bool op_removed = false;
  bool op_ready = false;   // operators: Algorithm 1 done (params valid)
  phic_params params_in{}; // solves on a registered operator: (xi, s) uploaded at admission
  phic_request r{};
  int state = PHIC_REQ_QUEUED;
  int status = PHIC_OK;
  int64_t t_submit = 0, t_admit = 0, t_done = 0;
  int slices = 0;
  bool selected = false;
  size_t es = 8;
  // blocks in the pool
  size_t off_main = 0, bytes_main = 0, off_sel = 0, bytes_sel = 0;
  bool have_sel = false;
  char* base = nullptr;
  char* sel_base = nullptr;
  size_t o_rowptr = 0, o_colidx = 0, o_values = 0, o_V = 0, o_W = 0, o_params = 0, o_stats = 0, o_solve = 0;
  SolveLayout sl{};
  SelectLayout sel{};
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  phic_params params{};
  phic_stats stats{};
  double s_hint = 0.0;

  int vrows() const { return r.p + 1 - ((r.flags & PHIC_NO_V0) ? 1 : 0); }
  bool own_csr() const { return is_op || op == nullptr; }
};

void plan_blocks(Req& q, int m) {
  const int64_t n = q.r.n, nnz = q.op ? q.op->r.nnz : q.r.nnz;
  q.es = q.r.prec == PHIC_F32 ? 4 : 8;
  size_t off = 0;
  if (q.own_csr()) {
    q.o_rowptr = off; off += align_up((size_t)(n + 1) * 4);
    q.o_colidx = off; off += align_up((size_t)std::max<int64_t>(nnz, 1) * 4);
    q.o_values = off; off += align_up((size_t)std::max<int64_t>(nnz, 1) * q.es);
  }
  q.o_params = off; off += align_up(sizeof(phic_params));
  if (!q.is_op) {
    q.o_V = off; off += align_up((size_t)q.vrows() * n * q.es);
    q.o_W = off; off += align_up((size_t)q.r.r * n * q.es);
    q.o_stats = off; off += align_up(sizeof(phic_stats));
    q.sl = solve_layout(n, nnz, q.r.p, q.r.r, q.r.prec, q.r.prec == PHIC_F64);
    q.o_solve = off; off += q.sl.total;
  }
  q.bytes_main = off;
  q.bytes_sel = 0;
  if (q.own_csr()) {
    q.sel.ctl = 0;
    q.sel.part = 0;
    q.sel.basis = align_up(select_partials_bytes(n));
    q.sel.total = q.sel.basis + align_up((size_t)n * (size_t)((m + 2) / 2 * 2) * sizeof(double));
    q.bytes_sel = q.sel.total;
  }
}

// s for tolerance tol from a selection's s0 and f(xi*): s = s0 f* / (tol m!)^(1/m).
double s_for_tol(const phic_params& p, double tol, int m) {
  if (!(p.s0 > 0.0) || !(p.f_star > 0.0)) return p.s;
  return p.s0 * p.f_star / std::exp((std::log(tol) + std::lgamma(m + 1.0)) / (double)m);
}

bool request_ok(const phic_request& r) {
  if (r.n < 1 || r.n >= (int64_t)INT32_MAX) return false;
  if (r.op == 0 && (r.nnz < 0 || r.nnz >= (int64_t)INT32_MAX || !r.rowptr || (r.nnz > 0 && (!r.colidx || !r.values))))
    return false;
  if (!r.V || !r.W) return false;
  if (r.prec != PHIC_F64 && r.prec != PHIC_F32) return false;
  if (r.p < 0 || r.p > PHIC_MAX_P || r.r < 1 || r.r > PHIC_MAX_R || (r.p + 1) * r.r > PHIC_MAX_WIDTH) return false;
  if ((r.flags & ~PHIC_NO_V0) != 0 || ((r.flags & PHIC_NO_V0) && r.p == 0)) return false;
  if (!(r.tol > 0.0) || !std::isfinite(r.tol)) return false;
  for (int i = 0; i < r.r; ++i)
    if (!std::isfinite(r.t[i]) || !std::isfinite(r.alpha[i])) return false;
  return true;
}

}  // namespace
}  // namespace phic

struct phic_server {
  phic_server_config cfg{};
  phic_select_opts sel_opts{};
  int sms = 0, grid = 0, minb = 2, gmax = 0;
  char* arena = nullptr;
  // head of the arena
  size_t h_ctl = 0, h_inst = 0, h_ptr = 0, h_sched = 0, h_done = 0, h_stats = 0, h_params = 0, head = 0;
  size_t sched_cap = 0;
  phic::ArenaAlloc pool;
  // page-locked staging
  phic::BatchInst* st_inst = nullptr;
  int* st_ptr = nullptr;
  phic::SchedEntry* st_sched = nullptr;
  int* hb_done = nullptr;
  phic_stats* hb_stats = nullptr;
  phic_params* hb_params = nullptr;
  cudaStream_t s_compute = nullptr, s_copy = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int64_t next_id = 1;
  std::deque<phic::Req*> incoming;
  std::unordered_map<int64_t, phic::Req*> all;
  std::vector<phic::Req*> ops;  // registered operators not yet freed
  phic_server_counters ctr{};
  // worker-private
  std::deque<phic::Req*> queued;
  std::vector<phic::Req*> loading, running, copying, slice;
  bool inflight = false;
  cudaError_t launch_err = cudaSuccess;
};

namespace phic {
namespace {

void set_state(phic_server& S, Req* q, int st) {
  std::lock_guard<std::mutex> lk(S.mu);
  q->state = st;
}

void finish_req(phic_server& S, Req* q, int status) {
  {
    std::lock_guard<std::mutex> lk(S.mu);
    q->status = status;
    q->t_done = now_ns();
    q->state = PHIC_REQ_DONE;
    S.ctr.completed += 1;
    if (status != PHIC_OK) S.ctr.failed += 1;
  }
  S.cv_done.notify_all();
}

void release_blocks(phic_server& S, Req* q) {
  if (q->have_sel) {
    S.pool.release(q->off_sel, q->bytes_sel);
    q->have_sel = false;
  }
  if (q->base) {
    S.pool.release(q->off_main, q->bytes_main);
    q->base = nullptr;
  }
}

// A solve that used a registered operator lets go of it; a removed operator with no users is freed.
void drop_op_ref(phic_server& S, Req* q) {
  if (!q->op) return;
  std::lock_guard<std::mutex> lk(S.mu);
  q->op->op_refs -= 1;
}

void collect_removed_ops(phic_server& S) {
  std::vector<Req*> dead;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    for (size_t k = 0; k < S.ops.size();) {
      Req* o = S.ops[k];
      if (o->op_removed && o->op_refs == 0 && o->state == PHIC_REQ_DONE && o->base) {
        dead.push_back(o);
        S.ops.erase(S.ops.begin() + k);
      } else {
        ++k;
      }
    }
  }
  for (Req* o : dead) release_blocks(S, o);
}

void retire_copies(phic_server& S) {
  for (size_t k = 0; k < S.copying.size();) {
    Req* q = S.copying[k];
    const cudaError_t e = cudaEventQuery(q->ev_out);
    if (e == cudaErrorNotReady) {
      ++k;
      continue;
    }
    release_blocks(S, q);
    drop_op_ref(S, q);
    finish_req(S, q, e == cudaSuccess ? q->status : PHIC_CUDA_ERROR);
    S.copying.erase(S.copying.begin() + k);
  }
}

// Admits queued jobs in arrival order while their blocks fit; a solve waiting for its registered operator
// to finish Algorithm 1 is passed over (jobs behind it may go first).
void admit(phic_server& S) {
  for (auto itq = S.queued.begin(); itq != S.queued.end();) {
    Req* q = *itq;
    if (q->op && !q->op->op_ready) {
      if (q->op->state == PHIC_REQ_DONE) {  // the operator failed
        itq = S.queued.erase(itq);
        drop_op_ref(S, q);
        finish_req(S, q, q->op->status != PHIC_OK ? q->op->status : PHIC_INVALID_ARG);
        continue;
      }
      ++itq;
      continue;
    }
    size_t a = 0, b = 0;
    if (!S.pool.alloc(q->bytes_main, &a)) break;
    if (q->bytes_sel && !S.pool.alloc(q->bytes_sel, &b)) {
      S.pool.release(a, q->bytes_main);
      break;
    }
    q->off_main = a;
    q->base = S.arena + S.head + a;
    if (q->bytes_sel) {
      q->off_sel = b;
      q->have_sel = true;
      q->sel_base = S.arena + S.head + b;
    }
    if (!q->ev_in) cudaEventCreateWithFlags(&q->ev_in, cudaEventDisableTiming);
    if (!q->ev_out) cudaEventCreateWithFlags(&q->ev_out, cudaEventDisableTiming);
    const phic_request& r = q->r;
    bool ok = true;
    if (q->own_csr()) {
      ok = ok && cudaMemcpyAsync(q->base + q->o_rowptr, r.rowptr, (size_t)(r.n + 1) * 4, cudaMemcpyHostToDevice,
                                 S.s_copy) == cudaSuccess;
      if (r.nnz > 0) {
        ok = ok && cudaMemcpyAsync(q->base + q->o_colidx, r.colidx, (size_t)r.nnz * 4, cudaMemcpyHostToDevice,
                                   S.s_copy) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(q->base + q->o_values, r.values, (size_t)r.nnz * q->es, cudaMemcpyHostToDevice,
                                   S.s_copy) == cudaSuccess;
      }
    }
    if (!q->is_op) {
      ok = ok && cudaMemcpyAsync(q->base + q->o_V, r.V, (size_t)q->vrows() * r.n * q->es, cudaMemcpyHostToDevice,
                                 S.s_copy) == cudaSuccess;
      if (q->op) {  // the operator's selection, with s for this request's tol
        q->params_in = q->op->params;
        q->params_in.s = s_for_tol(q->op->params, r.tol, S.sel_opts.m);
        q->params = q->params_in;
        ok = ok && cudaMemcpyAsync(q->base + q->o_params, &q->params_in, sizeof(phic_params), cudaMemcpyHostToDevice,
                                   S.s_copy) == cudaSuccess;
      }
    }
    ok = ok && cudaEventRecord(q->ev_in, S.s_copy) == cudaSuccess;
    itq = S.queued.erase(itq);
    {
      std::lock_guard<std::mutex> lk(S.mu);
      q->t_admit = now_ns();
      q->state = PHIC_REQ_LOADING;
      S.ctr.admitted += 1;
      S.ctr.arena_in_use = (int64_t)S.pool.in_use();
      S.ctr.arena_peak = (int64_t)S.pool.peak();
    }
    if (!ok) {
      // copies enqueued before the failing one may still be writing into the request's blocks: let them
      // end before the blocks go back to the pool, where the next request could take the same ranges
      cudaStreamSynchronize(S.s_copy);
      release_blocks(S, q);
      drop_op_ref(S, q);
      finish_req(S, q, PHIC_CUDA_ERROR);
      continue;
    }
    S.loading.push_back(q);
  }
}

void promote_loaded(phic_server& S) {
  for (size_t k = 0; k < S.loading.size();) {
    Req* q = S.loading[k];
    const cudaError_t e = cudaEventQuery(q->ev_in);
    if (e == cudaErrorNotReady) {
      ++k;
      continue;
    }
    S.loading.erase(S.loading.begin() + k);
    if (e != cudaSuccess) {
      release_blocks(S, q);
      drop_op_ref(S, q);
      finish_req(S, q, PHIC_CUDA_ERROR);
      continue;
    }
    set_state(S, q, PHIC_REQ_RUNNING);
    S.running.push_back(q);
  }
}

phic_csr device_csr(const Req* q) {
  const Req* o = q->own_csr() ? q : q->op;
  phic_csr c;
  c.n = o->r.n;
  c.nnz = o->r.nnz;
  c.rowptr = reinterpret_cast<const int32_t*>(o->base + o->o_rowptr);
  c.colidx = reinterpret_cast<const int32_t*>(o->base + o->o_colidx);
  c.values = o->base + o->o_values;
  c.prec = o->r.prec;
  return c;
}

// The requests of the next slice: every running request that has already taken part in a slice (its
// per-slice work is bounded by max_steps), then new ones in arrival order while the estimated work,
// spread over the launch's CTAs, stays within the slice budget (at least one request per slice).
void pick_slice(phic_server& S) {
  S.slice.clear();
  double work = 0.0;  // estimated CTA-microseconds
  // the budget grows with the backlog: short slices (latency) at light load, longer ones (throughput)
  // when many requests wait
  size_t fresh = 0;
  for (const Req* q : S.running) fresh += q->slices == 0 ? 1 : 0;
  const double scale = std::min(16.0, std::max(1.0, (double)(fresh + S.queued.size()) / 16.0));
  const double budget = S.cfg.slice_us * scale * (double)S.grid;
  const CostModel cm;
  for (int pass = 0; pass < 2; ++pass) {
    for (Req* q : S.running) {
      if ((int)S.slice.size() >= S.cfg.max_active) return;
      const bool fresh = q->slices == 0;
      if ((pass == 0) == fresh) continue;
      phic_batch_item it;
      std::memset(&it, 0, sizeof(it));
      it.A.n = q->r.n;
      it.A.prec = q->r.prec;
      it.p = q->r.p;
      it.r = q->r.r;
      it.flags = q->selected ? 0u : PHIC_BATCH_SELECT;
      it.s_hint = q->s_hint;
      for (int j = 0; j < q->r.r; ++j) it.t[j] = q->r.t[j];
      const long long want = (q->r.n + S.cfg.rows_per_cta - 1) / S.cfg.rows_per_cta;
      const int team = (int)std::max<long long>(1, std::min<long long>(want, S.grid));
      const double d = item_duration(it, S.sel_opts, team, fresh, cm) * team;
      if (pass == 1 && !S.slice.empty() && work + d > budget) return;
      work += d;
      S.slice.push_back(q);
    }
  }
}

void start_slice(phic_server& S) {
  pick_slice(S);
  const int k = (int)S.slice.size();
  std::vector<phic_batch_item> items(k);
  std::vector<char> first(k);
  for (int i = 0; i < k; ++i) {
    const Req* q = S.slice[i];
    phic_batch_item& it = items[i];
    std::memset(&it, 0, sizeof(it));
    it.A = device_csr(q);
    it.p = q->r.p;
    it.r = q->r.r;
    it.flags = (q->r.flags & PHIC_NO_V0) | (q->selected ? 0u : PHIC_BATCH_SELECT) |
               (q->is_op ? PHIC_BATCH_NO_SOLVE : 0u);
    it.max_terms = q->r.max_terms;
    it.tol = q->r.tol;
    it.s_hint = q->s_hint;
    for (int j = 0; j < q->r.r; ++j) {
      it.t[j] = q->r.t[j];
      it.alpha[j] = q->r.alpha[j];
    }
    first[i] = q->slices == 0 ? 1 : 0;
  }
  Schedule plan;
  plan_core(items.data(), k, S.sel_opts, S.grid, S.cfg.rows_per_cta, true, plan, &first);
  Ctl* ctl = reinterpret_cast<Ctl*>(S.arena + S.h_ctl);
  for (int i = 0; i < k; ++i) {
    Req* q = S.slice[i];
    BatchInst& bi = S.st_inst[i];
    std::memset(&bi, 0, sizeof(bi));
    const phic_csr A = device_csr(q);
    if (!q->is_op)
      fill_solve_args(bi.sa, &A, q->r.p, q->r.r, q->base + q->o_V, q->r.t, q->r.alpha, q->r.tol,
                      reinterpret_cast<phic_params*>(q->base + q->o_params), q->r.flags & PHIC_NO_V0, q->r.max_terms,
                      q->base + q->o_W, q->base + q->o_solve, q->sl,
                      reinterpret_cast<phic_stats*>(q->base + q->o_stats), spin_limit_ns());
    bi.sa.ctlS = bi.sa.ctlR = ctl + i;
    bi.phases = 0;
    if (!q->is_op) bi.phases = q->slices == 0 ? (kPhaseSeries | kPhaseRecover) : kPhaseRecover;
    if (!q->selected) {
      phic_select_opts o = S.sel_opts;
      o.tol = q->r.tol;
      fill_select_args(bi.sel, &A, o, nullptr, q->sel_base, q->sel, reinterpret_cast<phic_params*>(q->base + q->o_params));
      bi.sel.ctl = ctl + i;
      bi.phases |= kPhaseSelect;
    }
    bi.team = plan.team[i];
    bi.prec = q->r.prec;
    bi.max_steps = S.cfg.max_steps;
  }
  std::memcpy(S.st_ptr, plan.sched_ptr.data(), plan.sched_ptr.size() * sizeof(int));
  if (!plan.sched.empty()) std::memcpy(S.st_sched, plan.sched.data(), plan.sched.size() * sizeof(SchedEntry));
  cudaStream_t st = S.s_compute;
  bool ok = cudaMemcpyAsync(S.arena + S.h_inst, S.st_inst, (size_t)k * sizeof(BatchInst), cudaMemcpyHostToDevice, st) ==
            cudaSuccess;
  ok = ok && cudaMemcpyAsync(S.arena + S.h_ptr, S.st_ptr, plan.sched_ptr.size() * sizeof(int), cudaMemcpyHostToDevice,
                             st) == cudaSuccess;
  if (!plan.sched.empty())
    ok = ok && cudaMemcpyAsync(S.arena + S.h_sched, S.st_sched, plan.sched.size() * sizeof(SchedEntry),
                               cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(S.arena + S.h_ctl, 0, (size_t)k * sizeof(Ctl), st) == cudaSuccess;
  ok = ok && cudaEventRecord(S.ev_start, st) == cudaSuccess;
  BatchArgs a;
  a.inst = reinterpret_cast<const BatchInst*>(S.arena + S.h_inst);
  a.sched_ptr = reinterpret_cast<const int*>(S.arena + S.h_ptr);
  a.sched = reinterpret_cast<const SchedEntry*>(S.arena + S.h_sched);
  a.spin_ns = spin_limit_ns();
  ok = ok && launch_batch(a, S.grid, S.minb, st) == cudaSuccess;
  int* d_done = reinterpret_cast<int*>(S.arena + S.h_done);
  phic_stats* d_stats = reinterpret_cast<phic_stats*>(S.arena + S.h_stats);
  phic_params* d_params = reinterpret_cast<phic_params*>(S.arena + S.h_params);
  ok = ok && launch_batch_collect(a.inst, k, d_done, d_stats, d_params, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(S.hb_done, d_done, (size_t)k * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(S.hb_stats, d_stats, (size_t)k * sizeof(phic_stats), cudaMemcpyDeviceToHost, st) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(S.hb_params, d_params, (size_t)k * sizeof(phic_params), cudaMemcpyDeviceToHost, st) ==
                 cudaSuccess;
  ok = ok && cudaEventRecord(S.ev_end, st) == cudaSuccess;
  S.launch_err = ok ? cudaSuccess : cudaErrorLaunchFailure;
  S.inflight = true;
  std::lock_guard<std::mutex> lk(S.mu);
  S.ctr.slices += 1;
  S.ctr.max_slice_requests = std::max<int64_t>(S.ctr.max_slice_requests, k);
}

void finish_slice(phic_server& S, cudaError_t e) {
  if (e == cudaSuccess && S.launch_err != cudaSuccess) e = S.launch_err;
  float ms = 0.f;
  if (e == cudaSuccess && cudaEventElapsedTime(&ms, S.ev_start, S.ev_end) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(S.mu);
    S.ctr.gpu_busy_ms += ms;
  }
  const int k = (int)S.slice.size();
  for (int i = 0; i < k; ++i) {
    Req* q = S.slice[i];
    q->slices += 1;
    if (e != cudaSuccess) {
      S.running.erase(std::find(S.running.begin(), S.running.end(), q));
      if (!q->is_op) release_blocks(S, q);
      drop_op_ref(S, q);
      finish_req(S, q, PHIC_CUDA_ERROR);
      continue;
    }
    q->params = S.hb_params[i];
    if (q->is_op) {  // a registered operator: Algorithm 1 is all it runs
      q->selected = true;
      if (q->have_sel) {
        S.pool.release(q->off_sel, q->bytes_sel);
        q->have_sel = false;
      }
      S.running.erase(std::find(S.running.begin(), S.running.end(), q));
      {
        std::lock_guard<std::mutex> lk(S.mu);
        q->op_ready = q->params.status == PHIC_OK;
        q->status = q->params.status;
        q->t_done = now_ns();
        q->state = PHIC_REQ_DONE;
      }
      S.cv_done.notify_all();
      continue;
    }
    if (!q->selected) {
      q->selected = true;
      q->s_hint = std::isfinite(q->params.s) ? q->params.s : 0.0;
      if (q->have_sel) {  // Algorithm 1's basis is no longer needed
        S.pool.release(q->off_sel, q->bytes_sel);
        q->have_sel = false;
      }
    }
    if (!S.hb_done[i]) continue;
    q->stats = S.hb_stats[i];
    q->status = q->stats.status;
    S.running.erase(std::find(S.running.begin(), S.running.end(), q));
    bool ok = cudaStreamWaitEvent(S.s_copy, S.ev_end, 0) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(q->r.W, q->base + q->o_W, (size_t)q->r.r * q->r.n * q->es, cudaMemcpyDeviceToHost,
                               S.s_copy) == cudaSuccess;
    ok = ok && cudaEventRecord(q->ev_out, S.s_copy) == cudaSuccess;
    if (!ok) {
      release_blocks(S, q);
      drop_op_ref(S, q);
      finish_req(S, q, PHIC_CUDA_ERROR);
      continue;
    }
    set_state(S, q, PHIC_REQ_COPYING);
    S.copying.push_back(q);
  }
  S.slice.clear();
  S.inflight = false;
  std::lock_guard<std::mutex> lk(S.mu);
  S.ctr.arena_in_use = (int64_t)S.pool.in_use();
}

void worker_main(phic_server* Sp) {
  phic_server& S = *Sp;
  cudaSetDevice(S.cfg.device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S.mu);
      if (S.stop) break;
      while (!S.incoming.empty()) {
        S.queued.push_back(S.incoming.front());
        S.incoming.pop_front();
      }
      const bool idle = S.queued.empty() && S.loading.empty() && S.running.empty() && S.copying.empty() && !S.inflight;
      if (idle) {
        S.cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    retire_copies(S);
    collect_removed_ops(S);
    admit(S);
    promote_loaded(S);
    if (S.inflight) {
      const cudaError_t e = cudaEventQuery(S.ev_end);
      if (e == cudaErrorNotReady) {
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        continue;
      }
      finish_slice(S, e);
      retire_copies(S);
      admit(S);
      promote_loaded(S);
    }
    if (!S.inflight && !S.running.empty()) {
      start_slice(S);
    } else if (!S.inflight) {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  cudaStreamSynchronize(S.s_compute);
  cudaStreamSynchronize(S.s_copy);
}

void destroy_server(phic_server* S) {
  if (!S) return;
  if (S->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    S->worker.join();
  }
  for (auto& kv : S->all) {
    if (kv.second->ev_in) cudaEventDestroy(kv.second->ev_in);
    if (kv.second->ev_out) cudaEventDestroy(kv.second->ev_out);
    delete kv.second;
  }
  if (S->ev_start) cudaEventDestroy(S->ev_start);
  if (S->ev_end) cudaEventDestroy(S->ev_end);
  if (S->s_compute) cudaStreamDestroy(S->s_compute);
  if (S->s_copy) cudaStreamDestroy(S->s_copy);
  cudaFreeHost(S->st_inst);
  cudaFreeHost(S->st_ptr);
  cudaFreeHost(S->st_sched);
  cudaFreeHost(S->hb_done);
  cudaFreeHost(S->hb_stats);
  cudaFreeHost(S->hb_params);
  delete S;
}

}  // namespace
}  // namespace phic

using namespace phic;

extern "C" {

phic_status phic_server_create(const phic_server_config* cfg, phic_server** out) {
  if (!cfg || !out || !cfg->arena || !aligned(cfg->arena)) return PHIC_INVALID_ARG;
  *out = nullptr;
  phic_server* S = new (std::nothrow) phic_server();
  if (!S) return PHIC_CUDA_ERROR;
  S->cfg = *cfg;
  if (S->cfg.rows_per_cta <= 0) S->cfg.rows_per_cta = 4096;
  if (S->cfg.blocks_per_sm <= 0) S->cfg.blocks_per_sm = 2;
  if (S->cfg.max_steps <= 0) S->cfg.max_steps = 4;
  if (!(S->cfg.slice_us > 0.0)) S->cfg.slice_us = 20000.0;
  if (S->cfg.max_active <= 0) S->cfg.max_active = 1024;
  if (S->cfg.m <= 0) S->cfg.m = 61;
  if (S->cfg.rows_per_cta < 256 || S->cfg.blocks_per_sm > 3 || S->cfg.m > 128) {
    delete S;
    return PHIC_INVALID_ARG;
  }
  phic_select_opts_default(&S->sel_opts);
  S->sel_opts.m = S->cfg.m;
  if (cudaSetDevice(S->cfg.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->cfg.device) != cudaSuccess) {
    delete S;
    return PHIC_CUDA_ERROR;
  }
  S->minb = S->cfg.blocks_per_sm >= 3 ? 3 : 2;
  const int occ = batch_occupancy(S->minb);
  if (occ < 1) {
    delete S;
    return PHIC_CUDA_ERROR;
  }
  S->grid = S->sms * std::min(S->cfg.blocks_per_sm, occ);
  S->sched_cap = (size_t)S->cfg.max_active * (size_t)S->grid;
  const int A = S->cfg.max_active;
  size_t off = 0;
  S->h_ctl = off; off += align_up((size_t)A * sizeof(Ctl));
  S->h_inst = off; off += align_up((size_t)A * sizeof(BatchInst));
  S->h_ptr = off; off += align_up((size_t)(S->grid + 1) * sizeof(int));
  S->h_sched = off; off += align_up(S->sched_cap * sizeof(SchedEntry));
  S->h_done = off; off += align_up((size_t)A * sizeof(int));
  S->h_stats = off; off += align_up((size_t)A * sizeof(phic_stats));
  S->h_params = off; off += align_up((size_t)A * sizeof(phic_params));
  S->head = off;
  if (cfg->arena_bytes <= S->head) {
    delete S;
    return PHIC_WORKSPACE_TOO_SMALL;
  }
  S->arena = static_cast<char*>(cfg->arena);
  S->pool.init((cfg->arena_bytes - S->head) / 256 * 256);
  bool ok = cudaMallocHost(&S->st_inst, (size_t)A * sizeof(BatchInst)) == cudaSuccess;
  ok = ok && cudaMallocHost(&S->st_ptr, (size_t)(S->grid + 1) * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&S->st_sched, S->sched_cap * sizeof(SchedEntry)) == cudaSuccess;
  ok = ok && cudaMallocHost(&S->hb_done, (size_t)A * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&S->hb_stats, (size_t)A * sizeof(phic_stats)) == cudaSuccess;
  ok = ok && cudaMallocHost(&S->hb_params, (size_t)A * sizeof(phic_params)) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&S->s_compute, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&S->s_copy, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreate(&S->ev_start) == cudaSuccess;
  ok = ok && cudaEventCreate(&S->ev_end) == cudaSuccess;
  if (!ok) {
    destroy_server(S);
    return PHIC_CUDA_ERROR;
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return PHIC_OK;
}

static phic_status enqueue_job(phic_server* S, Req* q, int64_t* id) {
  plan_blocks(*q, S->cfg.m);
  const size_t pool_total = (S->cfg.arena_bytes - S->head) / 256 * 256;
  if (align_up(q->bytes_main) + align_up(q->bytes_sel) > pool_total) {
    if (q->op) {
      std::lock_guard<std::mutex> lk(S->mu);
      q->op->op_refs -= 1;
    }
    delete q;
    return PHIC_WORKSPACE_TOO_SMALL;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->id = S->next_id++;
    if (q->is_op) S->ops.push_back(q);
    q->t_submit = now_ns();
    S->all[q->id] = q;
    S->incoming.push_back(q);
    S->ctr.submitted += 1;
    *id = q->id;
  }
  S->cv_work.notify_one();
  return PHIC_OK;
}

phic_status phic_server_submit(phic_server* S, const phic_request* req, int64_t* id) {
  if (!S || !req || !id || !request_ok(*req)) return PHIC_INVALID_ARG;
  Req* q = new (std::nothrow) Req();
  if (!q) return PHIC_CUDA_ERROR;
  q->r = *req;
  if (req->op != 0) {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(req->op);
    if (it == S->all.end() || !it->second->is_op || it->second->op_removed || it->second->r.n != req->n ||
        it->second->r.prec != req->prec) {
      delete q;
      return PHIC_INVALID_ARG;
    }
    q->op = it->second;
    q->op->op_refs += 1;
    q->selected = true;  // Algorithm 1 ran for the operator
  }
  return enqueue_job(S, q, id);
}

phic_status phic_server_add_operator(phic_server* S, const phic_operator* op, int64_t* id) {
  if (!S || !op || !id) return PHIC_INVALID_ARG;
  if (op->n < 1 || op->n >= (int64_t)INT32_MAX || op->nnz < 0 || op->nnz >= (int64_t)INT32_MAX || !op->rowptr ||
      (op->nnz > 0 && (!op->colidx || !op->values)) || (op->prec != PHIC_F64 && op->prec != PHIC_F32))
    return PHIC_INVALID_ARG;
  Req* q = new (std::nothrow) Req();
  if (!q) return PHIC_CUDA_ERROR;
  q->is_op = true;
  q->r.n = op->n;
  q->r.nnz = op->nnz;
  q->r.rowptr = op->rowptr;
  q->r.colidx = op->colidx;
  q->r.values = op->values;
  q->r.prec = op->prec;
  q->r.p = 0;
  q->r.r = 1;
  q->r.tol = std::ldexp(1.0, -53);  // the reference tolerance; requests rescale s for their own
  return enqueue_job(S, q, id);
}

phic_status phic_server_operator_params(phic_server* S, int64_t id, int32_t* ready, phic_params* params) {
  if (!S || !ready) return PHIC_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end() || !it->second->is_op) return PHIC_INVALID_ARG;
  *ready = it->second->op_ready ? 1 : 0;
  if (params) *params = it->second->params;
  return it->second->state == PHIC_REQ_DONE ? (phic_status)it->second->status : PHIC_OK;
}

phic_status phic_server_remove_operator(phic_server* S, int64_t id) {
  if (!S) return PHIC_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end() || !it->second->is_op) return PHIC_INVALID_ARG;
    it->second->op_removed = true;
  }
  S->cv_work.notify_one();
  return PHIC_OK;
}

static void fill_info(const Req* q, phic_request_info* info) {
  std::memset(info, 0, sizeof(*info));
  info->state = q->state;
  info->status = q->status;
  info->submit_ns = q->t_submit;
  info->admit_ns = q->t_admit;
  info->done_ns = q->t_done;
  info->slices = q->slices;
  info->params = q->params;
  info->stats = q->stats;
}

phic_status phic_server_query(phic_server* S, int64_t id, phic_request_info* info) {
  if (!S || !info) return PHIC_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return PHIC_INVALID_ARG;
  fill_info(it->second, info);
  return PHIC_OK;
}

phic_status phic_server_wait(phic_server* S, int64_t id, double timeout_ms, phic_request_info* info) {
  if (!S) return PHIC_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return PHIC_INVALID_ARG;
  Req* q = it->second;
  auto done = [&] { return q->state == PHIC_REQ_DONE; };
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, done);
  } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds((long long)(timeout_ms * 1000.0)), done)) {
    if (info) fill_info(q, info);
    return PHIC_TIMEOUT;
  }
  if (info) fill_info(q, info);
  return PHIC_OK;
}

phic_status phic_server_counters_get(phic_server* S, phic_server_counters* out) {
  if (!S || !out) return PHIC_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->ctr;
  return PHIC_OK;
}

void phic_server_destroy(phic_server* S) { destroy_server(S); }

}  // extern "C"
