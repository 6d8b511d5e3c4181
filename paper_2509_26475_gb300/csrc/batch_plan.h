// Planner of the batched launches (shared by the batch C ABI and the serving loop).
//
// Instance i gets a team of c_i = min(G, ceil(n_i / rows_per_cta)) CTAs out of the launch's G.  A cost
// model (microseconds per pass of the kernels: a fixed barrier-and-latency part plus a part proportional
// to the rows times the tile width divided among the team) estimates each instance's duration d_i from
// its expected number of passes (Algorithm 1's power basis and Brent evaluations, the series terms, the
// recovery steps from s_hint).  Instances are taken in decreasing order of their area c_i d_i; each goes
// to the c_i CTAs that are free earliest, starting when the last of them is free (list scheduling of
// rigid parallel jobs).  Each CTA receives its instances in that one global order, so with every CTA
// resident (cooperative launch) team barriers cannot wait in a cycle.
#pragma once

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "kernels.h"
#include "phicomb.h"

namespace phic {

// Cost model, microseconds.
struct CostModel {
  double fixed_multi = 3.0;   // one pass of a team of several CTAs: barrier and load latencies
  double fixed_single = 1.5;  // one pass of a single-CTA team
  double per_elem = 0.0032;   // one row x one column on one CTA
  double pass(double rows, double width, int team) const {
    return (team > 1 ? fixed_multi : fixed_single) + per_elem * rows * width / team;
  }
};

inline double item_duration(const phic_batch_item& it, const phic_select_opts& o, int team, bool first_launch,
                     const CostModel& cm) {
  const bool do_select = (it.flags & PHIC_BATCH_SELECT) != 0, do_solve = (it.flags & PHIC_BATCH_NO_SOLVE) == 0;
  const double n = (double)it.A.n;
  double d = 0.0;
  if (first_launch && do_select) d += (double)(o.m + 1 + 100) * cm.pass(n, 2.0, team);
  if (do_solve) {
    const bool f32 = it.A.prec == PHIC_F32;
    const double terms = f32 ? 30.0 : 45.0;
    double tmax = 0.0;
    for (int i = 0; i < it.r; ++i) tmax = std::max(tmax, std::fabs(it.t[i]));
    const double sint = std::max(1.0, std::ceil(std::max(it.s_hint, 0.0) * tmax));
    const double wS = (double)(it.p + 1) * it.r, wF = it.p == 0 ? (double)it.r : 2.0 * it.r;
    if (first_launch) d += (terms + 2.0) * cm.pass(n, wS, team);
    d += (sint - 1.0) * (terms + 1.0) * cm.pass(n, wF, team) + 2.0 * cm.pass(n, wF, team);
  }
  return d;
}

struct Schedule {
  std::vector<int> team, sched_ptr;
  std::vector<SchedEntry> sched;
  double makespan = 0.0, busy = 1.0;
};

// Teams and schedule of one launch of G CTAs: list scheduling of the instances by decreasing area.
inline void plan_core(const phic_batch_item* items, int count, const phic_select_opts& o, int G, int rows_per_cta,
               bool first_launch, Schedule& out, const std::vector<char>* first_of = nullptr) {
  const CostModel cm;
  std::vector<double> dur(count), area(count);
  out.team.assign(count, 1);
  for (int i = 0; i < count; ++i) {
    const long long want = (items[i].A.n + rows_per_cta - 1) / rows_per_cta;
    out.team[i] = (int)std::max<long long>(1, std::min<long long>(want, G));
    dur[i] = item_duration(items[i], o, out.team[i], first_of ? (*first_of)[i] != 0 : first_launch, cm);
    area[i] = dur[i] * out.team[i];
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return area[x] > area[y]; });
  std::vector<double> load(G, 0.0);
  std::vector<int> idx(G);
  std::vector<std::vector<SchedEntry>> lists(G);
  double busy = 0.0;
  for (int i : order) {
    const int c = out.team[i];
    std::iota(idx.begin(), idx.end(), 0);
    auto earlier = [&](int x, int y) { return load[x] < load[y] || (load[x] == load[y] && x < y); };
    std::nth_element(idx.begin(), idx.begin() + (c - 1), idx.end(), earlier);
    std::sort(idx.begin(), idx.begin() + c);
    double start = 0.0;
    for (int q = 0; q < c; ++q) start = std::max(start, load[idx[q]]);
    for (int q = 0; q < c; ++q) {
      load[idx[q]] = start + dur[i];
      lists[idx[q]].push_back(SchedEntry{i, q});
    }
    busy += dur[i] * c;
  }
  out.sched_ptr.assign(G + 1, 0);
  out.sched.clear();
  for (int g = 0; g < G; ++g) {
    out.sched_ptr[g] = (int)out.sched.size();
    out.sched.insert(out.sched.end(), lists[g].begin(), lists[g].end());
  }
  out.sched_ptr[G] = (int)out.sched.size();
  out.makespan = *std::max_element(load.begin(), load.end());
  out.busy = out.makespan > 0.0 ? busy / ((double)G * out.makespan) : 1.0;
}

}  // namespace phic
