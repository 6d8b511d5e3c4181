"""The batched launch's planner on the host (phic_batch_plan_host, no GPU): every instance gets its team
exactly once with ranks 0..c-1, team sizes follow rows_per_cta, and the CTAs' lists follow one global
order, so that a run in which each team starts only when all its members have reached it can never
wait in a cycle (checked by simulating that run)."""
import ctypes

import numpy as np
import pytest

from paper_2509_26475_gb300 import capi
from paper_2509_26475_gb300 import workloads as wl


def _items(specs):
    arr = (capi.phic_batch_item * len(specs))()
    fake = 0x1000  # never dereferenced by the host planner
    for i, sp in enumerate(specs):
        it = arr[i]
        it.A = capi.phic_csr(sp["n"], sp["nnz"], fake, fake, fake, sp.get("prec", 0))
        it.p, it.r = sp["p"], len(sp["t"])
        it.flags = sp.get("flags", capi.PHIC_BATCH_SELECT)
        it.V, it.W, it.params = fake, fake, fake
        it.tol = 2.0**-53
        it.s_hint = sp.get("s_hint", 0.0)
        for j, tj in enumerate(sp["t"]):
            it.t[j], it.alpha[j] = tj, 1.0
    return arr


def _plan(specs, grid, rows):
    lib = capi.load(build_if_missing=True)
    arr = _items(specs)
    cfg = capi.phic_batch_config(rows, 2, 0, 0)
    cap = sum(min(grid, -(-sp["n"] // 256)) for sp in specs) + 8
    team = (ctypes.c_int32 * len(specs))()
    ptr = (ctypes.c_int32 * (grid + 1))()
    sched = (ctypes.c_int32 * (2 * cap))()
    ent = ctypes.c_int64(0)
    mk = ctypes.c_double(0.0)
    st = lib.phic_batch_plan_host(arr, len(specs), None, ctypes.byref(cfg), grid, team, ptr, sched, cap,
                                  ctypes.byref(ent), ctypes.byref(mk))
    assert st == capi.PHIC_OK
    lists = [[(sched[2 * e], sched[2 * e + 1]) for e in range(ptr[g], ptr[g + 1])] for g in range(grid)]
    return list(team), lists, mk.value, ent.value


def _simulate(lists, team):
    """Each CTA works through its list; an instance runs once every member is at it.  Returns True when
    every list is consumed."""
    pos = [0] * len(lists)
    progress = True
    while progress:
        progress = False
        waiting = {}
        for g, lst in enumerate(lists):
            if pos[g] < len(lst):
                waiting.setdefault(lst[pos[g]][0], []).append(g)
        for inst, members in waiting.items():
            if len(members) == team[inst]:
                for g in members:
                    pos[g] += 1
                progress = True
    return all(pos[g] == len(lst) for g, lst in enumerate(lists))


def _specs_from_workload(count, seed, n_hi=256000):
    out = []
    for i in range(count):
        rng = np.random.default_rng([seed, i])
        n = int(np.exp(rng.uniform(np.log(1000), np.log(n_hi))))
        p = int(rng.integers(1, 5))
        r = int(rng.integers(1, 4))
        out.append(dict(n=n, nnz=5 * n, p=p, t=list(np.linspace(1e-3, 2e-3, r)), s_hint=float(rng.uniform(0, 5e3)),
                        prec=int(rng.integers(0, 2))))
    return out


@pytest.mark.parametrize("grid,rows", [(304, 4096), (456, 1024), (7, 512), (1, 4096)])
def test_every_instance_once_with_its_team(grid, rows):
    specs = _specs_from_workload(64, 11)
    team, lists, mk, ent = _plan(specs, grid, rows)
    for i, sp in enumerate(specs):
        assert team[i] == max(1, min(grid, -(-sp["n"] // rows)))
    seen = {}
    for lst in lists:
        for inst, rank in lst:
            seen.setdefault(inst, []).append(rank)
    assert sorted(seen) == list(range(len(specs)))
    for inst, ranks in seen.items():
        assert sorted(ranks) == list(range(team[inst]))
    assert ent == sum(team)
    assert mk > 0.0


@pytest.mark.parametrize("grid,rows", [(304, 4096), (456, 512), (13, 256)])
def test_lists_follow_one_global_order_and_never_deadlock(grid, rows):
    specs = _specs_from_workload(96, 12)
    team, lists, _, _ = _plan(specs, grid, rows)
    # a global order exists: the precedence pairs of all lists form no cycle (Kahn's algorithm)
    n = len(specs)
    succ = [set() for _ in range(n)]
    indeg = [0] * n
    for lst in lists:
        for (a, _), (b, _) in zip(lst, lst[1:]):
            if b not in succ[a]:
                succ[a].add(b)
                indeg[b] += 1
    ready = [i for i in range(n) if indeg[i] == 0]
    done = 0
    while ready:
        a = ready.pop()
        done += 1
        for b in succ[a]:
            indeg[b] -= 1
            if indeg[b] == 0:
                ready.append(b)
    assert done == n
    assert _simulate(lists, team)


def test_longest_instances_start_first():
    specs = [dict(n=1000, nnz=5000, p=1, t=[1e-3]), dict(n=250000, nnz=1250000, p=3, t=[1e-3, 2e-3]),
             dict(n=5000, nnz=25000, p=2, t=[1e-3])]
    team, lists, _, _ = _plan(specs, 16, 4096)
    firsts = [lst[0][0] for lst in lists if lst]
    assert firsts.count(1) == team[1]  # the large instance heads the lists of all its members


def test_host_checks_reject_bad_items():
    lib = capi.load(build_if_missing=True)
    arr = _items([dict(n=1000, nnz=5000, p=2, t=[1e-3])])
    size = ctypes.c_size_t(0)
    arr[0].p = 16  # above PHIC_MAX_P
    assert lib.phic_batch_workspace_size(arr, 1, None, ctypes.byref(size)) == capi.PHIC_INVALID_ARG
    arr[0].p = 2
    arr[0].flags = capi.PHIC_BATCH_NO_SOLVE  # Algorithm 1 only, but not requested
    assert lib.phic_batch_workspace_size(arr, 1, None, ctypes.byref(size)) == capi.PHIC_INVALID_ARG
    arr[0].flags = 0
    arr[0].params = None
    assert lib.phic_batch_workspace_size(arr, 1, None, ctypes.byref(size)) == capi.PHIC_INVALID_ARG
    assert lib.phic_batch_workspace_size(arr, 0, None, ctypes.byref(size)) == capi.PHIC_INVALID_ARG


def test_hints_steer_the_cost_model():
    """s_hint sets an instance's outer steps ceil(s_hint max|t|): of two otherwise equal instances the one
    with the larger hint is costed longer and placed first, and the estimated makespan grows with it."""
    base = dict(n=50000, nnz=250000, p=3, t=[1e-3, 2e-3], prec=1)
    small = dict(base, s_hint=500.0)    # one outer step
    large = dict(base, s_hint=20000.0)  # 40 outer steps
    team, lists, mk_mix, _ = _plan([small, large], 16, 4096)
    firsts = [lst[0][0] for lst in lists if lst]
    assert firsts.count(1) == team[1]  # the long instance heads the lists of all its members
    _, _, mk_small, _ = _plan([small, dict(small)], 16, 4096)
    _, _, mk_large, _ = _plan([large, dict(large)], 16, 4096)
    assert mk_small < mk_mix < mk_large
