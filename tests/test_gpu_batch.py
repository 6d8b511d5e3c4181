"""Batched launches on the GPU, through the C ABI.

A solve's result does not depend on its team size or on the other instances of the launch (the
truncation decisions use infinity norms, i.e. maxima, and the per-row arithmetic is the same code), so a
batched solve must equal the single-instance solve with the same (s, xi) bit for bit, alone or in any
mix, in one launch or in slices.  Algorithm 1 inside a batch is compared with the oracle like the
single-instance selection (s within 5 %), and the batched results with the oracle at the parity bars
(1e-12 FP64 at tol 2^-53, 5e-6 FP32 at tol 2^-24).
"""
import numpy as np
import pytest
import torch

from paper_2509_26475_gb300 import api, capi
from paper_2509_26475_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_26475_gb300 import build

    build.build()
    capi.load()
    torch.cuda.set_device(0)


def _dev(inst):
    dt = torch.float32 if inst["prec"] == "f32" else torch.float64
    A = api.DeviceCSR.from_host(inst["A"], dtype=dt)
    V = torch.as_tensor(inst["V"]).to(dt).cuda()
    return A, V


def _instances(count, seed, n_lo=300, n_hi=30000, precision="mixed"):
    return [wl.batch_instance(seed, i, n_lo, n_hi, precision) for i in range(count)]


def _single(inst, A, V):
    P = api.select_params(A, tol=inst["tol"])
    W, st = api.solve(A, V, inst["t"], inst["alpha"], inst["tol"], P)
    torch.cuda.synchronize()
    return P, W, api.read_stats(st)


def _items(insts, devs, params=None, select=False):
    out = []
    for k, (inst, (A, V)) in enumerate(zip(insts, devs)):
        P = params[k].clone() if params is not None else None
        out.append(api.BatchItem(A, V, inst["t"], inst["alpha"], tol=inst["tol"], select=select, params=P,
                                 s_hint=(api.read_params(params[k])["s"] if params is not None else 0.0)))
    return out


def test_batch_equals_single_instance_bitwise():
    insts = _instances(12, 7)
    devs = [_dev(x) for x in insts]
    singles = [_single(x, *d) for x, d in zip(insts, devs)]
    items = _items(insts, devs, params=[s[0] for s in singles])
    b = api.Batch(items, config={"rows_per_cta": 1024, "blocks_per_sm": 2})
    b.launch()
    torch.cuda.synchronize()
    info = b.info()
    assert info["count"] == 12 and info["grid"] >= 2
    for k, (it, (P, W, st)) in enumerate(zip(items, singles)):
        bs = api.read_stats(it.stats)
        assert bs["status"] == 0, (k, bs)
        assert bs["s_int"] == st["s_int"] and bs["series_terms"] == st["series_terms"]
        assert bs["recovery_terms"] == st["recovery_terms"]
        assert torch.equal(it.W, W), k


def test_wide_tiles_equal_single_instance_bitwise():
    """Series tiles of 36 to 128 columns (4 or 8 columns per lane) in both precisions, with the
    recoveries of 8 and 16 columns: the batched solve equals the single-instance solve bit for bit."""
    insts = []
    for k, (p, r, prec) in enumerate([(15, 8, "f64"), (10, 4, "f64"), (8, 4, "f32"), (15, 8, "f32")]):
        A = wl.convection_diffusion(20 + 3 * k, 2, 5.0)
        rng = np.random.default_rng(70 + k)
        insts.append(dict(A=A, V=rng.standard_normal((p + 1, A.n)), t=np.linspace(8e-3, 1.6e-2, r),
                          alpha=np.linspace(0.6, 1.2, r), tol=2.0**-53 if prec == "f64" else 2.0**-24, prec=prec,
                          p=p, r=r))
    devs = [_dev(x) for x in insts]
    singles = [_single(x, *d) for x, d in zip(insts, devs)]
    items = _items(insts, devs, params=[s[0] for s in singles])
    b = api.Batch(items, config={"rows_per_cta": 256, "blocks_per_sm": 2})
    b.launch()
    torch.cuda.synchronize()
    for k, (it, (P, W, st)) in enumerate(zip(items, singles)):
        bs = api.read_stats(it.stats)
        assert bs["status"] == 0 and st["status"] == 0, (k, bs, st)
        assert bs["s_int"] >= 2 and bs["recovery_terms"] == st["recovery_terms"], (k, bs, st)
        assert torch.equal(it.W, W), k


def test_batch_residency_and_team_size_do_not_change_results():
    insts = _instances(6, 8, precision="f64")
    devs = [_dev(x) for x in insts]
    params = [api.select_params(A, tol=x["tol"]) for x, (A, V) in zip(insts, devs)]
    ref = None
    for cfg in ({"rows_per_cta": 256, "blocks_per_sm": 2}, {"rows_per_cta": 16384, "blocks_per_sm": 3},
                {"rows_per_cta": 2048, "blocks_per_sm": 3}):
        items = _items(insts, devs, params=params)
        api.Batch(items, config=cfg).launch()
        torch.cuda.synchronize()
        Ws = [it.W.clone() for it in items]
        if ref is None:
            ref = Ws
        else:
            assert all(torch.equal(a, c) for a, c in zip(ref, Ws))


def test_batch_with_selection_against_oracle(oracle_mod):
    """Algorithm 1 inside the batch equals phic_select_params bit for bit (its sums are formed per fixed
    chunk of rows, whatever the team), and the batched results match the oracle run with those (s, xi)."""
    insts = _instances(6, 9, n_lo=300, n_hi=3000)
    devs = [_dev(x) for x in insts]
    items = _items(insts, devs, select=True)
    b = api.Batch(items, config={"rows_per_cta": 256})
    b.launch()
    torch.cuda.synchronize()
    for it, inst, (A, V) in zip(items, insts, devs):
        prm = api.read_params(it.params)
        st = api.read_stats(it.stats)
        assert prm["status"] == 0 and st["status"] == 0
        single = api.read_params(api.select_params(A, tol=inst["tol"]))
        assert prm == single, (prm, single)
        ref, _ = oracle_mod.solve(inst["A"], inst["V"], inst["t"], inst["alpha"], 2.0**-53, prm["s"], prm["xi"])
        W = it.W.double().cpu().numpy()
        err = max(np.linalg.norm(W[i] - ref[i]) / np.linalg.norm(ref[i]) for i in range(ref.shape[0]))
        assert err <= (5e-6 if inst["prec"] == "f32" else 1e-12), (inst["name"], err)


def test_alone_equals_in_the_mix():
    insts = _instances(10, 10)
    devs = [_dev(x) for x in insts]
    params = [api.select_params(A, tol=x["tol"]) for x, (A, V) in zip(insts, devs)]
    mix = _items(insts, devs, params=params)
    api.Batch(mix).launch()
    torch.cuda.synchronize()
    for k in (0, 4, 9):
        alone = _items([insts[k]], [devs[k]], params=[params[k]])
        api.Batch(alone).launch()
        torch.cuda.synchronize()
        assert torch.equal(alone[0].W, mix[k].W), k


def test_slices_equal_one_launch():
    insts = _instances(8, 11)
    for x in insts:  # longer steps: several recovery steps, so several slices
        x["t"] = x["t"] * 40.0
    devs = [_dev(x) for x in insts]
    params = [api.select_params(A, tol=x["tol"]) for x, (A, V) in zip(insts, devs)]
    whole = _items(insts, devs, params=params)
    api.Batch(whole).launch()
    sliced = _items(insts, devs, params=params)
    b = api.Batch(sliced, config={"max_steps": 1})
    b.launch()
    launches = 1
    while b.pending() > 0:
        b.resume()
        launches += 1
        assert launches < 10000
    torch.cuda.synchronize()
    assert launches > 1  # some instance needs more than one recovery step
    for a, c in zip(whole, sliced):
        assert api.read_stats(c.stats)["status"] == 0
        assert torch.equal(a.W, c.W)
        assert api.read_stats(a.stats)["recovery_terms"] == api.read_stats(c.stats)["recovery_terms"]


def test_graph_capture_and_replay():
    insts = _instances(6, 12)
    devs = [_dev(x) for x in insts]
    params = [api.select_params(A, tol=x["tol"]) for x, (A, V) in zip(insts, devs)]
    items = _items(insts, devs, params=params)
    b = api.Batch(items)
    b.launch()
    torch.cuda.synchronize()
    eager = [it.W.clone() for it in items]
    for it in items:
        it.W.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.launch(stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, it.W) for a, it in zip(eager, items))


def test_autotune_picks_a_candidate():
    insts = _instances(8, 13, precision="f64")
    devs = [_dev(x) for x in insts]
    items = _items(insts, devs, select=True)
    cands = [{"rows_per_cta": 512, "blocks_per_sm": 2}, {"rows_per_cta": 4096, "blocks_per_sm": 3}]
    best, ms = api.autotune(items, candidates=cands, reps=2)
    assert best in [dict(c, max_steps=0) for c in cands]
    assert ms > 0.0
    assert all(api.read_stats(it.stats)["status"] == 0 for it in items)


def test_planner_hints_from_operator_norms():
    """Items that run Algorithm 1 without an s_hint are planned with ||A||_inf / (2 (tol m!)^(1/m)),
    the norms taken on the device: the batch's plan equals the host planner's for the same hints
    computed on the host (row sums in the same order, in FP64 of the stored values)."""
    import ctypes
    import math

    insts = _instances(10, 23)
    devs = [_dev(x) for x in insts]
    items = _items(insts, devs, select=True)
    b = api.Batch(items, config={"rows_per_cta": 1024, "blocks_per_sm": 2})
    info = b.info()
    m = b.opts.m
    arr = api._item_array(items)
    for k, x in enumerate(insts):
        A = x["A"]
        lens = np.diff(A.rowptr)
        dt = np.float32 if x["prec"] == "f32" else np.float64
        vals = np.abs(np.asarray(A.values).astype(dt)).astype(np.float64)
        sums = np.zeros(A.n)
        for q in range(int(lens.max())):  # entry q of every row, in the device's order
            has = lens > q
            sums[has] = sums[has] + vals[A.rowptr[:-1][has] + q]
        theta = math.exp((math.log(x["tol"]) + math.lgamma(m + 1.0)) / m)
        arr[k].s_hint = float(sums.max()) / (2.0 * theta)
        assert arr[k].s_hint > 0.0
    grid = info["grid"]
    cfg = capi.phic_batch_config(1024, 2, 0, 0)
    cap = info["entries"] + 8
    team = (ctypes.c_int32 * len(items))()
    ptr = (ctypes.c_int32 * (grid + 1))()
    sched = (ctypes.c_int32 * (2 * cap))()
    ent = ctypes.c_int64(0)
    mk = ctypes.c_double(0.0)
    st = capi.load().phic_batch_plan_host(arr, len(items), ctypes.byref(b.opts), ctypes.byref(cfg), grid, team, ptr,
                                          sched, cap, ctypes.byref(ent), ctypes.byref(mk))
    assert st == capi.PHIC_OK
    assert ent.value == info["entries"]
    assert mk.value == pytest.approx(info["est_makespan_us"], rel=1e-12)
    # without the hints every instance counts as one outer step: a shorter estimate
    for k in range(len(items)):
        arr[k].s_hint = 0.0
    st = capi.load().phic_batch_plan_host(arr, len(items), ctypes.byref(b.opts), ctypes.byref(cfg), grid, team, ptr,
                                          sched, cap, ctypes.byref(ent), ctypes.byref(mk))
    assert st == capi.PHIC_OK and mk.value < info["est_makespan_us"]
