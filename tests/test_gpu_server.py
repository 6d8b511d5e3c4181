"""The continuous-batching request loop (phic_server_*) on the GPU.

Requests are admitted by device memory and run together in batched slices; requests that arrive while
others run join the next slice.  A result does not depend on its neighbours or on the slicing (the
solve's decisions use maxima, Algorithm 1's sums are formed per fixed chunk of rows), so each result
must equal, bit for bit, the same request served alone, and match the oracle at the parity bars.
"""
import threading
import time

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


def _req(inst):
    return api.HostRequest(inst["A"], inst["V"], inst["t"], inst["alpha"], tol=inst["tol"], prec=inst["prec"])


def _instances(count, seed, n_lo=300, n_hi=20000):
    return [wl.batch_instance(seed, i, n_lo, n_hi, "mixed") for i in range(count)]


def test_results_match_oracle_and_single_selection(oracle_mod):
    insts = _instances(8, 21, n_hi=3000)
    srv = api.Server(arena_bytes=1 << 30)
    ids = [srv.submit(_req(x)) for x in insts]
    for rid, inst in zip(ids, insts):
        info = srv.wait(rid, timeout_ms=60000)
        assert info["state"] == capi.PHIC_REQ_DONE and info["status"] == 0, info
        prm = info["params"]
        dt = torch.float32 if inst["prec"] == "f32" else torch.float64
        single = api.read_params(api.select_params(api.DeviceCSR.from_host(inst["A"], dtype=dt), tol=inst["tol"]))
        assert prm == single
        ref, _ = oracle_mod.solve(inst["A"], inst["V"], inst["t"], inst["alpha"], 2.0**-53, prm["s"], prm["xi"])
        W = srv.result(rid).double().numpy()
        err = max(np.linalg.norm(W[i] - ref[i]) / np.linalg.norm(ref[i]) for i in range(ref.shape[0]))
        assert err <= (5e-6 if inst["prec"] == "f32" else 1e-12), (inst["name"], err)
    srv.close()


def test_same_result_alone_and_in_the_mix():
    insts = _instances(24, 22)
    k = 11
    alone = api.Server(arena_bytes=1 << 30, max_steps=1)
    rid = alone.submit(_req(insts[k]))
    assert alone.wait(rid, 60000)["status"] == 0
    W_alone = alone.result(rid).clone()
    alone.close()

    mix = api.Server(arena_bytes=1 << 30, max_steps=4)
    reqs = [_req(x) for x in insts]
    ids = [None] * len(insts)
    rng = np.random.default_rng(5)

    def arrivals():
        for i, q in enumerate(reqs):
            ids[i] = mix.submit(q)
            time.sleep(float(rng.exponential(0.002)))

    th = threading.Thread(target=arrivals)
    th.start()
    th.join()
    infos = [mix.wait(i, 120000) for i in ids]
    assert all(x["status"] == 0 for x in infos)
    assert torch.equal(mix.result(ids[k]), W_alone)
    c = mix.counters()
    assert c["completed"] == len(insts) and c["failed"] == 0
    assert c["max_slice_requests"] > 1  # requests did share slices
    mix.close()


def test_memory_admission_bounds_the_working_set():
    insts = _instances(10, 23, n_lo=20000, n_hi=30000)
    probe = api.Server(arena_bytes=1 << 30)
    rid = probe.submit(_req(insts[0]))
    probe.wait(rid, 60000)
    one = probe.counters()["arena_peak"]
    probe.close()
    # room for about two requests at a time
    srv = api.Server(arena_bytes=int(2.6 * one) + (64 << 20))
    ids = [srv.submit(_req(x)) for x in insts]
    infos = [srv.wait(i, 120000) for i in ids]
    assert all(x["status"] == 0 for x in infos)
    c = srv.counters()
    assert c["completed"] == 10
    assert c["max_slice_requests"] < 10  # admission held some requests back
    assert c["arena_peak"] <= int(2.6 * one) + (64 << 20)
    srv.close()


def test_request_larger_than_the_arena_is_refused():
    inst = _instances(1, 24, n_lo=50000, n_hi=60000)[0]
    srv = api.Server(arena_bytes=64 << 20)
    with pytest.raises(capi.PhicError) as e:
        srv.submit(_req(inst))
    assert e.value.status == capi.PHIC_WORKSPACE_TOO_SMALL
    srv.close()


def test_short_request_overtakes_a_long_one():
    """Continuous batching: a short request that arrives while a long one runs joins the next slice and
    finishes first."""
    A = wl.convection_diffusion(48, 3, 10.0)
    rng = np.random.default_rng(6)
    long_req = api.HostRequest(A, rng.standard_normal((4, A.n)), [2e-2, 1e-2], [0.5, 1.0])
    short = _instances(1, 25, n_lo=1000, n_hi=2000)[0]
    srv = api.Server(arena_bytes=1 << 30, max_steps=1)
    lid = srv.submit(long_req)
    time.sleep(0.02)
    sid = srv.submit(_req(short))
    si = srv.wait(sid, 60000)
    li = srv.wait(lid, 120000)
    assert si["status"] == 0 and li["status"] == 0
    assert li["stats"]["s_int"] > 4  # several slices
    assert si["done_ns"] < li["done_ns"]
    assert si["admit_ns"] < li["done_ns"]
    srv.close()


def test_registered_operator_is_shared_by_requests(oracle_mod):
    """Requests naming a registered operator reuse its Algorithm 1 result (s rescaled to each request's
    tol) and equal a direct solve with those parameters; FP64 and FP32 requests share one FP64 selection."""
    A = wl.convection_diffusion(30, 2, 20.0)
    srv = api.Server(arena_bytes=1 << 30, max_steps=2)
    oid = srv.add_operator(api.HostOperator(A))
    rng = np.random.default_rng(8)
    reqs = [api.HostRequest(A.n, rng.standard_normal((3, A.n)), [3e-3 * (k + 1), 1e-3], [1.0, 0.5], op=oid)
            for k in range(4)]
    ids = [srv.submit(q) for q in reqs]
    infos = [srv.wait(i, 60000) for i in ids]
    assert all(x["status"] == 0 for x in infos)
    prm = srv.operator_params(oid)
    single = api.read_params(api.select_params(api.DeviceCSR.from_host(A)))
    assert prm == single
    for q, info in zip(reqs, infos):
        assert info["params"]["xi"] == prm["xi"] and info["params"]["s"] == pytest.approx(prm["s"], rel=1e-14)
        ref, _ = oracle_mod.solve(A, q.V.numpy(), q.t, q.alpha, 2.0**-53, info["params"]["s"], prm["xi"])
        W = q.W.numpy()
        err = max(np.linalg.norm(W[i] - ref[i]) / np.linalg.norm(ref[i]) for i in range(2))
        assert err <= 1e-12
    srv.remove_operator(oid)
    srv.close()
