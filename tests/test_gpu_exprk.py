"""expRK4s6 on the paper's ADR problem (Section 6, fourth experiment) with every phi-combination on the
GPU: one step agrees with the same scheme evaluated by the oracle, and step halving shows fourth-order
convergence.  The paper's reference (a stiff MATLAB solver at 1e-12) is not available; the order test
replaces it."""
import math

import numpy as np
import pytest
import torch

from paper_2509_26475_gb300 import api, capi, exprk
from paper_2509_26475_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_26475_gb300 import build

    build.build()
    capi.load()
    torch.cuda.set_device(0)


def test_one_step_matches_the_oracle(oracle_mod):
    A_h = wl.adr_operator(100)
    A = api.DeviceCSR.from_host(A_h)
    g = exprk.adr_reaction()
    u0 = wl.adr_initial(100)
    drv = exprk.ExpRK4s6(A, g)
    h = 2.0**-8 * 0.5 / 2
    u1 = drv.step(torch.as_tensor(u0).cuda(), h)
    drv.check()
    assert drv.calls == 4
    prm = api.read_params(drv.params)
    osel = oracle_mod.select(A_h)
    assert abs(prm["s"] - osel["s"]) <= 0.05 * osel["s"]

    def comb(ci):
        W, _ = oracle_mod.solve(A_h, np.stack(ci.V), ci.t, ci.alpha, 2.0**-53, prm["s"], prm["xi"])
        return W

    gu = g(u0)
    hg = h * gu
    U2 = comb(exprk.stage2_inputs(u0, hg, h))[0]
    D2 = g(U2) - gu
    W34 = comb(exprk.stage34_inputs(u0, hg, D2, h))
    D3, D4 = g(W34[0]) - gu, g(W34[1]) - gu
    W56 = comb(exprk.stage56_inputs(u0, hg, D3, D4, h))
    D5, D6 = g(W56[0]) - gu, g(W56[1]) - gu
    ref = comb(exprk.final_inputs(u0, hg, D5, D6, h))[0]
    got = u1.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-12


def test_adr_fourth_order_by_step_halving():
    A_h = wl.adr_operator(100)
    A = api.DeviceCSR.from_host(A_h)
    drv = exprk.ExpRK4s6(A, exprk.adr_reaction())
    u0 = torch.as_tensor(wl.adr_initial(100)).cuda()
    T = 1.0 / 64
    sols = [drv.integrate(u0, 0.0, T, 16 * 2**k) for k in range(4)]
    drv.check()
    diffs = [float((sols[k] - sols[k + 1]).abs().max() / sols[-1].abs().max()) for k in range(3)]
    orders = [math.log2(diffs[k] / diffs[k + 1]) for k in range(2)]
    print("ADR expRK4s6 step-halving differences", diffs, "orders", orders)
    assert all(3.5 <= o <= 4.6 for o in orders), (diffs, orders)


def test_captured_step_replays_the_eager_steps():
    """A step captured as a CUDA graph and replayed gives bit for bit the eager steps."""
    A = api.DeviceCSR.from_host(wl.adr_operator(100))
    drv = exprk.ExpRK4s6(A, exprk.adr_reaction())
    h = 1.0 / 512
    u0 = torch.as_tensor(wl.adr_initial(100)).cuda()
    ue = u0.clone()
    for _ in range(3):
        ue = drv.step(ue, h)
    drv.check()
    ug = u0.clone()
    sg = drv.capture(ug, h)
    sg.replay(3)
    sg.check()
    assert torch.equal(ug, ue)
