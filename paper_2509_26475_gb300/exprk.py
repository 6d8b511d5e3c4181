"""The fourth-order six-stage exponential Runge-Kutta scheme expRK4s6 (Luan; eq. (1.4) of the paper) for
u' = A u + g(u), with every phi-function combination evaluated by Algorithm 3 in four block calls per
step, and Algorithm 1's (s, xi) selected once for A and reused across stages and steps (Section 6).

Stage k of the scheme is u_n + phi_1(c_k h A) c_k h f(u_n) + sum_{j>=2} c_k^j phi_j(c_k h A) b_j with
f(u_n) = A u_n + g(u_n).  Since u_n + phi_1(z) z u_n = phi_0(z) u_n, it is the combination
    w = sum_{j=0}^{p} alpha^j phi_j(t A) v_j,   t = c_k h,  alpha = c_k,
    v_0 = u_n,  v_1 = h g(u_n),  v_j = b_j (j >= 2),
so no product A u_n is needed, and the stage pairs (3, 4) and (5, 6) share one call each, with their
own t_i = c_i h and alpha_i = c_i (the block form decouples the two).

The integrator's own vector arithmetic (g, the increments D_ni and the v_j) is plain elementwise work on
torch tensors, as a caller of the library would write it; every phi-combination runs in the library.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import api

C2, C3, C4, C5, C6 = 0.5, 0.5, 1.0 / 3.0, 5.0 / 6.0, 1.0 / 3.0


@dataclass
class CallInputs:
    """One phi-combination call: rows v_0..v_p, abscissae t_i and weights alpha_i."""

    V: list
    t: list
    alpha: list


def stage2_inputs(u, hg, h):
    """U_n2 = u_n + phi_1(c2 h A) c2 h f(u_n)."""
    return CallInputs([u, hg], [C2 * h], [C2])


def stage34_inputs(u, hg, D2, h):
    """U_nk = u_n + phi_1(c_k h A) c_k h f(u_n) + phi_2(c_k h A) (c_k^2 / c2) h D_n2, k = 3, 4."""
    return CallInputs([u, hg, (h / C2) * D2], [C3 * h, C4 * h], [C3, C4])


def stage56_inputs(u, hg, D3, D4, h):
    """U_nj, j = 5, 6: the phi_2 and phi_3 terms built from D_n3 and D_n4."""
    b2 = (h / (C3 - C4)) * (-(C4 / C3) * D3 + (C3 / C4) * D4)
    b3 = (2.0 * h / (C3 - C4)) * (D3 / C3 - D4 / C4)
    return CallInputs([u, hg, b2, b3], [C5 * h, C6 * h], [C5, C6])


def final_inputs(u, hg, D5, D6, h):
    """u_{n+1}: the phi_2 and phi_3 terms built from D_n5 and D_n6, at t = h with weight 1."""
    b2 = (h / (C5 - C6)) * (-(C6 / C5) * D5 + (C5 / C6) * D6)
    b3 = (2.0 * h / (C5 - C6)) * (D5 / C5 - D6 / C6)
    return CallInputs([u, hg, b2, b3], [h], [1.0])


class ExpRK4s6:
    """expRK4s6 on the GPU for u' = A u + g(u) (g autonomous, elementwise or not; a callable on CUDA
    tensors).  ``tol`` is the truncation tolerance of every phi-combination (2^-53 for FP64 accuracy)."""

    def __init__(self, A: api.DeviceCSR, g, tol: float = 2.0**-53, params=None, stream=None):
        self.A, self.g, self.tol, self.stream = A, g, float(tol), stream
        self.params = params if params is not None else api.select_params(A, tol=self.tol, stream=stream)
        self.calls = 0
        self.stats = []

    def _combine(self, ci: CallInputs):
        V = torch.stack(ci.V).contiguous()
        W, st = api.solve(self.A, V, ci.t, ci.alpha, self.tol, self.params, stream=self.stream)
        self.calls += 1
        self.stats.append(st)
        return W

    def step(self, u: torch.Tensor, h: float) -> torch.Tensor:
        g = self.g
        gu = g(u)
        hg = h * gu
        U2 = self._combine(stage2_inputs(u, hg, h))[0]
        D2 = g(U2) - gu
        W34 = self._combine(stage34_inputs(u, hg, D2, h))
        D3, D4 = g(W34[0]) - gu, g(W34[1]) - gu
        W56 = self._combine(stage56_inputs(u, hg, D3, D4, h))
        D5, D6 = g(W56[0]) - gu, g(W56[1]) - gu
        return self._combine(final_inputs(u, hg, D5, D6, h))[0]

    def integrate(self, u0: torch.Tensor, t0: float, t1: float, steps: int) -> torch.Tensor:
        h = (t1 - t0) / steps
        u = u0
        for _ in range(steps):
            u = self.step(u, h)
        return u

    def check(self):
        """Synchronises and raises if any call reported a device status."""
        torch.cuda.synchronize()
        _check_stats(self.stats)
        self.stats.clear()

    def capture(self, u: torch.Tensor, h: float) -> "StepGraph":
        """Records one step of size h on the device vector u as a CUDA graph: each replay of the result
        advances u in place (u <- step(u)) with the four phi-combination launches, the reaction terms and
        the copy back into u, and no host work per step beyond the replay call.  (s, xi), t and alpha
        are fixed at capture."""
        cur = torch.cuda.current_stream(u.device)
        side = torch.cuda.Stream(device=u.device)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            self.step(u.clone(), h)  # warm-up outside the capture: workspaces and allocator state
            side.synchronize()
            self.check()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                u.copy_(self.step(u, h))
        cur.wait_stream(side)
        stats, self.stats = self.stats, []
        return StepGraph(g, stats)


class StepGraph:
    """A captured expRK4s6 step (ExpRK4s6.capture)."""

    def __init__(self, graph, stats):
        self.graph, self.stats = graph, stats

    def replay(self, steps: int = 1):
        for _ in range(steps):
            self.graph.replay()

    def check(self):
        """Synchronises and raises if a call of the last replay reported a device status."""
        torch.cuda.synchronize()
        _check_stats(self.stats)


def _check_stats(stats):
    for st in stats:
        s = api.read_stats(st)["status"]
        if s != 0:
            from . import capi

            capi.check(s, "expRK4s6 stage")


def adr_reaction(gamma: float = 1000.0):
    """g(u) = gamma u (u - 1/2) (1 - u), the reaction of the paper's ADR problem."""

    def g(u):
        return gamma * u * (u - 0.5) * (1.0 - u)

    return g
