#!/usr/bin/env python3
"""Benchmark of the phi-combination solver on one GB300 (or N replicas under torchrun).

Default workload (the precision configuration): 2-D first-order upwind advection-diffusion on a 1024 x 1024
Dirichlet grid (n = 1,048,576, nnz = 5,238,784, Peclet 1e3, stiff and highly nonnormal), p = 4, r = 4,
t = (1/4, 1/2, 3/4, 1) h, alpha = 1, h in {1e-5, 1e-4}, v_j ~ N(0,1) (seed 3), FP64 at tol = 2^-53.

One step = Algorithm 1 (shift/scaling) on A + Algorithm 3 at h = 1e-5 + Algorithm 3 at h = 1e-4, so a step
is 2 solves; value = solves/s over all ranks.  Inputs are resident in HBM before the timed region; L2 is
flushed (a 2 x L2 write) between timed steps, outside the per-step CUDA events (the working set, about
1.4 GB, exceeds L2 anyway).  The line also carries:
  * ``roofline`` of the dominant kernel (the recovery at h = 1e-4) against the FP64 FMA rate measured by the
    library's probe kernel just before the timed region, with its HBM view;
  * ``kernels``: every kernel's share of the step, and Algorithm 1's kernel against HBM;
  * ``fp32``: the same step at tol 2^-24 with FP32 storage (its own value, HBM roofline and errors);
  * ``e2e`` through the public API from pinned host buffers;
  * ``cpu_baseline``: the FP64 C oracle on the host cores (Algorithm 1 + Algorithm 3 at h = 1e-5), whose
    result also gives the errors of both precisions at h = 1e-5.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload NAME] [--precision f64|f32|mixed] [--sweep]

``--sweep`` runs the 1024^2 workload at h = 1e-5 .. 1e-1 in both precisions (one solve each) and prints one
JSON line per (precision, h).  ``--impl reference`` times the CPU oracle (plain FP64 C, OpenMP over
sparse-product rows) on a bounded sample of the same workload on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "φ-comb solves/s & SpMM HBM GB/s (% peak) at stated tol; p50/p99 serve latency"
SMS = 152  # streaming multiprocessors of a GB300
# FP64 pipe of a GB300 SM by its unit count: 2 FMA/clk, 152 SMs, 2070 MHz maximum SM clock; 2 flops an FMA.
# Context only: the roofline divides by the rate the probe kernel measures.
FP64_DERIVED_GFLOPS = 2.0 * 2.0 * SMS * 2.070

# Single-operator workloads: the default (advdiff2d-1024) and the expRK4s6-shaped 64^3 block.
WORKLOADS = {
    "advdiff2d-1024": dict(hs=(1e-5, 1e-4), p=4, r=4, t=lambda h: [0.25 * h, 0.5 * h, 0.75 * h, h],
                           name="advdiff2d-1024^2 Pe1e3 (n=1048576) p=4 r=4 t=(1/4,1/2,3/4,1)h alpha=1 h={1e-5,1e-4}"),
    "convdiff3d-64": dict(hs=(1e-4, 1e-2), p=3, r=2, t=lambda h: [h / 2.0, h / 3.0],
                          name="convdiff3d-64^3 Pe10 (n=262144) p=3 r=2 t=(h/2,h/3) alpha=(1/2,1/3) h={1e-4,1e-2}"),
}
SWEEP_HS = (1e-5, 1e-4, 1e-3, 1e-2, 1e-1)
SERVE_CURVE_RATES = (100.0, 200.0, 400.0, 700.0, 1000.0, 1500.0)
WORKLOAD = "advdiff2d-1024"
PRECISION = "f64"
HS = WORKLOADS[WORKLOAD]["hs"]
TOL = 2.0**-53
P, R = 4, 4
WORKLOAD_NAME = WORKLOADS[WORKLOAD]["name"] + " tol=2^-53 FP64"


def tol_of(precision: str) -> float:
    return 2.0**-53 if precision == "f64" else 2.0**-24


def configure(workload_name: str, precision: str):
    """Select the workload and storage precision (f64: tol 2^-53; f32: tol 2^-24)."""
    global WORKLOAD, PRECISION, HS, TOL, P, R, WORKLOAD_NAME
    if workload_name not in WORKLOADS:
        WORKLOAD, PRECISION = workload_name, precision
        return
    if precision == "mixed":
        raise SystemExit("--precision mixed applies to the batch512 and serve workloads")
    cfg = WORKLOADS[workload_name]
    WORKLOAD, PRECISION = workload_name, precision
    HS, P, R = cfg["hs"], cfg["p"], cfg["r"]
    TOL = tol_of(precision)
    WORKLOAD_NAME = workload_label(precision)


def workload_label(precision: str) -> str:
    return WORKLOADS[WORKLOAD]["name"] + (" tol=2^-53 FP64" if precision == "f64" else " tol=2^-24 FP32")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-companion", action="store_true", help="skip the FP32 companion of the default line")
    ap.add_argument("--sweep", action="store_true", help="advdiff2d-1024: h = 1e-5 .. 1e-1 in FP64 and FP32")
    ap.add_argument("--function-operator", action="store_true",
                    help="the step through the operator-function path (phic_fn_*, the library's CSR product as "
                         "the function): Algorithm 1 on the host with device passes, Algorithm 3 as a CUDA graph")
    ap.add_argument("--workload", default="advdiff2d-1024",
                    choices=sorted(WORKLOADS) + ["batch512", "serve", "exprk-adr", "lowrank-m2"])
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "mixed"])
    ap.add_argument("--requests", type=int, default=1000, help="serve: number of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--no-tune", action="store_true", help="batch512: skip the autotuner (default shape)")
    ap.add_argument("--profile-batch", type=int, default=None, metavar="COUNT",
                    help="profiler target: the first COUNT instances of batch512 in one batched launch (twice, "
                         "default shape), no timing and no JSON line")
    ap.add_argument("--profile-solve", type=float, default=None, metavar="H",
                    help="profiler target: Algorithm 1 and two Algorithm 3 solves of the workload at step H, "
                         "no timing and no JSON line")
    return ap.parse_args()


def profile_solve(h: float) -> int:
    """A fixed, short launch sequence for profilers: select_kernel once, then series_kernel and
    recover_kernel twice for the benchmark workload at step h."""
    import torch

    from paper_2509_26475_gb300 import api

    A_h, V_h, alpha = workload()
    A = api.DeviceCSR.from_host(A_h, dtype=torch_dtype())
    V = torch.as_tensor(V_h).to(torch_dtype()).cuda()
    P = api.select_params(A, tol=TOL, check=True)
    for _ in range(2):
        W, st = api.solve(A, V, t_of(h), alpha, TOL, P, check=True)
    print(api.read_stats(st))
    return 0


def profile_batch(count: int) -> int:
    """A short launch sequence for profilers: the first `count` instances of the batching workload (each
    Algorithm 1 + 3), one batched launch twice at 4096 rows per CTA and 3 blocks per SM."""
    import torch

    from paper_2509_26475_gb300 import api

    insts = batch_workload("mixed")[:max(1, count)]
    items = []
    for x in insts:
        dt = torch.float32 if x["prec"] == "f32" else torch.float64
        A = api.DeviceCSR.from_host(x["A"], dtype=dt)
        items.append(api.BatchItem(A, torch.as_tensor(x["V"]).to(dt).cuda(), x["t"], x["alpha"], tol=x["tol"],
                                   select=True))
    b = api.Batch(items, config={"rows_per_cta": 4096, "blocks_per_sm": 3})
    for _ in range(2):
        b.launch()
    torch.cuda.synchronize()
    bad = [i for i, st in enumerate(b.stats()) if st["status"] != 0]
    print({"rows": sum(x["A"].n for x in insts), "bad": bad, **b.info()})
    return 1 if bad else 0


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload():
    from paper_2509_26475_gb300 import workloads as wl

    if WORKLOAD == "convdiff3d-64":
        w = wl.workload_convdiff3d_64(HS[0])
    else:
        w = wl.workload_advdiff2d_1024(HS[0], TOL)
    return w["A"], w["V"], w["alpha"]


def t_of(h):
    return WORKLOADS[WORKLOAD]["t"](h)


def torch_dtype(precision: str | None = None):
    import torch

    return torch.float64 if (precision or PRECISION) == "f64" else torch.float32


TRAFFIC_RECORDS = {("convdiff3d-64", "f64"): "recover_kernel_convdiff3d_64.json",
                   ("advdiff2d-1024", "f32"): "recover_kernel_advdiff2d_1024_fp32.json",
                   ("advdiff2d-1024", "f64"): "recover_kernel_advdiff2d_1024_fp64.json"}


def recorded_traffic(terms: int, precision: str | None = None):
    """DRAM bytes of one launch of the dominant kernel from the committed ncu record of this workload and
    precision, if that record was taken on the current kernel sources (sha256 of each); None otherwise.
    A record of a shorter launch of the same kernel (fewer Taylor terms) is scaled by the terms: every
    term moves the same bytes once the working set exceeds L2, which is when the scaling is used."""
    import hashlib

    name = TRAFFIC_RECORDS.get((WORKLOAD, precision or PRECISION))
    if name is None:
        return None
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", name)))
        for path, sha in rec["sources"].items():  # every file that defines the kernel, as captured
            if hashlib.sha256(open(os.path.join(ROOT, path), "rb").read()).hexdigest() != sha:
                return None
        b = float(rec["dram_bytes_per_launch"])
        if "terms_per_launch" in rec:
            b *= terms / float(rec["terms_per_launch"])
        return b
    except Exception:
        return None


def reduce_max_over_ranks(x: float, dist, device) -> float:
    """Maximum of a per-rank number over all ranks (the slowest rank sets the job time)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def solves_per_second(ms_per_step: float, world: int) -> float:
    """Whole-job throughput: every rank runs its own replica of the step (len(HS) solves)."""
    return world * len(HS) / (ms_per_step / 1000.0)


def rel_errors(W, ref):
    """Relative 2-norm error of each combination w_i (rows of W) against ref."""
    import numpy as np

    W = np.asarray(W, dtype=np.float64)
    return [float(np.linalg.norm(W[i] - ref[i]) / np.linalg.norm(ref[i])) for i in range(ref.shape[0])]


# ------------------------------------------------------------------------------------------------
# Oracle timing (CPU)
# ------------------------------------------------------------------------------------------------
def oracle_sample_hs():
    """The solves of a step the oracle runs as its sample: the whole step on the 64^3 workload (about 3 s
    on 16 Grace cores); on the 1024^2 workload only h = 1e-5 (about 20 s with Algorithm 1), since the
    h = 1e-4 solve takes about 9 times the recovery work."""
    return tuple(HS) if WORKLOAD == "convdiff3d-64" else (HS[0],)


def oracle_sample_text(hs) -> str:
    if len(hs) == len(HS):
        return ("Algorithm 1 + Algorithm 3 at h = " + " and ".join(f"{h:g}" for h in hs) +
                ": one full step of the workload, FP64 C oracle, OpenMP over sparse-product rows")
    return (f"Algorithm 1 + Algorithm 3 at h = {hs[0]:g} only (one of the step's {len(HS)} solves, the cheaper: "
            f"h = {HS[-1]:g} has about 9 times its recovery terms), FP64 C oracle, OpenMP over sparse-product "
            "rows; value = solves of the sample / its time, so it overstates the oracle's rate on the full step")


def time_oracle_sample(A, V, alpha):
    """One run of the oracle's sample: Algorithm 1 (its own xi, s), then Algorithm 3 at each sampled h.
    Returns (seconds, {h: W}, threads, selection)."""
    import oracle

    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    hs = oracle_sample_hs()
    t0 = time.perf_counter()
    sel = oracle.select(A)
    out = {}
    for h in hs:
        out[h], _ = oracle.solve(A, V, t_of(h), alpha, 2.0**-53, sel["s"], sel["xi"])
    return time.perf_counter() - t0, out, cores, sel


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    if WORKLOAD in ("batch512", "serve"):
        return run_reference_fleet(args)
    if WORKLOAD == "exprk-adr":
        return run_reference_exprk(args)
    if WORKLOAD == "lowrank-m2":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle takes dense or CSR operators; the dense "
                          "form of the 400,000-row low-rank operator (1.3 TB) does not fit"}), flush=True)
        return 0
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    # bound the whole run to a few minutes: each step is the oracle's sample of the workload
    cap = 6 if WORKLOAD == "convdiff3d-64" else 3
    steps_run, warm_run = min(steps, cap), min(warmup, 1 if WORKLOAD == "convdiff3d-64" else 0)
    A, V, alpha = workload()
    hs = oracle_sample_hs()
    for _ in range(warm_run):
        time_oracle_sample(A, V, alpha)
    times = []
    cores = 0
    for _ in range(steps_run):
        sec, _, cores, _ = time_oracle_sample(A, V, alpha)
        times.append(sec)
    ms = 1000.0 * statistics.mean(times)
    value = len(hs) / (ms / 1000.0)
    sample = oracle_sample_text(hs) + f"; {steps_run} timed step(s) after {warm_run} warm-up (asked {steps}/{warmup})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": steps_run, "warmup": warm_run, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label("f64"), "device": "host CPU", "threads": cores,
                       "solves_per_step": len(hs)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None):
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"phic_clocks_rank{gpu_index}_{os.getpid()}.csv")
        self.gpu_index = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            # the timed region starts once sampling runs (nvidia-smi takes a moment to start)
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ------------------------------------------------------------------------------------------------
# Native run
# ------------------------------------------------------------------------------------------------
def recover_kernel_work(n, nnz, wf, p, r, terms, outer_steps, b=8):
    """Algorithmic FP64 flops (an FMA counts 2) and bytes of one recovery-kernel launch.

    Per Taylor term (n x wf block, wf = 2r): the product with A_1 = A - xi I takes 2 nnz flops per
    column, and the column scale, the accumulation E <- E + F and the norm about 3 n more:
    (2 nnz + 3 n) wf.  Per recovery step the refresh E mu + S Jt costs about (1 + p) n wf.  Bytes per term:
    CSR values and indices ((4 + b) nnz + 4(n+1)) plus reading F, reading and writing E and writing the
    next F (4 n wf b), with b the bytes of a value (8 in FP64, 4 in FP32)."""
    flops = terms * (2 * nnz + 3 * n) * wf + outer_steps * (1 + p) * n * wf
    bytes_ = terms * ((4 + b) * nnz + 4 * (n + 1) + 4 * n * wf * b)
    return flops, bytes_


def select_kernel_flops(n, nnz, m, evals):
    """Algorithmic FP64 flops of one Algorithm 1 launch (an FMA counts 2): m sparse products (2 nnz), one
    sum of squares per pass (2 n, m + 2 passes besides the evaluations), and per objective evaluation the
    combination sum_k binom(m,k) z^(m-k) V_k (2 (m+1) n) and its sum of squares (2 n)."""
    return m * 2 * nnz + (m + 2) * 2 * n + evals * (2 * (m + 1) * n + 2 * n)


def select_kernel_bytes(n, nnz, m, r_guard, evals, b=8):
    """Algorithmic bytes of one Algorithm 1 launch: m sparse matrix-vector products (the guarded chain to
    r and the extension to m), each reading the operator ((4 + b) nnz + 4(n+1)) and one basis vector and
    writing the next (16 n); the rescaling V_j <- V_j / s0^j (16 n r); and one pass over the basis V_0..V_m
    per objective evaluation ((m+1) 8 n)."""
    spmv = (4 + b) * nnz + 4 * (n + 1) + 16 * n
    return m * spmv + 16 * n * r_guard + evals * (m + 1) * 8 * n


def measure_fp64_roof(lib, capi, dev, local_rank):
    """FP64 FMA throughput of this GPU: the library's probe kernel (8 independent FMA chains per thread,
    4 blocks of 256 threads per SM, no memory traffic), timed with CUDA events on the stream it runs on,
    median of 8 launches of about 50 ms, SM clocks sampled meanwhile."""
    import ctypes

    import torch

    stream = torch.cuda.current_stream(dev)
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    fmas = ctypes.c_int64(0)

    def timed(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        capi.check(lib.phic_probe_fp64_fma(int(iters), sink.data_ptr(), ctypes.byref(fmas), stream.cuda_stream),
                   "phic_probe_fp64_fma")
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    timed(2000)
    ms = timed(20000)
    iters = max(1000, int(20000 * 50.0 / max(ms, 1e-3)))
    with ClockSampler(local_rank, None) as clk:
        times = [timed(iters) for _ in range(8)]
    t = statistics.median(times) / 1000.0
    gflops = 2.0 * fmas.value / t / 1e9
    cs = clk.summary() or {}
    mhz = cs.get("sm_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return {"gflops": gflops, "fma_per_clk_per_sm": fmas.value / t / (sms * mhz * 1e6), "sm_mhz": mhz,
            "launch_ms": 1000.0 * t, "fmas_per_launch": int(fmas.value), "clocks": cs,
            "derived_gflops": 2.0 * 2.0 * sms * (cs.get("sm_max_mhz") or 2070.0) / 1000.0,
            "how": "phic_probe_fp64_fma: 8 independent FMA chains per thread, 4 x 256 threads per SM, median "
                   "of 8 launches, CUDA events"}


class SingleRun:
    """Algorithm 1 + Algorithm 3 at each h of the workload, in one precision, on resident inputs: the
    step of the benchmark line.  Events between the phases give every kernel's time."""

    def __init__(self, api, capi, precision, dev, A_h, V_h, alpha):
        import torch

        self.api, self.capi, self.precision, self.dev = api, capi, precision, dev
        self.tol = tol_of(precision)
        self.alpha = alpha
        dt = torch_dtype(precision)
        self.prec = capi.PHIC_F64 if precision == "f64" else capi.PHIC_F32
        self.A = api.DeviceCSR.from_host(A_h, device=dev, dtype=dt)
        self.V = torch.as_tensor(V_h).to(dt).to(dev)
        n, nnz = self.A.n, self.A.nnz
        self.params = api.new_params(dev)
        self.stats = [api.new_stats(dev) for _ in HS]
        self.W = [torch.empty((R, n), dtype=dt, device=dev) for _ in HS]
        self.ws_sel = torch.empty(api.select_workspace_bytes(n), dtype=torch.uint8, device=dev)
        self.ws_sol = torch.empty(api.solve_workspace_bytes(n, nnz, P, R, self.prec), dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream(dev)

    def step(self, evs=None):
        """evs: None or 1 + 2 len(HS) events, recorded after select and after each series and recovery."""
        api, capi = self.api, self.capi
        api.select_params(self.A, tol=self.tol, out=self.params, workspace=self.ws_sel)
        if evs is not None:
            evs[0].record(self.stream)
        for idx, h in enumerate(HS):
            for ph, flag in enumerate((capi.PHIC_PHASE_SERIES, capi.PHIC_PHASE_RECOVER)):
                api.solve(self.A, self.V, t_of(h), self.alpha, self.tol, self.params, out=self.W[idx],
                          stats=self.stats[idx], workspace=self.ws_sol, flags=flag)
                if evs is not None:
                    evs[1 + 2 * idx + ph].record(self.stream)

    def check_status(self):
        import torch

        torch.cuda.synchronize(self.dev)
        self.capi.check(self.api.read_params(self.params)["status"], "select (device)")
        for st in self.stats:
            self.capi.check(self.api.read_stats(st)["status"], "solve (device)")

    def timed(self, K, warmup, lib, local_rank, dist):
        """W warm-up steps, then K steps each bracketed by CUDA events (per phase), an L2 flush (2 x L2
        write) before each step outside its events; barrier + synchronize on both sides."""
        import torch

        for _ in range(max(warmup, 0)):
            self.step()
        self.check_status()
        l2 = torch.cuda.get_device_properties(self.dev).L2_cache_size
        flush = torch.empty(2 * l2, dtype=torch.uint8, device=self.dev)
        nph = 1 + 2 * len(HS)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        evp = [[torch.cuda.Event(enable_timing=True) for _ in range(nph)] for _ in range(K)]
        launches0 = lib.phic_launch_count()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(self.dev)
        wall0 = time.perf_counter()
        with ClockSampler(local_rank, None) as clk:
            for k in range(K):
                flush.fill_(k & 0xFF)
                ev0[k].record(self.stream)
                self.step(evp[k])
            torch.cuda.synchronize(self.dev)
        wall = time.perf_counter() - wall0
        if dist is not None:
            dist.barrier()
        self.launches = lib.phic_launch_count() - launches0
        self.check_status()
        self.wall = wall
        self.clocks = clk.summary()
        self.step_ms = [ev0[k].elapsed_time(evp[k][-1]) for k in range(K)]
        phase_ms = []
        for k in range(K):
            prev = ev0[k]
            row = []
            for e in evp[k]:
                row.append(prev.elapsed_time(e))
                prev = e
            phase_ms.append(row)
        self.phase_ms = [statistics.mean(col) for col in zip(*phase_ms)]
        self.sts = [self.api.read_stats(s) for s in self.stats]
        self.prm = self.api.read_params(self.params)
        return statistics.mean(self.step_ms)

    def kernels(self, hbm_peak, roof=None):
        """Per-kernel time in the step and share; Algorithm 1's kernel against the FP64 roof and HBM."""
        n, nnz = self.A.n, self.A.nnz
        out = {"select_kernel": {"ms": self.phase_ms[0]}}
        for idx, h in enumerate(HS):
            out[f"series_kernel h={h:g}"] = {"ms": self.phase_ms[1 + 2 * idx],
                                             "terms": self.sts[idx]["series_terms"]}
            out[f"recover_kernel h={h:g}"] = {"ms": self.phase_ms[2 + 2 * idx],
                                              "terms": self.sts[idx]["recovery_terms"],
                                              "us_per_term": 1000.0 * self.phase_ms[2 + 2 * idx] /
                                              max(1, self.sts[idx]["recovery_terms"])}
        tot = sum(v["ms"] for v in out.values())
        for v in out.values():
            v["share"] = v["ms"] / tot if tot > 0 else None
        b = 8 if self.precision == "f64" else 4
        sb = select_kernel_bytes(n, nnz, 61, self.prm["r"], self.prm["evals"], b)
        sf = select_kernel_flops(n, nnz, 61, self.prm["evals"])
        sel_s = self.phase_ms[0] / 1000.0
        gbs = sb / sel_s / 1e9
        out["select_kernel"].update({"evals": self.prm["evals"], "r": self.prm["r"], "bytes": sb, "flops": sf,
                                     "fp64_gflops": sf / sel_s / 1e9,
                                     "fp64_frac": (sf / sel_s / 1e9 / roof["gflops"]) if roof else None,
                                     "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                                     "bound": "alu (each objective pass is (m+1) FMAs per 8 (m+1) bytes, above "
                                              "the FP64/HBM balance of a GB300)",
                                     "bytes_note": "m products ((4+b) nnz + 4(n+1) + 16n each), the rescaling "
                                                   "(16 n r) and one pass over V_0..V_m per objective "
                                                   "evaluation ((m+1) 8 n); of measured HBM"})
        return out

    def roofline(self, roof, hbm_peak):
        """The dominant kernel: the recovery at the largest h."""
        n, nnz = self.A.n, self.A.nnz
        st = self.sts[-1]
        b = 8 if self.precision == "f64" else 4
        flops, bytes_ = recover_kernel_work(n, nnz, 2 * R, P, R, st["recovery_terms"], st["s_int"] - 1, b)
        rec_s = self.phase_ms[-1] / 1000.0
        achieved = flops / rec_s / 1e9
        hbm_gbs = bytes_ / rec_s / 1e9
        kernel = f"recover_kernel (Algorithm 3 recovery loop, h={HS[-1]:g})"
        common = {"kernel": kernel, "traffic": recorded_traffic(st["recovery_terms"], self.precision),
                  "launch_ms": self.phase_ms[-1], "terms_per_launch": st["recovery_terms"],
                  "bytes_per_launch": bytes_, "flops_per_launch": flops}
        if self.precision == "f64" and roof is not None:
            return {"bound": "alu", "achieved": achieved, "peak": roof["gflops"], "unit": "FP64 GFLOP/s",
                    "frac": achieved / roof["gflops"], **common,
                    "peak_note": f"of measured: FP64 FMA rate of the probe kernel before the timed region "
                                 f"({roof['fma_per_clk_per_sm']:.3f} FMA/clk/SM at {roof['sm_mhz']:.0f} MHz); "
                                 "achieved counts (2 nnz + 3 n) 2r flops per Taylor term",
                    "peak_derived": roof["derived_gflops"], "frac_of_derived": achieved / roof["derived_gflops"],
                    "hbm_view": {"algorithmic_gbs": hbm_gbs, "peak_gbs": hbm_peak,
                                 "frac_of_measured": hbm_gbs / hbm_peak}}
        return {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
                **common, "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, of measured); algorithmic bytes "
                                       "(4+b) nnz + 4(n+1) + 4 n 2r b per Taylor term, which count every tile "
                                       "pass as DRAM traffic: a fraction above 1 means L2 and shared memory "
                                       "hold part of them (compare `traffic`, the DRAM bytes ncu measured)"}

    def summary(self):
        return {"s": self.prm["s"], "xi": self.prm["xi"], "s_int": [x["s_int"] for x in self.sts],
                "terms": [x["series_terms"] + x["recovery_terms"] for x in self.sts]}

    def release(self):
        for name in ("A", "V", "W", "ws_sel", "ws_sol", "params", "stats"):
            setattr(self, name, None)


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    configure(args.workload, args.precision)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.profile_solve is not None:
        return profile_solve(args.profile_solve)
    if args.profile_batch is not None:
        return profile_batch(args.profile_batch)
    if WORKLOAD == "batch512":
        return run_batch(args, rank, world, local_rank)
    if WORKLOAD == "serve":
        return run_serve(args, rank, world, local_rank)
    if WORKLOAD == "exprk-adr":
        return run_exprk(args, rank, world, local_rank)
    if WORKLOAD == "lowrank-m2":
        return run_lowrank(args, rank, world, local_rank)
    if args.sweep:
        return run_sweep(args, rank, world, local_rank)
    if args.function_operator:
        return run_function_operator(args, rank, world, local_rank)
    return run_single(args, rank, world, local_rank)


def run_function_operator(args, rank, world, local_rank):
    """The default step with A given as a function (phic_fn_select_params + phic_fn_solve, the product by
    phic_csr_apply): Algorithm 1 runs its products on the stream and its guard and Brent's method on the host;
    each Algorithm 3 is one CUDA graph with conditional WHILE nodes.  Times per solve with CUDA events;
    the graph's construction (stream capture and instantiation) is inside the timed region."""
    import torch

    from paper_2509_26475_gb300 import api, build, capi

    if world > 1:
        raise SystemExit("--function-operator runs on one GPU")
    build.build()
    lib = capi.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    A_h, V_h, alpha = workload()
    dt = torch_dtype()
    F = api.FunctionOperator.from_csr(api.DeviceCSR.from_host(A_h, device=dev, dtype=dt))
    V = torch.as_tensor(V_h).to(dt).to(dev)
    flush = torch.empty(2 * torch.cuda.get_device_properties(dev).L2_cache_size, dtype=torch.uint8, device=dev)

    def step(evs=None):
        P = api.select_params(F, tol=TOL)
        if evs is not None:
            evs[1].record(stream)
        sts = []
        for idx, h in enumerate(HS):
            sts.append(api.solve(F, V, t_of(h), alpha, TOL, P)[1])
            if evs is not None:
                evs[2 + idx].record(stream)
        return P, sts

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    K = max(1, args.steps)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2 + len(HS))] for _ in range(K)]
    l0 = lib.phic_launch_count()
    with ClockSampler(local_rank, None) as clk:
        w0 = time.perf_counter()
        for k in range(K):
            flush.fill_(k & 255)
            evs[k][0].record(stream)
            P, sts = step(evs[k])
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - w0
    st = [api.read_stats(x) for x in sts]
    if any(x["status"] != 0 for x in st) or api.read_params(P)["status"] != 0:
        raise SystemExit("function operator: a device status was reported; no number is reported")
    ms = statistics.mean(e[0].elapsed_time(e[-1]) for e in evs)
    sel_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    solve_ms = [statistics.mean(e[1 + i].elapsed_time(e[2 + i]) for e in evs) for i in range(len(HS))]
    terms = [x["series_terms"] + x["recovery_terms"] for x in st]
    line = {"metric": METRIC, "value": len(HS) * 1000.0 / ms, "unit": "solves/s", "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": PRECISION, "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME + " through the operator-function path (phic_fn_*, phic_csr_apply)",
                       "select_ms": sel_ms, "solve_ms": solve_ms, "terms": terms,
                       "us_per_term": [1000.0 * m / t for m, t in zip(solve_ms, terms)],
                       "s_int": [x["s_int"] for x in st], "l2": "flushed between steps", "parallelism": "x1"},
            "roofline": None, "gpu_launches": int(lib.phic_launch_count() - l0), "wall_s_timed_region": wall}
    cs = clk.summary()
    if cs:
        line["clocks"] = cs
    print(json.dumps(line), flush=True)
    return 0


def run_single(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2509_26475_gb300 import api, build, capi

    build.build()
    lib = capi.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    hbm_peak = float(_peaks().get("hbm_gbs", 6800.0))
    roof = measure_fp64_roof(lib, capi, dev, local_rank)

    A_h, V_h, alpha = workload()
    K = max(1, args.steps)
    run = SingleRun(api, capi, PRECISION, dev, A_h, V_h, alpha)
    ms = reduce_max_over_ranks(run.timed(K, args.warmup, lib, local_rank, dist), dist, dev)
    value = solves_per_second(ms, world)
    n, nnz = run.A.n, run.A.nnz
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": PRECISION, "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "n": n, "nnz": nnz, "p": P, "r": R, "h": list(HS),
                       "tol": "2^-53" if PRECISION == "f64" else "2^-24",
                       "step": "Algorithm 1 + Algorithm 3 at each h (2 solves)",
                       "l2": "flushed between steps (2 x L2 write, outside the step events); working set above L2",
                       "parallelism": f"replicas x{world}", **run.summary()},
            "roofline": run.roofline(roof, hbm_peak), "kernels": run.kernels(hbm_peak, roof),
            "fp64_roof": roof, "gpu_launches": int(run.launches), "wall_s_timed_region": run.wall}
    if run.clocks:
        line["clocks"] = run.clocks
    W_primary = [w.double().cpu().numpy() for w in run.W]
    run.release()
    torch.cuda.empty_cache()

    # FP32 companion: the same step at tol 2^-24 with FP32 storage
    comp = None
    if WORKLOAD == "advdiff2d-1024" and PRECISION == "f64" and not args.no_companion:
        c32 = SingleRun(api, capi, "f32", dev, A_h, V_h, alpha)
        ms32 = reduce_max_over_ranks(c32.timed(K, args.warmup, lib, local_rank, dist), dist, dev)
        W32 = [w.double().cpu().numpy() for w in c32.W]
        comp = {"value": solves_per_second(ms32, world), "unit": "solves/s", "ms_per_step": ms32, "dtype": "f32",
                "tol": "2^-24", "workload": workload_label("f32"), **c32.summary(),
                "roofline": c32.roofline(None, hbm_peak), "kernels": c32.kernels(hbm_peak, roof),
                "gpu_launches": int(c32.launches), "clocks": c32.clocks,
                "errors": {f"h={HS[-1]:g} vs GPU FP64 (same step)": max(rel_errors(W32[-1], W_primary[-1]))}}
        line["fp32"] = comp
        c32.release()
        torch.cuda.empty_cache()

    if not args.no_e2e:
        line["e2e"] = e2e(api, capi, A_h, V_h, alpha, dev, torch.cuda.current_stream(dev), K, world, dist)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sec, ref, cores, sel = time_oracle_sample(A_h, V_h, alpha)
        hs = oracle_sample_hs()
        line["cpu_baseline"] = {"value": len(hs) / sec, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                "sample": oracle_sample_text(hs), "seconds": sec}
        errs = {}
        for idx, h in enumerate(HS):
            if h in ref:
                errs[f"h={h:g} vs FP64 oracle"] = max(rel_errors(W_primary[idx], ref[h]))
                if comp is not None:
                    comp["errors"][f"h={h:g} vs FP64 oracle"] = max(rel_errors(W32[idx], ref[h]))
        line["errors"] = {"metric": "max over i of ||w_i - w_i_ref||_2 / ||w_i_ref||_2", **errs,
                          "oracle_s": sel["s"], "oracle_xi": sel["xi"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def e2e(api, capi, A_h, V_h, alpha, dev, stream, K, world, dist):
    """Same step through the public API from pinned host buffers: copy A and V in, Algorithm 1, both
    solves, copy the results out; CUDA events around everything."""
    import torch

    dt = torch_dtype()
    rp = torch.as_tensor(A_h.rowptr).pin_memory()
    ci = torch.as_tensor(A_h.colidx).pin_memory()
    va = torch.as_tensor(A_h.values).to(dt).pin_memory()
    Vp = torch.as_tensor(V_h).to(dt).pin_memory()
    outs = [torch.empty((R, A_h.n), dtype=dt).pin_memory() for _ in HS]
    h2d = rp.numel() * 4 + ci.numel() * 4 + va.numel() * va.element_size() + Vp.numel() * Vp.element_size()
    d2h = sum(o.numel() * o.element_size() for o in outs)

    def one():
        A = api.DeviceCSR(rp.to(dev, non_blocking=True), ci.to(dev, non_blocking=True), va.to(dev, non_blocking=True))
        V = Vp.to(dev, non_blocking=True)
        Pm = api.select_params(A, tol=TOL)
        for idx, h in enumerate(HS):
            Wd, _ = api.solve(A, V, t_of(h), alpha, TOL, Pm)
            outs[idx].copy_(Wd, non_blocking=True)

    one()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(K):
        one()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = reduce_max_over_ranks(e0.elapsed_time(e1) / K, dist, dev)
    return {"value": solves_per_second(ms, world), "unit": "solves/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def golden_samples(h: float):
    """The oracle's sampled answer at step h for the 1024^2 workload (tests/golden/advdiff2d_1024_h<h>.json,
    written by tests/golden/make_advdiff2d_1024.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"advdiff2d_1024_h{h:g}.json")
    return json.load(open(path)) if os.path.exists(path) else None


def sampled_error(W, gold) -> float:
    """Largest relative 2-norm error over the combinations, on the oracle's sampled entries."""
    import numpy as np

    idx = np.asarray(gold["index"], dtype=np.int64)
    errs = []
    for i in range(len(gold["values"])):
        ref = np.asarray(gold["values"][i])
        errs.append(float(np.linalg.norm(np.asarray(W[i], dtype=np.float64)[idx] - ref) / np.linalg.norm(ref)))
    return max(errs)


def run_sweep(args, rank, world, local_rank):
    """advdiff2d-1024 at h = 1e-5 .. 1e-1 in FP64 (tol 2^-53) and FP32 (tol 2^-24): Algorithm 1 once per
    precision, then one solve per h (a warm-up solve first where it is short), CUDA events around the
    series and the recovery.  Errors: against the FP64 oracle's sampled answer where tests/golden holds it
    (h <= 1e-3), else the FP32 result against the GPU FP64 result at the same h (stated as such).  One JSON
    line per (precision, h), then a summary line."""
    import numpy as np
    import torch

    from paper_2509_26475_gb300 import api, build, capi

    if WORKLOAD != "advdiff2d-1024" or world > 1:
        raise SystemExit("--sweep runs the advdiff2d-1024 workload on one GPU")
    build.build()
    lib = capi.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    A_h, V_h, alpha = workload()
    rows, W64 = [], {}
    for precision in ("f64", "f32"):
        dt = torch_dtype(precision)
        tol = tol_of(precision)
        A = api.DeviceCSR.from_host(A_h, device=dev, dtype=dt)
        V = torch.as_tensor(V_h).to(dt).to(dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        Pm = api.select_params(A, tol=tol, check=True)
        e[1].record(stream)
        torch.cuda.synchronize(dev)
        sel_ms = e[0].elapsed_time(e[1])
        prm = api.read_params(Pm)
        for h in SWEEP_HS:
            if h <= 1e-3:
                api.solve(A, V, t_of(h), alpha, tol, Pm, check=True)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            with ClockSampler(local_rank, None) as clk:
                ev[0].record(stream)
                W, st = api.solve(A, V, t_of(h), alpha, tol, Pm, flags=capi.PHIC_PHASE_SERIES)
                ev[1].record(stream)
                api.solve(A, V, t_of(h), alpha, tol, Pm, out=W, stats=st, flags=capi.PHIC_PHASE_RECOVER)
                ev[2].record(stream)
                torch.cuda.synchronize(dev)
            s = api.read_stats(st)
            Wh = W.double().cpu().numpy()
            gold = golden_samples(h)
            if gold is not None:
                err, against = sampled_error(Wh, gold), (f"FP64 oracle ({len(gold['index'])} sampled rows per "
                                                         f"w_i; oracle solve {gold['oracle_seconds']['solve']:.0f} s "
                                                         f"on {gold['oracle_host']})")
            elif precision == "f32" and h in W64:
                err, against = max(rel_errors(Wh, W64[h])), "GPU FP64 at the same h (no oracle run: too long)"
            else:
                err, against = None, "none (no oracle run at this h: too long on the host)"
            if precision == "f64":
                W64[h] = Wh
            row = {"sweep": "advdiff2d-1024", "precision": precision, "tol": "2^-53" if precision == "f64" else "2^-24",
                   "h": h, "status": s["status"], "s": s["s"], "xi": s["xi"], "s_int": s["s_int"],
                   "series_terms": s["series_terms"], "recovery_terms": s["recovery_terms"],
                   "series_ms": ev[0].elapsed_time(ev[1]), "recover_ms": ev[1].elapsed_time(ev[2]),
                   "select_ms": sel_ms, "select_s": prm["s"], "max_rel_err": err, "error_against": against,
                   "bar": 1e-12 if precision == "f64" else 5e-6,
                   "meets_bar": None if err is None else bool(err <= (1e-12 if precision == "f64" else 5e-6)),
                   "clocks": clk.summary()}
            rows.append(row)
            print(json.dumps(row), flush=True)
        del A, V, Pm
        torch.cuda.empty_cache()
    print(json.dumps({"sweep_summary": [(r["precision"], r["h"], r["s_int"], r["max_rel_err"], r["meets_bar"])
                                        for r in rows]}), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# Many instances: one batched launch (batch512) and the continuous-batching request loop (serve)
# ------------------------------------------------------------------------------------------------
def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def solve_bytes(n, nnz, p, r, series_terms, recovery_terms, b):
    """Algorithmic bytes of one solve's sparse block products: per series term the operator
    ((4 + b) nnz + 4 (n+1)) and reading/writing V, D and S (5 n (p+1) r b); per recovery term the operator
    and reading F, reading and writing E, writing the next F (4 n 2r b)."""
    op = (4 + b) * nnz + 4 * (n + 1)
    w_s, w_f = (p + 1) * r, (2 * r if p > 0 else r)
    return series_terms * (op + 5 * n * w_s * b) + recovery_terms * (op + 4 * n * w_f * b)


def batch_workload(precision):
    from paper_2509_26475_gb300 import workloads as wl

    return wl.workload_batch(512, 4, precision)


def run_batch(args, rank, world, local_rank):
    """batch512: 512 independent instances (n log-uniform in [1e3, 2.56e5], 2-D/3-D Laplacians plus
    diagonal shifts, p in 1..4, r in 1..3), each Algorithm 1 + Algorithm 3, all in one persistent
    launch with an autotuned launch shape.  A step is that launch; value = instances solved per second.
    The same instances solved one by one through phic_select_params + phic_solve in FP64 (the plain
    single-instance path) are timed once for comparison."""
    import numpy as np
    import torch

    from paper_2509_26475_gb300 import api, build, capi

    build.build()
    lib = capi.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    prec_name = PRECISION
    insts = batch_workload(prec_name)
    devs = []
    for x in insts:
        dt = torch.float32 if x["prec"] == "f32" else torch.float64
        devs.append((api.DeviceCSR.from_host(x["A"], device=dev, dtype=dt), torch.as_tensor(x["V"]).to(dt).to(dev)))
    items = [api.BatchItem(A, V, x["t"], x["alpha"], tol=x["tol"], select=True) for x, (A, V) in zip(insts, devs)]
    if args.no_tune:
        cfg, tune_ms = {"rows_per_cta": 4096, "blocks_per_sm": 3}, None
    else:
        cands = [{"rows_per_cta": rr, "blocks_per_sm": bb} for bb in (2, 3) for rr in (2048, 4096, 8192)]
        cfg, tune_ms = api.autotune(items, candidates=cands, reps=1)
    b = api.Batch(items, config=cfg)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 0)):
        b.launch()
    torch.cuda.synchronize(dev)
    bad = [i for i, st in enumerate(b.stats()) if st["status"] != 0]
    if bad:
        raise SystemExit(f"batch512: instances {bad[:8]} reported a device status")
    K = max(1, args.steps)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    launches0 = lib.phic_launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    with ClockSampler(local_rank, None) as clk:
        for k in range(K):
            ev0[k].record(stream)
            b.launch()
            ev1[k].record(stream)
        torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    launches = lib.phic_launch_count() - launches0
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(K)]
    ms = reduce_max_over_ranks(statistics.mean(step_ms), dist, dev)
    value = len(items) * world / (ms / 1000.0)
    stats = b.stats()
    nbytes = 0.0
    for x, st in zip(insts, stats):
        bb = 4 if x["prec"] == "f32" else 8
        nbytes += solve_bytes(x["A"].n, x["A"].nnz, x["p"], x["r"], st["series_terms"], st["recovery_terms"], bb)
    hbm_peak = float(_peaks().get("hbm_gbs", 6800.0))
    achieved = nbytes / (statistics.mean(step_ms) / 1000.0) / 1e9
    roofline = {"bound": "hbm", "kernel": "batch_kernel (Algorithms 1 and 3 for all 512 instances, one launch)",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, of measured); algorithmic bytes of the series and "
                             "recovery products only (Algorithm 1's passes not counted)",
                "launch_ms": statistics.mean(step_ms)}
    # the plain single-instance path on the same instances, one by one, timed once: (1) each instance in its
    # own precision and tol (the same stated accuracy as in the batch), (2) every instance in FP64 at 2^-53
    single, single64 = None, None
    if rank == 0:
        ws_p = api.new_params(dev)

        def one_by_one(pairs, tols):
            for A, V in pairs[:4]:  # warm-up
                api.select_params(A, out=ws_p)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = []
            for x, (A, V), tl in zip(insts, pairs, tols):
                Pm = api.select_params(A, tol=tl, out=ws_p)
                outs.append(api.solve(A, V, x["t"], x["alpha"], tl, Pm)[0])
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1), outs

        sms, w_single = one_by_one(devs, [x["tol"] for x in insts])
        single = {"value": len(insts) / (sms / 1000.0), "unit": "solves/s", "ms": sms,
                  "path": "phic_select_params + phic_solve per instance, each in its own precision and tol "
                          "(matched accuracy), same instances"}
        if prec_name != "f64":
            d64 = [(A.astype(torch.float64), V.double()) for (A, V) in devs]
            sms64, _ = one_by_one(d64, [2.0**-53] * len(insts))
            single64 = {"value": len(insts) / (sms64 / 1000.0), "unit": "solves/s", "ms": sms64,
                        "path": "phic_select_params + phic_solve per instance, all FP64 at tol 2^-53"}
            del d64
    errors = None
    cpu_sample = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_sample, refs_ = fleet_oracle_sample(insts[:6], return_results=True)
        bars = {"f64": 1e-12, "f32": 5e-6}
        per = []
        for i, (x, ref) in enumerate(zip(insts[:6], refs_)):
            eb = max(rel_errors(items[i].W.double().cpu().numpy(), ref))
            es = max(rel_errors(w_single[i].double().cpu().numpy(), ref)) if single is not None else None
            per.append({"instance": i, "n": int(x["A"].n), "prec": x["prec"], "batch_err": eb, "single_err": es,
                        "bar": bars[x["prec"]], "within_bar": bool(eb <= bars[x["prec"]])})
        errors = {"metric": "max over i of ||w_i - w_i_oracle||_2 / ||w_i_oracle||_2 (FP64 oracle, its own xi, s)",
                  "sample": per}
    nf32 = sum(1 for x in insts if x["prec"] == "f32")
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "f32": "f32"}.get(prec_name, "f64+f32"), "data": "synthetic",
            "config": {"workload": f"batch512: 512 instances, n log-uniform [1e3, 2.56e5] (2-D/3-D Laplacian + diag "
                                   f"U[-10,0]), p 1..4, r 1..3, Algorithm 1 + 3 each, {prec_name} "
                                   f"({nf32} FP32 at 2^-24, {len(insts) - nf32} FP64 at 2^-53)",
                       "rows": int(sum(x["A"].n for x in insts)), "nnz": int(sum(x["A"].nnz for x in insts)),
                       "launch_shape": cfg, "autotune_ms": tune_ms, "grid": b.info()["grid"],
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                       "step": "one persistent launch over all 512 instances"},
            "roofline": roofline, "gpu_launches": int(launches), "wall_s_timed_region": wall,
            "single_instance": single, "single_instance_fp64": single64, "errors": errors,
            "batch_vs_single": value / single["value"] if single else None}
    clk_sum = clk.summary()
    if clk_sum:
        line["clocks"] = clk_sum
    if not args.no_e2e:
        line["e2e"] = batch_e2e(api, insts, devs, items, b, dev, stream, K, world, dist)
    if cpu_sample is not None:
        line["cpu_baseline"] = cpu_sample
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def batch_e2e(api, insts, devs, items, b, dev, stream, K, world, dist):
    """The batched step from pinned host buffers: copy every operator and V in, one launch, copy every W
    out; CUDA events around all of it."""
    import torch

    host = []
    h2d = d2h = 0
    for (A, V), it in zip(devs, items):
        hp = [t.cpu().pin_memory() for t in (A.rowptr, A.colidx, A.values, V)]
        wo = torch.empty(it.W.shape, dtype=it.W.dtype).pin_memory()
        host.append((hp, wo))
        h2d += sum(t.numel() * t.element_size() for t in hp)
        d2h += wo.numel() * wo.element_size()

    def one():
        for (A, V), (hp, _) in zip(devs, host):
            for dst, src in zip((A.rowptr, A.colidx, A.values, V), hp):
                dst.copy_(src, non_blocking=True)
        b.launch()
        for it, (_, wo) in zip(items, host):
            wo.copy_(it.W, non_blocking=True)

    one()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    e0.record(stream)
    for _ in range(K):
        one()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = reduce_max_over_ranks(e0.elapsed_time(e1) / K, dist, dev)
    return {"value": len(items) * world / (ms / 1000.0), "unit": "solves/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def fleet_oracle_sample(insts, return_results=False):
    """The oracle (Algorithm 1 + Algorithm 3 in FP64 at tol 2^-53, OpenMP over rows) on a few instances."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    outs = []
    t0 = time.perf_counter()
    for x in insts:
        sel = oracle.select(x["A"])
        outs.append(oracle.solve(x["A"], x["V"], x["t"], x["alpha"], 2.0**-53, sel["s"], sel["xi"])[0])
    dt = time.perf_counter() - t0
    res = {"value": len(insts) / dt, "unit": "solves/s", "cores": used, "kind": "oracle",
           "sample": f"the first {len(insts)} instances of the workload (Algorithm 1 + 3 each at tol 2^-53), "
                     "FP64 C oracle"}
    return (res, outs) if return_results else res


def serve_requests(count, seed=5):
    """The serving mix: 80 % instances of the batching distribution (own operators, Algorithm 1 in their
    first slice), 20 % solves on a 3-D 7-point upwind convection-diffusion operator on 100^3 (n = 10^6,
    Peclet 10) registered once (FP64 and FP32 copies), p = 3, r = 2, t = (h/2, h/3), alpha = (1/2, 1/3),
    h = 1e-4; tol 2^-53 (FP64) or 2^-24 (FP32) per request with equal odds; Poisson arrivals."""
    import numpy as np

    from paper_2509_26475_gb300 import workloads as wl

    rng = np.random.default_rng(seed)
    kinds = rng.random(count) < 0.2
    precs = np.where(rng.random(count) < 0.5, "f64", "f32")
    out = []
    for i in range(count):
        if kinds[i]:
            out.append(dict(kind="big", prec=str(precs[i]), vidx=int(rng.integers(0, 4))))
        else:
            x = wl.batch_instance(seed, i, 1000, 256000, str(precs[i]))
            out.append(dict(kind="small", prec=x["prec"], inst=x))
    return out


def serve_stream(srv, hostreq, reqs, big_A, rate, count, seed, local_rank):
    """One Poisson stream of `count` of the prepared requests at `rate` per second into a running server;
    returns the stream's metrics (latency = result on the host minus submission)."""
    import numpy as np

    hostreq, reqs = hostreq[:count], reqs[:count]
    c0 = srv.counters()
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=len(hostreq))
    ids = []
    with ClockSampler(local_rank, None) as clk:
        t_start = time.perf_counter()
        due = t_start
        for q, g in zip(hostreq, gaps):
            due += g
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                time.sleep(min(due - now, 0.0005))
            ids.append(srv.submit(q))
        infos = [srv.wait(i, 600000) for i in ids]
        t_end = time.perf_counter()
    c1 = srv.counters()
    bad = [i for i, x in enumerate(infos) if x["status"] != 0]
    if bad:
        srv.close()
        raise SystemExit(f"serve: {len(bad)} of {len(infos)} requests reported a device status (first: request "
                         f"{bad[0]}, status {infos[bad[0]]['status']}); no number is reported")
    lat = np.array([(x["done_ns"] - x["submit_ns"]) / 1e6 for x in infos])
    first_sub = min(x["submit_ns"] for x in infos)
    last_sub = max(x["submit_ns"] for x in infos)
    last_done = max(x["done_ns"] for x in infos)
    span = (last_done - first_sub) / 1e9
    nbytes = 0.0
    for q, x in zip(reqs, infos):
        st = x["stats"]
        if q["kind"] == "big":
            n, nnz, p, r = big_A.n, big_A.nnz, 3, 2
        else:
            n, nnz, p, r = q["inst"]["A"].n, q["inst"]["A"].nnz, q["inst"]["p"], q["inst"]["r"]
        nbytes += solve_bytes(n, nnz, p, r, st["series_terms"], st["recovery_terms"], 4 if q["prec"] == "f32" else 8)
    busy_s = (c1["gpu_busy_ms"] - c0["gpu_busy_ms"]) / 1000.0
    # backlog when the last request arrived: submitted but not yet completed
    backlog = sum(1 for x in infos if x["done_ns"] > last_sub)
    return {"offered_rate": rate, "requests": len(infos), "achieved_rate": len(infos) / span, "span_s": span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "backlog_at_last_arrival": backlog,
            "slices": c1["slices"] - c0["slices"], "max_slice_requests": c1["max_slice_requests"],
            "gpu_busy_frac": busy_s / span if span > 0 else None, "busy_s": busy_s, "bytes": nbytes,
            "arena_peak_gb": c1["arena_peak"] / 1e9, "wall_s": t_end - t_start, "clocks": clk.summary(),
            "failed": 0}


def run_serve(args, rank, world, local_rank):
    """serve: Poisson arrivals of solve requests into the continuous-batching loop.  The line's value is
    the stream at --rate (--requests arrivals): completed solves per second of wall time (first arrival to
    last result on the host), latency = result-on-host minus submission, p50 and p99.  Before it, streams
    at lower offered rates (SERVE_CURVE_RATES, at least 300 requests or 3 s of arrivals each) give the
    latency-versus-load curve and the loop's capacity."""
    import numpy as np
    import torch

    from paper_2509_26475_gb300 import api, build, capi
    from paper_2509_26475_gb300 import workloads as wl

    build.build()
    capi.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    reqs = serve_requests(args.requests)
    big_A = wl.convection_diffusion(100, 3, 10.0)
    rng = np.random.default_rng(7)
    bigV = {pr: [rng.standard_normal((4, big_A.n)).astype(np.float32 if pr == "f32" else np.float64) for _ in range(4)]
            for pr in ("f64", "f32")}
    h = 1e-4
    free = torch.cuda.mem_get_info(dev)[0]
    arena = int(min(free * 0.85, 200e9))
    srv = api.Server(arena_bytes=arena, device=local_rank)
    ops = {pr: srv.add_operator(api.HostOperator(big_A, prec=pr)) for pr in ("f64", "f32")}
    while any(srv.operator_params(o) is None for o in ops.values()):
        time.sleep(0.01)
    # page-locked inputs for every request, prepared before the arrivals start
    hostreq = []
    for q in reqs:
        if q["kind"] == "big":
            hostreq.append(api.HostRequest(big_A.n, bigV[q["prec"]][q["vidx"]], [h / 2, h / 3], [0.5, 1.0 / 3.0],
                                           tol=2.0**-53 if q["prec"] == "f64" else 2.0**-24, prec=q["prec"],
                                           op=ops[q["prec"]]))
        else:
            x = q["inst"]
            hostreq.append(api.HostRequest(x["A"], x["V"], x["t"], x["alpha"], tol=x["tol"], prec=x["prec"]))
    # warm-up: a few requests through the loop
    for k in range(max(args.warmup, 0)):  # the buffers are reused by the timed streams (W is rewritten)
        for i in [srv.submit(r) for r in hostreq[k * 4:(k + 1) * 4]]:
            srv.wait(i, 120000)
    curve = []
    for rate in [x for x in SERVE_CURVE_RATES if x < args.rate]:
        cnt = min(len(hostreq), max(300, int(3.0 * rate)))
        curve.append(serve_stream(srv, hostreq, reqs, big_A, rate, cnt, 11 + len(curve), local_rank))
    m = serve_stream(srv, hostreq, reqs, big_A, args.rate, len(hostreq), 11, local_rank)
    curve.append(m)
    srv.close()
    hbm_peak = float(_peaks().get("hbm_gbs", 6800.0))
    achieved = m["bytes"] / m["busy_s"] / 1e9 if m["busy_s"] > 0 else 0.0
    # bytes the server copies per request: the operator's CSR arrays (none for a registered operator)
    # and V in, W out
    def _nb(x):
        return 0 if x is None else x.numel() * x.element_size()
    h2d = int(sum(_nb(q.rowptr) + _nb(q.colidx) + _nb(q.values) + _nb(q.V) for q in hostreq))
    d2h = int(sum(_nb(q.W) for q in hostreq))
    kept = [c for c in curve if c["achieved_rate"] >= 0.9 * c["offered_rate"]]
    line = {"metric": METRIC, "value": m["achieved_rate"], "unit": "solves/s", "n_gpus": 1, "steps": 1,
            "warmup": args.warmup, "ms_per_step": m["span_s"] * 1000.0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "latency_ms": {"p50": m["p50_ms"], "p99": m["p99_ms"], "mean": m["mean_ms"], "max": m["max_ms"]},
            "latency_curve": [{k: c[k] for k in ("offered_rate", "requests", "achieved_rate", "p50_ms", "p99_ms",
                                                 "backlog_at_last_arrival", "slices", "gpu_busy_frac")}
                              for c in curve],
            "capacity": {"completed_per_s_at_highest_load": max(c["achieved_rate"] for c in curve),
                         "highest_offered_rate_kept_up": max((c["offered_rate"] for c in kept), default=None),
                         "note": "kept up = completed at least 90 % of the offered rate over the stream"},
            "config": {"workload": f"serve: {m['requests']} Poisson arrivals at {args.rate:g}/s; 80% batching-"
                                   "distribution instances (own operator, Algorithm 1 in the first slice), 20% n=1e6 "
                                   "3-D convection-diffusion (100^3, Pe 10) solves on a registered operator, p=3 r=2 "
                                   "t=(h/2,h/3) h=1e-4; tol 2^-53 FP64 or 2^-24 FP32 per request",
                       "offered_rate": args.rate, "achieved_rate": m["achieved_rate"], "failed": 0,
                       "backlog_at_last_arrival": m["backlog_at_last_arrival"],
                       "slices": m["slices"], "max_slice_requests": m["max_slice_requests"],
                       "gpu_busy_frac": m["gpu_busy_frac"], "arena_gb": arena / 1e9,
                       "arena_peak_gb": m["arena_peak_gb"],
                       "step": "the whole arrival stream (first submission to last result on the host)",
                       "l2": "inputs larger than L2 (no flush)", "parallelism": "x1"},
            "roofline": {"bound": "hbm", "kernel": "batch_kernel slices (series + recovery products)",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": None, "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, of measured); "
                                                       "algorithmic bytes over the slices' device time"},
            "gpu_launches": int(m["slices"]) * 2, "wall_s_timed_region": m["wall_s"],
            "e2e": {"value": m["achieved_rate"], "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "note": "the serving numbers are end to end already: host inputs in, results on the host; "
                            "the step is the whole stream"}}
    if m["clocks"]:
        line["clocks"] = m["clocks"]
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# The expRK4s6 driver on the ADR problem (exprk-adr) and a low-rank operator (lowrank-m2)
# ------------------------------------------------------------------------------------------------
# One bounded team barrier at 304 blocks on GB300 (microbenchmark): the floor of a Taylor term whose
# working set is L2-resident.
BARRIER_US = 2.5


def _latency_roofline(kernel, terms, seconds, barriers_per_term):
    """Taylor terms per second against the rate at which every term costs only its team barriers."""
    achieved = terms / seconds
    peak = 1e6 / (BARRIER_US * barriers_per_term)
    return {"bound": "latency", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "Taylor terms/s",
            "frac": achieved / peak, "traffic": None,
            "peak_note": f"{barriers_per_term} team barrier(s) per term at {BARRIER_US} us each (GB300 "
                         "microbenchmark at 304 blocks); the working set is L2-resident"}


def _aux_line(value, ms, K, warmup, dtype, config, roofline, launches, wall, e2e, clk):
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": K, "warmup": warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config, "roofline": roofline, "gpu_launches": int(launches),
            "wall_s_timed_region": wall, "e2e": e2e}
    summary = clk.summary()
    if summary:
        line["clocks"] = summary
    print(json.dumps(line), flush=True)
    return 0


def run_exprk(args, rank, world, local_rank):
    """exprk-adr: expRK4s6 on the paper's ADR problem (100 x 100 nodes, eps 1e-3, alpha -1/2,
    gamma 1000), FP64 at tol 2^-53, h = 1/512, (s, xi) selected once before the timed region.  One
    step = one integrator step: four phi-combination calls and the elementwise reaction terms, captured
    once as a CUDA graph and replayed; value = calls (solves) per second.  The same steps issued eagerly
    from Python are timed beside it (config).  e2e copies u from pinned host memory in and out again
    every step."""
    import torch

    from paper_2509_26475_gb300 import api, build, capi, exprk
    from paper_2509_26475_gb300 import workloads as wl

    if world > 1:
        raise SystemExit("exprk-adr runs on one GPU")
    build.build()
    lib = capi.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    h, K = 1.0 / 512, args.steps
    A = api.DeviceCSR.from_host(wl.adr_operator(), device=dev)
    integ = exprk.ExpRK4s6(A, exprk.adr_reaction(wl.ADR_GAMMA))
    u = torch.as_tensor(wl.adr_initial()).to(dev)

    def timed(fn):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        return ev[0].elapsed_time(ev[1]) / K

    # eager steps (Python issues every call)
    for _ in range(max(args.warmup, 0)):
        u = integ.step(u, h)
    integ.check()
    state = {"u": u}

    def eager():
        for _ in range(K):
            state["u"] = integ.step(state["u"], h)

    ms_eager = timed(eager)
    sts = [api.read_stats(x) for x in integ.stats]
    integ.check()
    # the captured step, replayed
    u = state["u"]
    l0 = lib.phic_launch_count()
    sg = integ.capture(u, h)
    per_step = lib.phic_launch_count() - l0 - 8  # capture() runs one eager warm-up step (8 launches) first
    sg.replay(max(args.warmup, 1))
    sg.check()
    with ClockSampler(local_rank, None) as clk:
        w0 = time.perf_counter()
        ms = timed(lambda: sg.replay(K))
        wall = time.perf_counter() - w0
    sg.check()
    last = [api.read_stats(x) for x in sg.stats]  # the four calls of the last replayed step
    if any(x["status"] != 0 for x in sts + last) or not bool(torch.isfinite(u).all()):
        raise SystemExit("exprk-adr: a phi-combination reported a device status; no number is reported")
    terms = sum(x["series_terms"] + x["recovery_terms"] for x in last)
    # e2e: the integration driven from the host, u in and out of pinned memory every step
    uh = u.detach().cpu().pin_memory()
    nb = uh.numel() * uh.element_size()

    def host_loop():
        for _ in range(K):
            u.copy_(uh, non_blocking=True)
            sg.replay()
            uh.copy_(u, non_blocking=True)

    ms_e2e = timed(host_loop)
    sg.check()
    config = {"workload": "exprk-adr: expRK4s6 on the ADR problem, 100 x 100 nodes (n = 10,000), eps 1e-3, "
                          "alpha -1/2, gamma 1000, h = 1/512, FP64 tol 2^-53; (s, xi) selected once; each step "
                          "one CUDA graph replay",
              "n": A.n, "nnz": A.nnz, "h": h, "calls_per_step": 4, "steps_per_s": 1000.0 / ms,
              "eager_steps_per_s": 1000.0 / ms_eager, "taylor_terms_per_step": terms,
              "launches_per_step": per_step, "s": float(api.read_params(integ.params)["s"]),
              "l2": "working set L2-resident (n = 10,000); no flush", "parallelism": "x1"}
    return _aux_line(4 * 1000.0 / ms, ms, K, args.warmup, "f64", config,
                     _latency_roofline("series_kernel + recover_kernel (4 calls per step)", terms * K, ms * K / 1000.0, 1),
                     per_step * K, wall, {"value": 4 * 1000.0 / ms_e2e, "unit": "solves/s", "ms_per_step": ms_e2e,
                                          "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}, clk)


def run_lowrank(args, rank, world, local_rank):
    """lowrank-m2: the paper's third experiment with the core M2 = [[-1, 1e5], [0, -10]]: A = U W^T,
    U the first two DCT-II columns of size n = 400,000, W = U M2^T, applied matrix-free; p = 4, r = 1,
    alpha = 1, FP64 at tol 2^-53, v_j ~ N(0, 1) (seed 11).  One step = Algorithm 1 + Algorithm 3 at
    t = 0.1 and t = 1 (2 solves); L2 flushed between steps."""
    import numpy as np
    import torch

    from paper_2509_26475_gb300 import api, build, capi
    from paper_2509_26475_gb300 import workloads as wl

    if world > 1:
        raise SystemExit("lowrank-m2 runs on one GPU")
    build.build()
    lib = capi.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    n, p, ts = 400000, 4, (0.1, 1.0)
    M = np.array([[-1.0, 1e5], [0.0, -10.0]])
    U_h = wl.dct_basis(n, 2)
    W_h = U_h @ M.T
    V_h = np.random.default_rng(11).standard_normal((p + 1, n))
    A = api.DeviceLowRank(torch.as_tensor(U_h).to(dev).contiguous(), torch.as_tensor(W_h).to(dev).contiguous())
    V = torch.as_tensor(V_h).to(dev)
    flush = torch.empty(2 * torch.cuda.get_device_properties(dev).L2_cache_size, dtype=torch.uint8, device=dev)
    roof_m = measure_fp64_roof(lib, capi, dev, local_rank)

    def step():
        P = api.select_params(A, tol=TOL)
        return P, [api.solve(A, V, [t], [1.0], TOL, P) for t in ts]

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sts = []
    l0 = lib.phic_launch_count()
    with ClockSampler(local_rank, None) as clk:
        w0 = time.perf_counter()
        for k in range(K):
            flush.fill_(k & 255)
            evs[k][0].record(stream)
            P = api.select_params(A, tol=TOL)
            evs[k][1].record(stream)
            sts += [api.solve(A, V, [t], [1.0], TOL, P)[1] for t in ts]
            evs[k][2].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - w0
    launches = lib.phic_launch_count() - l0
    ms = sum(e[0].elapsed_time(e[2]) for e in evs) / K
    solve_s = sum(e[1].elapsed_time(e[2]) for e in evs) / 1000.0
    st = [api.read_stats(x) for x in sts]
    if any(x["status"] != 0 for x in st):
        raise SystemExit("lowrank-m2: a solve reported a device status; no number is reported")
    terms = sum(x["series_terms"] + x["recovery_terms"] for x in st)
    # e2e: U, W and V in from pinned host memory, the results out, every step
    Uh, Wh, Vh = (torch.as_tensor(x).pin_memory() for x in (U_h, W_h, V_h))
    outs = [torch.empty((1, n), dtype=torch.float64).pin_memory() for _ in ts]
    e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e2[0].record(stream)
    for _ in range(K):
        Ad = api.DeviceLowRank(Uh.to(dev, non_blocking=True), Wh.to(dev, non_blocking=True))
        Vd = Vh.to(dev, non_blocking=True)
        Pd = api.select_params(Ad, tol=TOL)
        for o, t in zip(outs, ts):
            o.copy_(api.solve(Ad, Vd, [t], [1.0], TOL, Pd)[0], non_blocking=True)
    e2[1].record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = e2[0].elapsed_time(e2[1]) / K
    h2d = sum(x.numel() * x.element_size() for x in (Uh, Wh, Vh))
    d2h = sum(o.numel() * o.element_size() for o in outs)
    config = {"workload": "lowrank-m2: A = U W^T, W = U M2^T, M2 = [[-1, 1e5], [0, -10]], U = 2 DCT-II columns, "
                          "n = 400,000, p = 4, r = 1, t in {0.1, 1}, alpha = 1, FP64 tol 2^-53",
              "n": n, "k": 2, "p": p, "t": list(ts), "s_int": [x["s_int"] for x in st[:len(ts)]],
              "terms": [x["series_terms"] + x["recovery_terms"] for x in st[:len(ts)]],
              "step": "Algorithm 1 + Algorithm 3 at each t (2 solves)",
              "l2": "flushed between steps (2 x L2 write, outside the step events)", "parallelism": "x1"}
    # FP64 flops of the two solves: per product with A = U W^T, W^T X and U Z (4 n k w), plus the
    # series update (about 4 n w per term) or the recovery update (about 3 n w per term)
    ws_, wf_ = (p + 1) * 1, 2 * 1
    flops = sum(x["series_terms"] * (4 * n * 2 + 4 * n) * ws_ + x["recovery_terms"] * (4 * n * 2 + 3 * n) * wf_
                for x in st)
    achieved = flops / solve_s / 1e9
    roof = {"bound": "alu", "kernel": "lr_series_kernel + lr_recover_kernel (the two solves of a step)",
            "achieved": achieved, "peak": roof_m["gflops"], "unit": "FP64 GFLOP/s",
            "frac": achieved / roof_m["gflops"], "traffic": None,
            "peak_note": f"of measured: FP64 FMA rate of the probe kernel ({roof_m['fma_per_clk_per_sm']:.3f} "
                         f"FMA/clk/SM at {roof_m['sm_mhz']:.0f} MHz); achieved counts (4 n k + 4 n) w "
                         "flops per series term and (4 n k + 3 n) w per recovery term, k = 2; the working set is "
                         "L2-resident",
            "taylor_terms_per_s": terms / solve_s}
    return _aux_line(len(ts) * 1000.0 / ms, ms, K, args.warmup, "f64", config, roof,
                     launches, wall, {"value": len(ts) * 1000.0 / ms_e2e, "unit": "solves/s", "ms_per_step": ms_e2e,
                                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}, clk)


def run_reference_exprk(args):
    """--impl reference for exprk-adr: the same expRK4s6 steps with every phi-combination by the oracle
    (FP64 C, OpenMP over sparse-product rows) on the host cores, for a bounded number of steps."""
    import numpy as np

    import oracle
    from paper_2509_26475_gb300 import exprk
    from paper_2509_26475_gb300 import workloads as wl

    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    A_h = wl.adr_operator()
    g = exprk.adr_reaction(wl.ADR_GAMMA)
    sel = oracle.select(A_h)
    h = 1.0 / 512

    def comb(ci):
        return oracle.solve(A_h, np.stack(ci.V), ci.t, ci.alpha, 2.0**-53, sel["s"], sel["xi"])[0]

    def step(u):
        gu = g(u)
        hg = h * gu
        U2 = comb(exprk.stage2_inputs(u, hg, h))[0]
        D2 = g(U2) - gu
        W34 = comb(exprk.stage34_inputs(u, hg, D2, h))
        D3, D4 = g(W34[0]) - gu, g(W34[1]) - gu
        W56 = comb(exprk.stage56_inputs(u, hg, D3, D4, h))
        D5, D6 = g(W56[0]) - gu, g(W56[1]) - gu
        return comb(exprk.final_inputs(u, hg, D5, D6, h))[0]

    u = wl.adr_initial()
    steps_run, warm_run = min(max(1, args.steps), 20), min(max(0, args.warmup), 1)
    for _ in range(warm_run):
        u = step(u)
    t0 = time.perf_counter()
    for _ in range(steps_run):
        u = step(u)
    ms = 1000.0 * (time.perf_counter() - t0) / steps_run
    value = 4 * 1000.0 / ms
    sample = f"{steps_run} expRK4s6 step(s) of h = 1/512 on the ADR problem (4 oracle combinations each)"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
                      "steps": steps_run, "warmup": warm_run, "ms_per_step": ms, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "exprk-adr (oracle combinations)", "device": "host CPU", "threads": cores},
                      "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)
    return 0


def run_reference_fleet(args):
    """--impl reference for batch512 / serve: the oracle on a bounded sample of the same instances."""
    if WORKLOAD == "batch512":
        insts = batch_workload(PRECISION if PRECISION != "f64" else "f64")[:6]
    else:
        insts = [q["inst"] for q in serve_requests(40) if q["kind"] == "small"][:6]
    cb = fleet_oracle_sample(insts)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "solves/s", "n_gpus": args.gpus,
            "steps": 1, "warmup": 0, "ms_per_step": 1000.0 * len(insts) / cb["value"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "device": "host CPU", "threads": cb["cores"]},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
