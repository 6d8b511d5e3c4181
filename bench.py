#!/usr/bin/env python3
"""Benchmark of the phi-combination solver on one GB300 (or N replicas under torchrun).

Workload (expRK4s6-shaped block): 3-D 7-point first-order upwind convection-diffusion on a 64^3
Dirichlet grid (n = 262,144, nnz = 1,810,432, Peclet 10, FP64 CSR), p = 3, r = 2,
t = (h/2, h/3), alpha = (1/2, 1/3), h in {1e-4, 1e-2}, tol = 2^-53, v_j ~ N(0,1) (seed 2).

One step = Algorithm 1 (shift/scaling) on A + Algorithm 3 at h = 1e-4 + Algorithm 3 at h = 1e-2, so a
step is 2 solves; value = solves/s over all ranks.  Inputs are resident in HBM before the timed
region; L2 is flushed (a 2 x L2 write) between timed steps, outside the per-step CUDA events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

``--impl reference`` times the CPU oracle (plain FP64 C, OpenMP over sparse-product rows) on the same
workload on this machine's host cores.
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
# FP64 pipe of a GB300 SM: 2 FMA/clk (1.91 measured), 152 SMs, 2070 MHz maximum SM clock; 2 flops an FMA.
FP64_PEAK_GFLOPS = 2.0 * 2.0 * 152 * 2.070

# Workload of the benchmark line (defaults) and the auxiliary FP32/FP64 precision workload.
WORKLOADS = {
    "convdiff3d-64": dict(hs=(1e-4, 1e-2), p=3, r=2, t=lambda h: [h / 2.0, h / 3.0],
                          name="convdiff3d-64^3 Pe10 (n=262144) p=3 r=2 t=(h/2,h/3) alpha=(1/2,1/3) h={1e-4,1e-2}"),
    "advdiff2d-1024": dict(hs=(1e-5, 1e-4), p=4, r=4, t=lambda h: [0.25 * h, 0.5 * h, 0.75 * h, h],
                           name="advdiff2d-1024^2 Pe1e3 (n=1048576) p=4 r=4 t=(1/4,1/2,3/4,1)h alpha=1 h={1e-5,1e-4}"),
}
WORKLOAD = "convdiff3d-64"
PRECISION = "f64"
HS = WORKLOADS[WORKLOAD]["hs"]
TOL = 2.0**-53
P, R = 3, 2
WORKLOAD_NAME = WORKLOADS[WORKLOAD]["name"] + " tol=2^-53"


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
    TOL = 2.0**-53 if precision == "f64" else 2.0**-24
    WORKLOAD_NAME = cfg["name"] + (" tol=2^-53 FP64" if precision == "f64" else " tol=2^-24 FP32")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="convdiff3d-64",
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


def torch_dtype():
    import torch

    return torch.float64 if PRECISION == "f64" else torch.float32


def recorded_traffic(terms: int):
    """DRAM bytes of one launch of the dominant kernel from the committed ncu record of this workload and
    precision, if that record was taken on the current kernel sources (sha256 of each); None otherwise.
    A record of a shorter launch of the same kernel (fewer Taylor terms) is scaled by the terms: every
    term moves the same bytes once the working set exceeds L2, which is when the scaling is used."""
    import hashlib

    name = "recover_kernel_convdiff3d_64.json" if (WORKLOAD, PRECISION) == ("convdiff3d-64", "f64") else \
        "recover_kernel_advdiff2d_1024_fp32.json" if (WORKLOAD, PRECISION) == ("advdiff2d-1024", "f32") else None
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


# ------------------------------------------------------------------------------------------------
# Oracle timing (CPU)
# ------------------------------------------------------------------------------------------------
def oracle_step(oracle, A, V, alpha):
    sel = oracle.select(A)
    for h in HS:
        oracle.solve(A, V, t_of(h), alpha, TOL, sel["s"], sel["xi"])


def time_oracle(steps, warmup):
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    A, V, alpha = workload()
    for _ in range(warmup):
        oracle_step(oracle, A, V, alpha)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle_step(oracle, A, V, alpha)
        times.append(time.perf_counter() - t0)
    return times, used


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
    # bound the whole run to a few minutes: at most 6 timed steps and 1 warm-up of the full oracle step
    steps_run, warm_run = min(steps, 6), min(warmup, 1)
    times, cores = time_oracle(steps_run, warm_run)
    ms = 1000.0 * statistics.mean(times)
    value = len(HS) / (ms / 1000.0)
    sample = (f"full step (Algorithm 1 + Algorithm 3 at h=1e-4 and h=1e-2) on the benchmark workload; "
              f"{steps_run} timed step(s) after {warm_run} warm-up (asked {steps}/{warmup})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": steps_run, "warmup": warm_run, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "device": "host CPU", "threads": cores},
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

    A_h, V_h, alpha = workload()
    dt = torch_dtype()
    prec = capi.PHIC_F64 if PRECISION == "f64" else capi.PHIC_F32
    A = api.DeviceCSR.from_host(A_h, device=dev, dtype=dt)
    V = torch.as_tensor(V_h).to(dt).to(dev)
    n, nnz = A.n, A.nnz
    params = api.new_params(dev)
    stats = [api.new_stats(dev) for _ in HS]
    W = [torch.empty((R, n), dtype=dt, device=dev) for _ in HS]
    ws_sel = torch.empty(api.select_workspace_bytes(n), dtype=torch.uint8, device=dev)
    ws_sol = torch.empty(api.solve_workspace_bytes(n, nnz, P, R, prec), dtype=torch.uint8, device=dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(2 * l2, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev_rec=None):
        api.select_params(A, tol=TOL, out=params, workspace=ws_sel)
        for idx, h in enumerate(HS):
            if ev_rec is not None and idx == len(HS) - 1:
                api.solve(A, V, t_of(h), alpha, TOL, params, out=W[idx], stats=stats[idx], workspace=ws_sol,
                          flags=capi.PHIC_PHASE_SERIES)
                ev_rec[0].record(stream)
                api.solve(A, V, t_of(h), alpha, TOL, params, out=W[idx], stats=stats[idx], workspace=ws_sol,
                          flags=capi.PHIC_PHASE_RECOVER)
                ev_rec[1].record(stream)
            else:
                api.solve(A, V, t_of(h), alpha, TOL, params, out=W[idx], stats=stats[idx], workspace=ws_sol)

    def check_status():
        torch.cuda.synchronize(dev)
        capi.check(api.read_params(params)["status"], "select (device)")
        for st in stats:
            capi.check(api.read_stats(st)["status"], "solve (device)")

    for _ in range(max(args.warmup, 0)):
        step()
    check_status()

    K = max(1, args.steps)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    launches0 = lib.phic_launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    with ClockSampler(local_rank, None) as clk:
        for k in range(K):
            flush.fill_(k & 0xFF)  # 2 x L2 write between steps, outside the step's events
            ev0[k].record(stream)
            step(evr[k])
            ev1[k].record(stream)
        torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    launches = lib.phic_launch_count() - launches0
    check_status()
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(K)]
    rec_ms = [evr[k][0].elapsed_time(evr[k][1]) for k in range(K)]
    ms = reduce_max_over_ranks(statistics.mean(step_ms), dist, dev)
    value = solves_per_second(ms, world)

    st_last = api.read_stats(stats[-1])
    prm = api.read_params(params)
    wf = 2 * R
    b = 8 if PRECISION == "f64" else 4
    flops, bytes_ = recover_kernel_work(n, nnz, wf, P, R, st_last["recovery_terms"], st_last["s_int"] - 1, b)
    rec_s = statistics.mean(rec_ms) / 1000.0
    achieved = flops / rec_s / 1e9
    hbm_gbs = bytes_ / rec_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    kernel = f"recover_kernel (Algorithm 3 recovery loop, h={HS[-1]:g})"
    if PRECISION == "f64":
        roofline = {"bound": "alu", "kernel": kernel,
                    "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "FP64 GFLOP/s",
                    "frac": achieved / FP64_PEAK_GFLOPS,
                    "traffic": recorded_traffic(st_last["recovery_terms"]),
                    "peak_note": "FP64 pipe: 2 FMA/clk/SM x 2 flop x 152 SMs x 2070 MHz (probe measured "
                                 "1.91 FMA/clk/SM); achieved counts (2 nnz + 3 n) 2r flops per Taylor term",
                    "launch_ms": statistics.mean(rec_ms), "terms_per_launch": st_last["recovery_terms"],
                    "hbm_view": {"algorithmic_gbs": hbm_gbs, "peak_gbs": hbm_peak,
                                 "frac_of_measured": hbm_gbs / hbm_peak}}
    else:
        roofline = {"bound": "hbm", "kernel": kernel, "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_gbs / hbm_peak, "traffic": recorded_traffic(st_last["recovery_terms"]),
                    "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, of measured)",
                    "launch_ms": statistics.mean(rec_ms), "terms_per_launch": st_last["recovery_terms"]}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": PRECISION, "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "n": n, "nnz": nnz, "p": P, "r": R, "h": list(HS),
                       "tol": "2^-53" if PRECISION == "f64" else "2^-24",
                       "step": "Algorithm 1 + Algorithm 3 at each h (2 solves)",
                       "l2": "flushed between steps (2 x L2 write, outside the step events)",
                       "parallelism": f"replicas x{world}",
                       "s": prm["s"], "xi": prm["xi"], "s_int": [api.read_stats(s)["s_int"] for s in stats],
                       "terms": [api.read_stats(s)["series_terms"] + api.read_stats(s)["recovery_terms"] for s in stats]},
            "roofline": roofline, "gpu_launches": int(launches), "wall_s_timed_region": wall}
    clk_sum = clk.summary()
    if clk_sum:
        line["clocks"] = clk_sum

    if not args.no_e2e:
        line["e2e"] = e2e(api, capi, A_h, V_h, alpha, dev, stream, K, world, dist)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and WORKLOAD == "convdiff3d-64":
        times, cores = time_oracle(1, 0)
        line["cpu_baseline"] = {"value": len(HS) / times[0], "unit": "solves/s", "cores": cores, "kind": "oracle",
                                "sample": "one full step (Algorithm 1 + Algorithm 3 at h=1e-4 and 1e-2) of the "
                                          "benchmark workload, FP64 C oracle, OpenMP over sparse-product rows"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def e2e(api, capi, A_h, V_h, alpha, dev, stream, K, world, dist):
    """Same step through the public API from pinned host buffers: copy A and V in, Algorithm 1, both
    solves, copy the results out; CUDA events around everything."""
    import numpy as np
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
    # the plain single-instance FP64 path on the same instances (one by one), timed once
    single = None
    if rank == 0:
        ws_p = api.new_params(dev)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d64 = [(A.astype(torch.float64), V.double()) for (A, V) in devs]
        for A, V in d64[:4]:  # warm-up
            api.select_params(A, out=ws_p)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for x, (A, V) in zip(insts, d64):
            P = api.select_params(A, out=ws_p)
            api.solve(A, V, x["t"], x["alpha"], 2.0**-53, P)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sms = e0.elapsed_time(e1)
        single = {"value": len(insts) / (sms / 1000.0), "unit": "solves/s", "ms": sms,
                  "path": "phic_select_params + phic_solve per instance, FP64 at tol 2^-53, same 512 instances"}
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
            "single_instance_fp64": single}
    clk_sum = clk.summary()
    if clk_sum:
        line["clocks"] = clk_sum
    if not args.no_e2e:
        line["e2e"] = batch_e2e(api, insts, devs, items, b, dev, stream, K, world, dist)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = fleet_oracle_sample(insts[:6])
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


def fleet_oracle_sample(insts):
    """The oracle (Algorithm 1 + Algorithm 3 in FP64, OpenMP over rows) on a few instances."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    t0 = time.perf_counter()
    for x in insts:
        sel = oracle.select(x["A"], tol=x["tol"])
        oracle.solve(x["A"], x["V"], x["t"], x["alpha"], x["tol"], sel["s"], sel["xi"])
    dt = time.perf_counter() - t0
    return {"value": len(insts) / dt, "unit": "solves/s", "cores": used, "kind": "oracle",
            "sample": f"the first {len(insts)} instances of the workload (Algorithm 1 + 3 each), FP64 C oracle"}


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


def run_serve(args, rank, world, local_rank):
    """serve: Poisson arrivals at --rate of --requests solve requests into the continuous-batching loop;
    value = completed solves per second of wall time (first arrival to last result on the host),
    latency = result-on-host minus submission, p50 and p99."""
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
    for k in range(max(args.warmup, 0)):  # the buffers are reused by the timed stream (W is rewritten)
        for i in [srv.submit(r) for r in hostreq[k * 4:(k + 1) * 4]]:
            srv.wait(i, 120000)
    c0 = srv.counters()
    gaps = np.random.default_rng(11).exponential(1.0 / args.rate, size=len(hostreq))
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
    last_done = max(x["done_ns"] for x in infos)
    span = (last_done - first_sub) / 1e9
    failed = sum(1 for x in infos if x["status"] != 0)
    nbytes = 0.0
    for q, x in zip(reqs, infos):
        st = x["stats"]
        if q["kind"] == "big":
            n, nnz, p, r = big_A.n, big_A.nnz, 3, 2
        else:
            n, nnz, p, r = q["inst"]["A"].n, q["inst"]["A"].nnz, q["inst"]["p"], q["inst"]["r"]
        nbytes += solve_bytes(n, nnz, p, r, st["series_terms"], st["recovery_terms"], 4 if q["prec"] == "f32" else 8)
    busy_s = (c1["gpu_busy_ms"] - c0["gpu_busy_ms"]) / 1000.0
    hbm_peak = float(_peaks().get("hbm_gbs", 6800.0))
    achieved = nbytes / busy_s / 1e9 if busy_s > 0 else 0.0
    value = len(infos) / span
    # bytes the server copies per request: the operator's CSR arrays (none for a registered operator)
    # and V in, W out
    def _nb(x):
        return 0 if x is None else x.numel() * x.element_size()
    h2d = int(sum(_nb(q.rowptr) + _nb(q.colidx) + _nb(q.values) + _nb(q.V) for q in hostreq))
    d2h = int(sum(_nb(q.W) for q in hostreq))
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
            "ms_per_step": span * 1000.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32", "data": "synthetic",
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "config": {"workload": f"serve: {len(reqs)} Poisson arrivals at {args.rate:g}/s; 80% batching-distribution "
                                   "instances (own operator, Algorithm 1 in the first slice), 20% n=1e6 3-D "
                                   "convection-diffusion (100^3, Pe 10) solves on a registered operator, p=3 r=2 "
                                   "t=(h/2,h/3) h=1e-4; tol 2^-53 FP64 or 2^-24 FP32 per request",
                       "offered_rate": args.rate, "achieved_rate": value, "failed": failed,
                       "slices": c1["slices"] - c0["slices"], "max_slice_requests": c1["max_slice_requests"],
                       "gpu_busy_frac": busy_s / span if span > 0 else None, "arena_gb": arena / 1e9,
                       "arena_peak_gb": c1["arena_peak"] / 1e9,
                       "step": "the whole arrival stream (first submission to last result on the host)",
                       "l2": "inputs larger than L2 (no flush)", "parallelism": "x1"},
            "roofline": {"bound": "hbm", "kernel": "batch_kernel slices (series + recovery products)",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": None, "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, of measured); "
                                                       "algorithmic bytes over the slices' device time"},
            "gpu_launches": int(c1["slices"] - c0["slices"]) * 2, "wall_s_timed_region": t_end - t_start,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "note": "the serving numbers are end to end already: host inputs in, results on the host; "
                            "the step is the whole stream"}}
    clk_sum = clk.summary()
    if clk_sum:
        line["clocks"] = clk_sum
    srv.close()
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
            "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "FP64 GFLOP/s",
            "frac": achieved / FP64_PEAK_GFLOPS, "traffic": None,
            "peak_note": "FP64 pipe: 2 FMA/clk/SM x 2 flop x 152 SMs x 2070 MHz; achieved counts (4 n k + 4 n) w "
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
