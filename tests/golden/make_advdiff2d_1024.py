#!/usr/bin/env python3
"""Writes tests/golden/advdiff2d_1024_h<h>.json: the oracle's answer on the 1024^2 workload, reduced to
what a test can compare against at full size.

Workload: 2-D first-order upwind advection-diffusion on a 1024 x 1024 Dirichlet grid (n = 1,048,576,
Peclet 1e3), p = 4, r = 4, t = (1/4, 1/2, 3/4, 1) h, alpha = 1, v_j ~ N(0, 1) from seed 3, tol = 2^-53
(the precision configuration of the benchmark, eq. 1.2 with Algorithms 1 and 3).

The script calls only the oracle (Algorithm 1, then Algorithm 3 with the oracle's own xi and s) and
stores, per combination w_i:
  * the 2-norm of w_i,
  * w_i at SAMPLES seeded indices (numpy PCG64 seed 1234, plus the first and last rows),
  * the projections g_q . w_i on PROJ seeded N(0, 1) vectors (seeds 100 + q),
together with xi, s, the solve's counts and the oracle's run time.  A full-size parity test recomputes the
same indices and vectors and compares a GPU result with these values.

    python tests/golden/make_advdiff2d_1024.py 1e-5 1e-4 1e-3
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SAMPLES = 2048
PROJ = 4


def sample_indices(n: int) -> np.ndarray:
    idx = np.random.default_rng(1234).choice(n, size=SAMPLES, replace=False)
    return np.unique(np.concatenate([[0, n - 1], idx])).astype(np.int64)


def projection_vector(q: int, n: int) -> np.ndarray:
    return np.random.default_rng(100 + q).standard_normal(n)


def path_for(h: float) -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), f"advdiff2d_1024_h{h:g}.json")


def main(hs):
    import oracle
    from paper_2509_26475_gb300 import workloads as wl

    oracle.build()
    threads = oracle.set_threads(os.cpu_count() or 1)
    tol = 2.0**-53
    w = wl.workload_advdiff2d_1024(1.0, tol)
    A, V = w["A"], w["V"]
    t0 = time.perf_counter()
    sel = oracle.select(A, tol=tol)
    t_sel = time.perf_counter() - t0
    idx = sample_indices(A.n)
    G = [projection_vector(q, A.n) for q in range(PROJ)]
    for h in hs:
        t = [0.25 * h, 0.5 * h, 0.75 * h, h]
        t0 = time.perf_counter()
        W, st = oracle.solve(A, V, t, np.ones(4), tol, sel["s"], sel["xi"])
        t_solve = time.perf_counter() - t0
        rec = {
            "source": "oracle/ (Algorithm 1, then Algorithm 3 with its xi and s), written by "
                      "tests/golden/make_advdiff2d_1024.py",
            "workload": "2-D upwind advection-diffusion 1024^2 (n=1048576), Pe 1e3, p=4, r=4, "
                        "t=(1/4,1/2,3/4,1)h, alpha=1, v_j ~ N(0,1) seed 3, tol=2^-53",
            "h": h, "t": t, "n": int(A.n), "nnz": int(A.nnz),
            "select": {k: (float(v) if isinstance(v, float) else v) for k, v in sel.items() if k != "L"},
            "stats": {k: int(v) for k, v in st.items()},
            "oracle_seconds": {"select": t_sel, "solve": t_solve},
            "oracle_threads": threads, "oracle_host": f"{platform.machine()} {os.cpu_count()} cores",
            "sample_seed": 1234, "projection_seeds": [100 + q for q in range(PROJ)],
            "index": idx.tolist(),
            "norm2": [float(np.linalg.norm(W[i])) for i in range(4)],
            "values": [W[i, idx].tolist() for i in range(4)],
            "proj": [[float(G[q] @ W[i]) for q in range(PROJ)] for i in range(4)],
        }
        with open(path_for(h) + ".tmp", "w") as fh:
            json.dump(rec, fh)
        os.replace(path_for(h) + ".tmp", path_for(h))
        print(f"h={h:g}: s_int={st['s_int']} terms={st['series_terms']}+{st['recovery_terms']} "
              f"solve {t_solve:.1f} s", flush=True)


if __name__ == "__main__":
    main([float(x) for x in sys.argv[1:]] or [1e-5, 1e-4, 1e-3])
