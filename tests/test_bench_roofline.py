"""The roofline arithmetic of bench.py against the per-term figures the method's cost model fixes:
bytes (4 + b) nnz + 4 (n + 1) + 4 n w b and flops (2 nnz + 3 n) w per recovery Taylor term (w = 2r
columns, b bytes per value), evaluated for the benchmark operators (no GPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b

    return b


def test_recovery_term_bytes_and_flops(bench):
    # 1024^2 advection-diffusion (n = 1,048,576, nnz = 5,238,784, r = 4): 335.5 MB per FP64 term,
    # 180.3 MB per FP32 term, about 109 MFLOP per term
    n, nnz, wf = 1048576, 5238784, 8
    flops64, bytes64 = bench.recover_kernel_work(n, nnz, wf, 4, 4, 1, 0, 8)
    _, bytes32 = bench.recover_kernel_work(n, nnz, wf, 4, 4, 1, 0, 4)
    assert bytes64 / 1e6 == pytest.approx(335.5, abs=0.1)
    assert bytes32 / 1e6 == pytest.approx(180.3, abs=0.1)
    assert flops64 / 1e6 == pytest.approx(109.0, abs=0.5)
    # 64^3 convection-diffusion (n = 262,144, nnz = 1,810,432, r = 2): 56.4 MB per FP64 term
    _, b3 = bench.recover_kernel_work(262144, 1810432, 4, 3, 2, 1, 0, 8)
    assert b3 / 1e6 == pytest.approx(56.4, abs=0.1)


def test_terms_and_steps_scale_the_counts(bench):
    f1, b1 = bench.recover_kernel_work(1000, 5000, 4, 3, 2, 1, 0, 8)
    f7, b7 = bench.recover_kernel_work(1000, 5000, 4, 3, 2, 7, 0, 8)
    assert f7 == 7 * f1 and b7 == 7 * b1
    f_steps, _ = bench.recover_kernel_work(1000, 5000, 4, 3, 2, 7, 3, 8)
    assert f_steps == f7 + 3 * (1 + 3) * 1000 * 4  # the refresh of each outer step


def test_derived_fp64_figure_is_the_pipe_in_flops(bench):
    # context beside the measured roof: 2 FMA per clock per SM, 2 flops per FMA, 152 SMs, 2070 MHz
    assert bench.FP64_DERIVED_GFLOPS == pytest.approx(1258.56)


def test_select_kernel_bytes(bench):
    # Algorithm 1 with m = 61: 61 sparse products, the rescaling of r vectors and one pass over the 62
    # basis vectors per objective evaluation; on the 1024^2 operator a pass is 520 MB
    n, nnz = 1048576, 5238784
    spmv = 12 * nnz + 4 * (n + 1) + 16 * n
    assert bench.select_kernel_bytes(n, nnz, 61, 32, 0) == 61 * spmv + 16 * n * 32
    one_eval = bench.select_kernel_bytes(n, nnz, 61, 32, 1) - bench.select_kernel_bytes(n, nnz, 61, 32, 0)
    assert one_eval / 1e6 == pytest.approx(520.1, abs=0.1)


def test_default_line_is_the_1024_workload_in_fp64(bench):
    assert bench.WORKLOAD == "advdiff2d-1024" and bench.PRECISION == "f64"
    assert bench.HS == (1e-5, 1e-4) and (bench.P, bench.R) == (4, 4)
    # the oracle's timed sample on this workload is Algorithm 1 + the h = 1e-5 solve; the 64^3 step is whole
    assert bench.oracle_sample_hs() == (1e-5,)
    bench.configure("convdiff3d-64", "f64")
    try:
        assert bench.oracle_sample_hs() == (1e-4, 1e-2)
    finally:
        bench.configure("advdiff2d-1024", "f64")
