"""The synthetic operators that select each copy format of B in the GPU format tests, checked on the
host: their structure must fall where the setup's format rules send it (DIA for at most 16 diagonals
filling the rows, ELL when n times the longest row fits nnz + nnz/4 + 64, CSR otherwise)."""
import numpy as np

from paper_2509_26475_gb300 import workloads as wl


def _structure(A):
    lens = np.diff(A.rowptr)
    rows = np.repeat(np.arange(A.n), lens)
    offsets = np.unique(A.colidx - rows)
    return lens, offsets


def _dense(A):
    M = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    np.add.at(M, (rows, A.colidx), A.values)
    return M


def test_graph_operator_is_symmetric_negative_definite_with_scattered_diagonals():
    A = wl.graph_operator(600, 6, 11)
    M = _dense(A)
    assert np.allclose(M, M.T)
    ev = np.linalg.eigvalsh(M)
    assert ev.max() <= -1.0 + 1e-9  # -(L + I) with L positive semidefinite
    lens, offsets = _structure(A)
    assert len(offsets) > 16  # too many diagonals for the DIA copy
    assert lens.max() <= 64 and lens.max() * A.n <= A.nnz + A.nnz // 4 + 64  # fits the ELL copy


def test_graph_operator_with_hubs_needs_csr_order():
    A = wl.graph_operator(2600, 6, 12, hubs=20, hub_degree=80)
    lens, offsets = _structure(A)
    assert len(offsets) > 16
    assert lens.max() > 64  # longer than the ELL copy's slots


def test_stencils_fall_in_the_dia_rule():
    for A, nd in ((wl.convection_diffusion(37, 2, 6.0), 5), (wl.convection_diffusion(13, 3, 6.0), 7),
                  (wl.convection_diffusion(1500, 1, 6.0), 3)):
        lens, offsets = _structure(A)
        assert len(offsets) == nd
        assert nd * A.n <= A.nnz + A.nnz // 2 + 64  # the DIA cells fill the rows well
