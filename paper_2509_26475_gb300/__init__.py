"""GB300-native solver for linear combinations of phi-function actions (Al-Mohy, arXiv 2509.26475).

    w_i = sum_{j=0}^{p} alpha_i^j phi_j(t_i A) v_j,   i = 1..r

The method runs in the CUDA library ``libphicomb.so`` (C ABI in ``include/phicomb.h``): Algorithm 1
(shift and scaling) and Algorithm 3 (block scaling-and-recovering Taylor method).  This package holds
the build step, a ctypes binding with the ABI's names (:mod:`.capi`), a PyTorch-facing API (:mod:`.api`)
and the seeded synthetic workloads (:mod:`.workloads`).  Importing it loads nothing; the library is
loaded on first use and its absence is an error.
"""

__version__ = "0.1.0"


def __getattr__(name):
    if name in ("api", "capi", "workloads", "build"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
