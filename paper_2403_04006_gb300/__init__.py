"""GB300-native permanents of matrices with repeated rows and columns,
boson-sampling probabilities and their gradients (after "Piquasso",
arXiv 2403.04006, Sec. 4.2 and Appendix A).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/pq.h``); ``pq`` is the ctypes binding with the same names and
``api`` the torch-facing layer (device batches, plans, autograd)."""
import importlib

from . import pq  # noqa: F401  (loads the library lazily, on first call)

__all__ = ["pq", "api", "workloads", "build"]


def __getattr__(name):
    if name in ("api", "workloads", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
