"""GB300-native data-volume hot path of the Warpspeed metric estimator.

The product is the C-ABI shared library ``libwarpspeed.so`` (CUDA for sm_103a,
declared in ``include/warpspeed.h``); :mod:`.binding` is its thin ctypes binding and
:mod:`.workloads` describes seeded synthetic candidates.  The binding is imported
lazily so that describing workloads never loads CUDA.
"""
from importlib import import_module

__all__ = ["binding", "workloads", "build"]


def build(force: bool = False) -> str:
    """Compiles libwarpspeed.so in-tree (nvcc, -gencode arch=compute_103a,code=sm_103a)."""
    from . import _build
    return _build.build(force=force)


def __getattr__(name):
    if name in ("binding", "workloads", "_build"):
        return import_module(f".{name}", __name__)
    raise AttributeError(name)
