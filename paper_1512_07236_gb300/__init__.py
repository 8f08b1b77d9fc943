"""Generalized canonical purification (GCP/HPCP) on GB300.

The CUDA path lives behind the C ABI of ``libgcp.so`` (see include/gcp.h);
``paper_1512_07236_gb300.gcp`` is its ctypes binding.  Importing this
package does not load the library, so ``paper_1512_07236_gb300.inputs`` is
usable on machines without a GPU.
"""
import importlib

__all__ = ["gcp", "inputs"]


def __getattr__(name):
    if name in ("gcp", "inputs", "autograd"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
