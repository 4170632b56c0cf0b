"""GB300-native (sm_103a) hot path of the GPU-screened diversified multi-start
method for the Unconstrained Binary Quadratic Problem (Lewis, arXiv 1706.00037).

The compute lives in ``libubqp.so`` (hand-written CUDA behind a C ABI declared
in ``include/ubqp.h``); ``paper_1706_00037_gb300.ubqp`` is its Python binding,
loaded on first use.  ``synth`` generates seeded synthetic instances.
"""
import importlib

__all__ = ["synth", "ubqp"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
