"""GB300-native sequential phase linking (SHP/GLRT, coherence, EMI, temporal
coherence, compressed SLCs) behind the C ABI declared in include/plk.h.

Importing the package loads nothing; the CUDA library is loaded on first use of
`paper_2511_12051_gb300.plk` and every call fails loudly if it is missing.
"""
import importlib

__all__ = ["synth", "plk"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
