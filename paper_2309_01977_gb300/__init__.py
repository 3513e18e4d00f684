"""GB300-native SPECT projector and OSEM (PyTomography, arXiv 2309.01977).

``paper_2309_01977_gb300.spect`` is the thin ctypes binding of the C-ABI
library ``libspect.so`` (CUDA, sm_103a); ``phantom`` draws the seeded
synthetic inputs.  The binding is imported lazily so that the input
generators work on machines without the compiled library.
"""
import importlib

__all__ = ["autograd", "phantom", "spect"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
