"""GB300-native spectral-element elliptic solver path (NekRS, Sections 2.3 and 3.2-3.4).

The compute lives in libsem.so (CUDA, sm_103a); this package holds its build
script and a thin Python binding. Nothing here falls back to the CPU: if the
library is not built, every call raises.
"""
from ._lib import SemError, load  # noqa: F401
from .sem import Projection, SemContext, default_opts, gll, measure_peaks  # noqa: F401

__all__ = ["Projection", "SemContext", "SemError", "default_opts", "gll", "load", "measure_peaks"]
