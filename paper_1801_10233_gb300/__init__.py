"""GB300-native coupled spin-lattice dynamics (arXiv 1801.10233).

The hot path lives in libsl.so (CUDA, sm_103a) behind the C ABI of
include/sl.h; this package holds its build script, a ctypes binding and
the seeded input generators.
"""
from . import inputs
from ._lib import SlError, load, strerror, workspace_bytes

__all__ = ["System", "SlError", "inputs", "load", "strerror", "workspace_bytes"]


def __getattr__(name):
    if name == "System":
        from .system import System
        return System
    raise AttributeError(name)
