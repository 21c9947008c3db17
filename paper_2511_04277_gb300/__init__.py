"""GB300-native radiative hot path: MCRT view factors -> enforcement -> Gebhart REFs.

The work happens in libradgeb.so (hand-written CUDA for sm_103a behind the C ABI of
include/radgeb.h); ``api`` marshals torch tensors into those calls and ``autograd``
wraps the REF and temperature solves with their adjoints. Importing ``api`` without
the built library raises ImportError: there is no fallback.
"""
from .buildlib import LIB_PATH


def build(force: bool = False) -> str:
    """Compile libradgeb.so for sm_103a (in-tree); returns its path."""
    from . import buildlib
    return buildlib.build(force=force)


__all__ = ["build", "LIB_PATH", "api", "autograd"]


def __getattr__(name):
    if name in ("api", "autograd"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
