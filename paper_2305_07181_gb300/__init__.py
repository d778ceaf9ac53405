"""GB300-native entropy-split SBP-SAT residual (Euler / compressible Navier-Stokes).

The compute path is the CUDA library ``_lib/libesplit.so`` (C ABI in
``include/esplit.h``); this package only marshals arguments to it.  Using any
of ``Solver``, ``Params``, ``EsplitError`` or ``capi`` without the built
library raises ImportError: there is no fallback.  ``build`` compiles it.
"""
import importlib

__all__ = ["Solver", "Params", "EsplitError", "capi", "build"]


def __getattr__(name):
    if name in ("Solver", "Params", "EsplitError"):
        return getattr(importlib.import_module(".solver", __name__), name)
    if name in ("capi", "build", "solver"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
