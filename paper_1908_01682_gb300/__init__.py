"""GB300-native SPH-IDIC: one two-fluid SPH step with implicit drag in cell.

The compute path is the CUDA library ``libtfsph.so`` (sources in ``csrc/``,
C ABI in ``include/tfsph.h``); ``binding`` is its ctypes binding and
``build`` compiles it for sm_103a. There is no CPU fallback: using the
binding without the built library raises ImportError.
"""
from .binding import (Context, TfsphError, load, make_params, params_from_dict)  # noqa: F401

__all__ = ["Context", "TfsphError", "load", "make_params", "params_from_dict"]
