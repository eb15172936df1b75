"""GB300-native exhaustive Kron-based reduction of three-phase radial feeders.

The computation lives in ``libokron.so`` (CUDA, sm_103a) behind the C ABI in
``include/okron.h``; this package holds the build script and a ctypes binding
with the same entry points.  The algorithm is Algorithm 1 of arXiv 2510.19608
(Sec. IV), with the Kron reduction of Sec. II-B and the error model of Sec. III.
"""
from ._binding import (Context, Feeder, IncShape, OkrError, Params, Result, Summary,  # noqa: F401
                       default_params, device_feeder, lib, lib_path, power_flow_static)

__all__ = ["Context", "Feeder", "IncShape", "OkrError", "Params", "Result", "Summary", "default_params",
           "device_feeder", "lib", "lib_path", "power_flow_static"]
