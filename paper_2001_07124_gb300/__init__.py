"""GB300-native randomized HOSVD / Tucker hot path (sm_103a CUDA + C ABI).

``build()`` compiles librhosvd.so in-tree; ``rhosvd`` is the Python binding of
its C ABI (include/rhosvd.h).  There is no CPU fallback: the binding raises if
the library is missing.
"""
from ._build import build  # noqa: F401
from . import rhosvd  # noqa: F401
from .rhosvd import (  # noqa: F401
    RhosvdError, Workspace, rhosvd_core, rhosvd_decompose, rhosvd_device_status, rhosvd_omega,
    rhosvd_orth, rhosvd_plan, rhosvd_power, rhosvd_primitive_workspace_size, rhosvd_sketch,
    rhosvd_sketch_all, rhosvd_workspace_size,
)
