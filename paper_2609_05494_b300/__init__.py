"""B300-native (sm_103a) planar WCSPH hydrodynamic-ram step.

The hot path (neighbour search, Adami ghosts, fused interaction sums, Tait
EOS, kick-drift-kick integrator with the CFL gate, probes, FP64 diagnostics)
runs in the CUDA kernels of ``libhram.so`` behind the C-ABI of
include/hram.h; this package is its Python binding.
"""
from .api import (Batch, Case, DIAG_FIELDS, KERNEL_GROUPS, SCALAR_FIELDS, TANGENT_PARAMS,  # noqa: F401
                  fp32_rate, make_params)
from .grad import jacobian, peak_and_impulse  # noqa: F401
from ._lib import HramError, lib  # noqa: F401
