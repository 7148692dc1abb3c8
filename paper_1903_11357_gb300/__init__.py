"""dgasm: SIPG + two-level non-overlapping additive Schwarz PCG on one GB300 GPU (sm_103a).

The numerical work runs in libdgasm.so (CUDA kernels behind the C-ABI of include/dgasm.h);
``paper_1903_11357_gb300.dgasm`` is its ctypes binding.
"""
from . import dgasm  # noqa: F401
from .build import build  # noqa: F401
