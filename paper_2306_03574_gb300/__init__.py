"""GB300-native all-at-once wave solver: ABAC-preconditioned MINRES (Lin & Hon).

The compute path is libaao.so (hand-written sm_103a CUDA behind a C ABI,
include/aao.h).  `paper_2306_03574_gb300.aao` is a thin ctypes binding with the
same names as the C entry points; PyTorch is used only for device memory and
streams.  There is no CPU fallback: if libaao.so is missing the binding raises.
"""
from .aao import *  # noqa: F401,F403
