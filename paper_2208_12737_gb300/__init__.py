"""GB300-native differentiable DRRs: Siddon ray tracing of CT volumes on sm_103a.

The compute path is the CUDA library ``libdrr`` (C ABI declared in
``include/drr.h``); :mod:`paper_2208_12737_gb300.drr` is its ctypes binding and
``torch.autograd.Function`` wrapper.  Importing this package does not load the
library; the binding loads it on first use and raises if it is missing.
"""
__all__ = ["inputs"]
