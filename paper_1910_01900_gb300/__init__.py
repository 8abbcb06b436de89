"""GB300-native matrix-free SIPG operator and cph hybrid multigrid (arXiv:1910.01900).

The compute lives in ``libsipg.so`` (CUDA, sm_103a), declared in
``include/sipg.h``; ``native`` is its ctypes binding.  Nothing here falls back
to a CPU implementation: without the built library every call raises.
"""
from .native import (Batch, Context, SipgError, create_unstructured, fma_peak, launch_count, lib,  # noqa: F401
                     operator_apply_noalloc)
