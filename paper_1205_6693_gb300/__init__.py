"""GB300-native (sm_103a) exact truss decomposition.

The compute path is the CUDA library ``libtruss.so`` built from ``csrc/``
(C ABI in ``include/truss.h``); :mod:`.truss` is its ctypes binding.
"""
from .truss import (Context, TrussError, truss_ctx_create, truss_ctx_destroy,  # noqa: F401
                    truss_decompose, truss_decompose_batch, truss_last_stats,
                    truss_strerror, truss_support)
