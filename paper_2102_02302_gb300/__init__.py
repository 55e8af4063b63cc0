"""GB300-native Cleora propagation (arXiv 2102.02302): CUDA library + thin binding.

``libcleora.so`` (include/cleora.h) builds the transition matrix M = D^-1 A on the GPU,
fills the hash-seeded T_0 ~ U(-1, 1) and runs T_k = rownorm_L2(M T_{k-1}) with hand-written
sm_103a kernels.  This package only marshals arguments to it.
"""
from .cleora import *  # noqa: F401,F403
from .cleora import Batch, Context, CleoraError, Server, load  # noqa: F401
from . import build_native  # noqa: F401

__all__ = [n for n in dir() if n.startswith("cleora_")] + ["Batch", "Context", "CleoraError", "Server", "load",
                                                             "build_native"]
