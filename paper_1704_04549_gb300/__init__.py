"""GB300-native Kronecker-SVD preconditioned matrix-free GMRES for high-order DG.

The compute path is libtpp.so (CUDA, sm_103a) behind the C ABI of
include/tpp.h; this package only marshals arguments to it (ctypes) and uses
PyTorch for device memory and streams.  Importing ``Context`` loads the
library and fails loudly when it has not been built.
"""
from ._lib import (TPP_BF16, TPP_FEAT_BF16, TPP_FEAT_FULL_BLOCKS, TPP_FEAT_F32_SHIFTS, TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_LEARNED,
                   TPP_FEAT_MIXED, TPP_FEAT_TIME, TPP_FEAT_TWO_SIDED, TPP_FP32, TPP_FP64,
                   TPP_PC_BLOCK_JACOBI, TPP_PC_KRON,
                   TPP_PC_NONE, TPP_TS_BACKWARD_EULER, TPP_TS_DIRK3, TPP_TS_RK4, TppError)

__all__ = ["Context", "TppError", "TPP_FP64", "TPP_FP32", "TPP_BF16", "TPP_FEAT_BF16", "TPP_FEAT_FULL_BLOCKS", "TPP_FEAT_F32_SHIFTS", "TPP_PC_NONE", "TPP_PC_KRON",
           "TPP_PC_BLOCK_JACOBI", "TPP_FEAT_MIXED", "TPP_FEAT_BLOCK_JACOBI", "TPP_FEAT_TWO_SIDED",
           "TPP_FEAT_LEARNED", "TPP_FEAT_TIME", "TPP_TS_BACKWARD_EULER", "TPP_TS_DIRK3",
           "TPP_TS_RK4", "Mlp"]


def __getattr__(name):
    if name == "Context":
        from .solver import Context
        return Context
    if name == "Mlp":
        from .learned import Mlp
        return Mlp
    raise AttributeError(name)
