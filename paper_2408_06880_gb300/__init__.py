"""GB300-native sparse (indirect-addressing) lattice Boltzmann library.

The method (Suffa et al., Sec. 3.1 and Sec. 5.1): fluid cells compacted into a
direction-major PDF-list, a pull index-list with bounce-back folded in, and the
in-place AA even/odd stream-collide update with SRT, TRT, MRT, central-moment
and cumulant collisions, written as
hand-written CUDA for sm_103a behind the C ABI of include/sparse_lbm.h.
"""
from ._capi import (BF16, CM, CUMULANT, DENSE, FP16, FP32, MEM_DEVICE, MEM_HOST, ORDER_CELLS, ORDER_VOXELS,
                    MRT, ORDER_BRICK8, ORDER_HYBRID, ORDER_LEX, SPARSE, SPARSE_PULL, SRT, TRT, SlbmError, lib)
from .domain import Domain, TorchAllocator, auto_scale_exp
from .pool import Pool

__all__ = ["Domain", "Pool", "TorchAllocator", "auto_scale_exp", "SlbmError", "lib", "SRT", "MRT", "TRT", "CM", "CUMULANT", "FP32", "FP16",
           "BF16", "SPARSE", "SPARSE_PULL", "DENSE", "MEM_DEVICE", "MEM_HOST", "ORDER_CELLS", "ORDER_VOXELS", "ORDER_LEX", "ORDER_BRICK8", "ORDER_HYBRID"]
