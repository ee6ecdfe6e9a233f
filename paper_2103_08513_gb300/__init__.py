"""GB300 (sm_103a) implementation of the MRCM pressure solve (arXiv 2103.08513).

The compute path is libmrcm.so (hand-written CUDA behind a C ABI, see
include/mrcm.h); this package is its thin Python binding.
"""
from ._lib import MRCMError, load
from .build import build

__all__ = ["MRCM", "MRCMError", "build", "load"]


def __getattr__(name):
    if name == "MRCM":
        from .solver import MRCM
        return MRCM
    raise AttributeError(name)
