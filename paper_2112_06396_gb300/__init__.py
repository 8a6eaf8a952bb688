"""GB300 (sm_103a) CKKS key-switching library: NTT/iNTT, ModUp, KSKInnerProd,
ModDown, Rescale, Automorph, KeySwitch, Rotate, HRotate and PtMatVecMult of
arXiv 2112.06396 as hand-written CUDA kernels behind a C ABI.

Importing the package does not load the CUDA library; ``ckks.lib()`` does, and
raises when it is missing (there is no CPU fallback).
"""
from . import build  # noqa: F401

__all__ = ["build", "ckks", "traffic"]
