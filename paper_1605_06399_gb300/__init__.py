"""GB300-native per-pixel stencil operators (ImageCL's method, arXiv 1605.06399).

The compute path is ``libimagecl.so`` (hand-written sm_103a CUDA behind the C ABI in
``include/imagecl.h``); this package only marshals arguments to it.  Build the library
with ``python -m paper_1605_06399_gb300.build``; calls fail loudly if it is missing.
"""
from .ops import (conv2d, sepconv, harris, default_variant, device_status, image, problem, tune, tune_clear,
                  tune_load, tune_model, tune_save, tune_set, variants, version)
from ._abi import ImclError
from . import autograd
from .ops import Batch, conv2d_backward, harris_backward, sepconv_backward

__all__ = ["conv2d", "sepconv", "harris", "default_variant", "device_status", "image", "problem", "tune", "tune_clear",
           "tune_load", "tune_model", "tune_save", "tune_set", "variants", "version", "ImclError", "autograd", "conv2d_backward",
           "sepconv_backward", "harris_backward", "Batch"]
