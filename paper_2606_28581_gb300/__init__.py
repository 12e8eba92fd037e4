"""GB300-native affine 2D-Gaussian-splat rasterizer (SatSplat hot path).

The compute path is the CUDA library ``_build/libsatsplat.so`` (hand-written
kernels for sm_103a) behind the C ABI in ``include/satsplat.h``; this package
is its thin Python binding plus the training forms built on it:

  * ``_lib``      ctypes binding, one function per C entry point
  * ``frame``     workspace / output management for one frame of targets
  * ``autograd``  torch.autograd.Function (form a) with BF16 storage (form c)
  * ``batched``   many views + sun views in one persistent launch, captured in a
                  CUDA graph, with a tile-shape / batch autotuner (form b)
"""
from . import _lib
from ._lib import SS_PASS_MAIN, SS_PASS_SUN, SatSplatError, default_opts, load
__all__ = ["_lib", "SS_PASS_MAIN", "SS_PASS_SUN", "SatSplatError", "default_opts", "load"]
