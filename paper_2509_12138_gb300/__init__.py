"""GB300-native differentiable Gaussian-splat rasterizer for isosurface 3D-GS.

Hot path in libgs (hand-written sm_103a CUDA behind the C ABI in include/gs.h);
this package is the thin Python binding: buffer management, packing and the
torch.autograd wrapper.  Importing it does not load the library; the first
call that needs it does, and fails loudly if it cannot be built or loaded.
"""
from .raster import (Adam, Frame, LearningRates, Owned, RasterizeFunction, Units, pack_cameras, pack_params,
                     param_planes, rasterize, unpack_grads, unpack_params)

__all__ = ["Adam", "Frame", "LearningRates", "Owned", "RasterizeFunction", "Units", "pack_cameras", "pack_params",
           "param_planes", "rasterize", "unpack_grads", "unpack_params"]
