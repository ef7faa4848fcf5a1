"""GB300-native tile-based Gaussian splatting core (projection, tile sort,
front-to-back compositing of colour/depth/uncertainty, hand-written adjoint,
batched information gain over candidate views).

The CUDA library is loaded lazily on first use, so that importing the package
(e.g. for the scene generators) works on machines without a GPU.
"""
__all__ = ["scenes"]
