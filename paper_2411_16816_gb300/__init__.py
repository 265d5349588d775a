"""GB300-native SplatAD rasterizer: camera and lidar rendering of 3D Gaussians,
forward and backward, as hand-written sm_103a CUDA kernels behind a C ABI
(include/splat.h).  See :mod:`.render` for the torch-facing API."""
from . import scenes  # noqa: F401  (inputs only; no renderer arithmetic)

__all__ = ["scenes"]
