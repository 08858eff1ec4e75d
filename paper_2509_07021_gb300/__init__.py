"""GB300-native (sm_103a) SG-splatting rasterizer: the data-parallel hot path of
MEGS^2 -- 3D Gaussians with a diffuse colour plus prunable, arbitrarily oriented
Spherical-Gaussian lobes, rendered forward and backward by hand-written CUDA
kernels behind a C ABI (include/sgsplat.h)."""
from . import synth  # noqa: F401
from .sgsplat import DeviceScene, SGError, sg_version  # noqa: F401


def __getattr__(name):
    if name in ("render_forward", "render_backward", "SGRasterize", "rasterize", "ForwardOut",
                "alloc_grads"):
        from . import render
        return getattr(render, name)
    raise AttributeError(name)
