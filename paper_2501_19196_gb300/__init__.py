"""GB300 (sm_103a) ray-traced Gaussian rendering -- the RaySplats path (arXiv 2501.19196).

The compute lives in libraysplats.so (hand-written CUDA behind the C ABI of
include/raysplats.h); this package only binds it.  Importing it does not load the library;
`native.load()` (called by Renderer) does, and raises if it is missing.
"""
from . import build, native  # noqa: F401

__all__ = ["build", "native", "Renderer", "RenderParams", "render_gaussians", "debug_rays", "ImageLoss",
           "TrainStep", "adam_step", "sigmoid", "sigmoid_backward"]


def __getattr__(name):
    if name in ("Renderer", "RenderParams", "render_gaussians", "debug_rays"):
        from . import renderer
        return getattr(renderer, name)
    if name in ("ImageLoss", "TrainStep", "adam_step", "sigmoid", "sigmoid_backward"):
        from . import train
        return getattr(train, name)
    raise AttributeError(name)
