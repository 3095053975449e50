"""GB300 (sm_103a) differentiable 2D Gaussian surfel rasterizer -- the
data-parallel hot path of Flash-Mono's mapping backend (render + refine).

The compute lives in libsplat2d (CUDA, C ABI in include/splat2d.h); this
package is its Python binding.  Importing the package does not touch the
GPU; the library is built/loaded on first use and any failure raises.
"""
from . import scenes  # noqa: F401  (inputs only; no rasterizer arithmetic)

__all__ = ["scenes", "RasterConfig", "Rasterizer", "Splat2DRender", "render", "load_library"]


def load_library():
    from . import _abi
    return _abi.load()


def __getattr__(name):
    if name in ("RasterConfig", "Rasterizer", "Splat2DRender", "render", "Images", "SurfelGrads"):
        from . import rasterizer
        return getattr(rasterizer, name)
    raise AttributeError(name)
