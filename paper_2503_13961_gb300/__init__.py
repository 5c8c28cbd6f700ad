"""GB300-native differentiable rasterizer for Bezier Gaussian Triangles.

Modules: `scenes` (seeded synthetic inputs), `render` (Renderer, render()),
`_abi` (ctypes binding of include/bgt.h), `build` (nvcc build of libbgt.so).
The CUDA library is loaded on first use of `render`; there is no CPU path.
"""

__all__ = ["scenes", "render", "build"]


def __getattr__(name):
    import importlib
    if name in ("scenes", "render", "build", "_abi"):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
