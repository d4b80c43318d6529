"""B300-native Top-K feature rendering (LangGS-SLAM, Sec. 3.2).

The compute path is the CUDA library built from csrc/ (C ABI in include/gs_topk.h);
this package is its thin Python binding.  Importing it does not need a GPU; building
and loading the library does (loading raises if it was not built).
"""
from . import _abi  # noqa: F401
from .build import LIB_PATH, build  # noqa: F401

__all__ = ["TopKRenderer", "render", "build", "LIB_PATH"]


def __getattr__(name):
    if name in ("TopKRenderer", "render"):
        from . import renderer as _r
        return getattr(_r, name)
    raise AttributeError(name)
