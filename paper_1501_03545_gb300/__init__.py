"""GB300-native generator of threshold random hyperbolic graphs.

The generator is the CUDA library libhrg.so (C ABI in include/hrg.h); this
package builds it in-tree (``build``), binds it with ctypes (``_lib``) and
holds the seeded workloads (``workloads``).  Importing the package does not
load the library; the first call does, and fails loudly if it cannot.
"""

__all__ = ["build", "workloads"]


def lib():
    from . import _lib

    return _lib
