"""GB300-native batched plain and cross-scale (zero-tree) OMP.

The compute lives in libcsp.so (CUDA, sm_103a) behind the C ABI of
include/csp.h.  This package holds the build script, the ctypes binding and a
context wrapper that passes torch tensors' device pointers and streams.
Importing the package does not load the library; ``Context`` does, and fails
loudly if it has not been built.
"""

__all__ = ["Context", "build", "load_library"]


def __getattr__(name):
    if name == "Context":
        from .context import Context
        return Context
    if name == "load_library":
        from ._binding import load_library
        return load_library
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
