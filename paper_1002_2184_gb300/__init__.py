"""GB300-native Fast Haar wavelet transform (arXiv:1002.2184).

The transforms run in libfasthaar.so (hand-written CUDA for sm_103a, C ABI in
include/fasthaar.h); this package is its thin PyTorch binding.  Importing it
does not load the library: the first call does, and fails loudly when it has
not been built.
"""
_API = ("dwt1d", "idwt1d", "dwt2d", "idwt2d", "describe", "workspace_size")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)


__all__ = list(_API)
