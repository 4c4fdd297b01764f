"""GB300-native (sm_103a) t-product library: Python binding.

The compute path lives in ``libtprod.so`` (CUDA kernels behind a C ABI,
declared in include/tprod.h).  This package only marshals arguments: it
checks shapes and layouts of torch CUDA tensors and passes raw device
pointers and the current CUDA stream to the C entry points.  There is no CPU
fallback: when the library is missing every entry point raises.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401
