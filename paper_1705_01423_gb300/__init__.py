"""GB300-native pressure-correction path of AFiD (arXiv 1705.01423).

The compute lives in libafid.so (CUDA kernels for sm_103a behind the C ABI of
include/afid.h); `afid` is its ctypes binding and `autodiff` wraps the
hand-written adjoints as torch.autograd Functions with a checkpointed rollout.
"""
from .afid import Context, MultiRes, Physics, AfidError, lib, LIB_PATH, exported_symbols  # noqa: F401
from . import autodiff  # noqa: F401

__all__ = ["Context", "MultiRes", "Physics", "AfidError", "lib", "LIB_PATH", "exported_symbols"]
