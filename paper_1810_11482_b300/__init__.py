"""B300 (sm_103a) heat-stencil library built on futures over CUDA streams.

The compute path lives in libhxc.so (C ABI: include/hxc.h); ``hxc`` is its
ctypes binding.  Importing this package does not load the library; the first
call into ``hxc`` does, and fails loudly if it has not been built.
"""
__all__ = ["hxc", "synth"]
