"""GB300-native inverse iteration with compact-WY reorthogonalization (arXiv:1209.1910).

The compute path is the CUDA library ``libtinv.so`` (C ABI declared in ``include/tinv.h``);
``paper_1209_1910_gb300.tinv`` is its thin ctypes binding.  Importing the package itself does
not load the library, so that ``paper_1209_1910_gb300.inputs`` can be used on machines
without a GPU.
"""
__all__ = ["inputs"]
