"""The diagnostic builds of the library compile and export the same C ABI as the product build
(CPU only; nothing is launched): the TINV_DEBUG variant with device bounds checks and the
phase-timing variant used by `python bench.py --phases`.  Each variant has
its own library file, so building one never replaces the product library."""
import ctypes
import os

import pytest

from paper_1209_1910_gb300 import binding, build


@pytest.mark.parametrize("variant", ["debug", "profile"])
def test_variant_builds_and_exports_the_abi(variant):
    product = build.build()
    before = os.path.getmtime(product)
    path = build.build(**{variant: True})
    assert os.path.basename(path) == {"debug": "libtinv_debug.so", "profile": "libtinv_prof.so"}[variant]
    assert os.path.getmtime(product) == before  # the product library is untouched
    lib = ctypes.CDLL(path)
    for name in binding.EXPORTS:
        assert hasattr(lib, name), (variant, name)
