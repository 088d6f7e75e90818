"""The CUDA library builds, loads and exports every function include/tinv.h declares; argument
checks that need no GPU reject bad input.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1209_1910_gb300 import binding, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "tinv.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tinv\w*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tinv" in names and "tinv_ex" in names and len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTS) == names


def test_opts_layout_matches_header(lib):
    o = binding.Opts()
    lib.tinv_opts_default(ctypes.byref(o))
    assert o.method == binding.TINV_CWY and o.device_ptrs == 0 and o.seed == 0
    assert ctypes.sizeof(binding.Opts) == 112


def test_strerror_and_version(lib):
    assert b"sm_103a" in lib.tinv_version()
    assert lib.tinv_strerror(0) == b"success"
    assert lib.tinv_strerror(-103) == b"a bounded device-side wait expired"
    assert lib.tinv_strerror(-3) == b"invalid argument"
    assert lib.tinv_strerror(2) == b"some eigenvectors did not converge"


def test_argument_checks_before_any_device_work(lib):
    d = np.zeros(4)
    e = np.ones(3)
    w = np.array([3.0, 1.0, 2.0, 4.0])  # not ascending
    Z = np.zeros((4, 4))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.tinv_ex(-1, None, None, 0, None, None, 1, None, None) == -1
    assert lib.tinv_ex(4, None, P(e), 4, P(w), P(Z), 4, None, None) == -2
    assert lib.tinv_ex(4, P(d), None, 4, P(w), P(Z), 4, None, None) == -3
    assert lib.tinv_ex(4, P(d), P(e), 5, P(w), P(Z), 4, None, None) == -4
    assert lib.tinv_ex(4, P(d), P(e), 4, P(w), P(Z), 3, None, None) == -7
    assert lib.tinv_ex(4, P(d), P(e), 4, P(w), P(Z), 4, None, None) == -5
    bad = np.array([0.0, np.nan, 1.0, 2.0])
    assert lib.tinv_ex(4, P(bad), P(e), 4, P(np.sort(w)), P(Z), 4, None, None) == -2
    o = binding.Opts()
    lib.tinv_opts_default(ctypes.byref(o))
    o.method = 7
    assert lib.tinv_ex(4, P(d), P(e), 4, P(np.sort(w)), P(Z), 4, ctypes.byref(o), None) == -8
    # n = 0 and m = 0 are no-ops
    assert lib.tinv_ex(0, None, None, 0, None, None, 1, None, None) == 0
    assert lib.tinv_ex(4, P(d), P(e), 0, None, None, 4, None, None) == 0
    # n = 1: Z = [1] without touching the device
    z1 = np.zeros(1)
    assert lib.tinv_ex(1, P(np.array([5.0])), None, 1, P(np.array([5.0])), P(z1), 1, None, None) == 0
    assert z1[0] == 1.0


def test_binding_refuses_missing_library(tmp_path):
    saved = binding._lib
    try:
        binding._lib = None
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "nope.so"))
    finally:
        binding._lib = saved
