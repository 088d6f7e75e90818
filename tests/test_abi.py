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


def test_batch_argument_checks_before_any_device_work(lib):
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ns = np.array([3, 2], dtype=np.int64)
    off_de = np.array([0, 3], dtype=np.int64)
    off_z = np.array([0, 9], dtype=np.int64)
    d = np.zeros(5)
    e = np.ones(5)
    w = np.array([-1.0, 0.0, 1.0, -1.0, 1.0])
    Z = np.zeros(13)
    info = np.zeros(2, dtype=np.int64)
    assert lib.tinv_batch(-1, None, None, None, None, None, None, None, None, None) == -1
    assert lib.tinv_batch(0, None, None, None, None, None, None, None, None, None) == 0
    assert lib.tinv_batch(2, None, P(off_de), P(off_z), P(d), P(e), P(w), P(Z), P(info), None) == -2
    assert lib.tinv_batch(2, P(ns), None, P(off_z), P(d), P(e), P(w), P(Z), P(info), None) == -3
    assert lib.tinv_batch(2, P(ns), P(off_de), None, P(d), P(e), P(w), P(Z), P(info), None) == -4
    neg = np.array([3, -2], dtype=np.int64)
    assert lib.tinv_batch(2, P(neg), P(off_de), P(off_z), P(d), P(e), P(w), P(Z), P(info), None) == -2
    assert lib.tinv_batch(2, P(ns), P(off_de), P(off_z), None, P(e), P(w), P(Z), P(info), None) == -5
    assert lib.tinv_batch(2, P(ns), P(off_de), P(off_z), P(d), None, P(w), P(Z), P(info), None) == -6
    assert lib.tinv_batch(2, P(ns), P(off_de), P(off_z), P(d), P(e), None, P(Z), P(info), None) == -7
    assert lib.tinv_batch(2, P(ns), P(off_de), P(off_z), P(d), P(e), P(w), None, P(info), None) == -8
    o = binding.Opts()
    lib.tinv_opts_default(ctypes.byref(o))
    o.method = 3
    assert lib.tinv_batch(2, P(ns), P(off_de), P(off_z), P(d), P(e), P(w), P(Z), P(info),
                          ctypes.byref(o)) == -10
    # values are checked per problem: non-ascending w of problem 1, non-finite d of problem 0
    wbad = np.array([-1.0, 0.0, 1.0, 1.0, -1.0])
    assert lib.tinv_batch(2, P(ns), P(off_de), P(off_z), P(d), P(e), P(wbad), P(Z), P(info), None) == -7
    dbad = np.array([0.0, np.inf, 0.0, 0.0, 0.0])
    assert lib.tinv_batch(2, P(ns), P(off_de), P(off_z), P(dbad), P(e), P(w), P(Z), P(info), None) == -5
    # the workspace grows with the sum of n^2
    small = lib.tinv_batch_workspace_size(2, P(ns), None)
    big = lib.tinv_batch_workspace_size(2, P(np.array([300, 200], dtype=np.int64)), None)
    assert 0 < small < big


def test_bisect_argument_checks(lib):
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    d, e, w = np.zeros(3), np.ones(2), np.zeros(3)
    assert lib.tinv_bisect(-1, None, None, None, None) == -1
    assert lib.tinv_bisect(0, None, None, None, None) == 0
    assert lib.tinv_bisect(3, None, P(e), P(w), None) == -2
    assert lib.tinv_bisect(3, P(d), None, P(w), None) == -3
    assert lib.tinv_bisect(3, P(d), P(e), None, None) == -4
    assert lib.tinv_bisect(3, P(np.array([0.0, np.nan, 1.0])), P(e), P(w), None) == -2
    ns = np.array([3], dtype=np.int64)
    assert lib.tinv_bisect_batch(1, P(ns), None, P(d), P(e), P(w), None) == -3
    big = np.zeros(70000, dtype=np.int64)
    assert lib.tinv_bisect_batch(70000, P(big), P(big), P(d), P(e), P(w), None) == -106


def test_split_and_eig_argument_checks(lib):
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    d, e, w = np.zeros(3), np.ones(2), np.zeros(3)
    Z = np.zeros(9)
    isplit = np.zeros(3, dtype=np.int64)
    nb = ctypes.c_int64(-7)
    assert lib.tinv_split(-1, None, None, None, ctypes.byref(nb), None) == -1
    assert lib.tinv_split(0, None, None, None, ctypes.byref(nb), None) == 0 and nb.value == 0
    assert lib.tinv_split(3, None, P(e), P(isplit), ctypes.byref(nb), None) == -2
    assert lib.tinv_split(3, P(d), None, P(isplit), ctypes.byref(nb), None) == -3
    assert lib.tinv_split(3, P(d), P(e), None, ctypes.byref(nb), None) == -4
    assert lib.tinv_split(3, P(d), P(e), P(isplit), None, None) == -5
    assert lib.tinv_split(3, P(d), P(np.array([1.0, np.inf])), P(isplit), ctypes.byref(nb), None) == -3
    assert lib.tinv_eig(-1, None, None, None, None, 0, None, None, None, None) == -1
    assert lib.tinv_eig(0, None, None, None, None, 0, None, None, ctypes.byref(nb), None) == 0
    assert nb.value == 0
    assert lib.tinv_eig(3, None, P(e), P(w), P(Z), 3, None, None, None, None) == -2
    assert lib.tinv_eig(3, P(d), None, P(w), P(Z), 3, None, None, None, None) == -3
    assert lib.tinv_eig(3, P(d), P(e), None, P(Z), 3, None, None, None, None) == -4
    assert lib.tinv_eig(3, P(d), P(e), P(w), None, 3, None, None, None, None) == -5
    assert lib.tinv_eig(3, P(d), P(e), P(w), P(Z), 2, None, None, None, None) == -6
    assert lib.tinv_eig(3, P(np.array([0.0, np.nan, 1.0])), P(e), P(w), P(Z), 3, None, None,
                        None, None) == -2
    o = binding.Opts()
    lib.tinv_opts_default(ctypes.byref(o))
    o.method = 7
    assert lib.tinv_eig(3, P(d), P(e), P(w), P(Z), 3, None, None, None, ctypes.byref(o)) == -10


def test_bdsvd_argument_checks(lib):
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    a, b, s = np.ones(3), np.ones(2), np.zeros(3)
    U, V = np.zeros(9), np.zeros(9)
    assert lib.tinv_bdsvd(-1, None, None, None, None, 0, None, 0, None) == -1
    assert lib.tinv_bdsvd(0, None, None, None, None, 0, None, 0, None) == 0
    assert lib.tinv_bdsvd(3, None, P(b), P(s), P(U), 3, P(V), 3, None) == -2
    assert lib.tinv_bdsvd(3, P(a), None, P(s), P(U), 3, P(V), 3, None) == -3
    assert lib.tinv_bdsvd(3, P(a), P(b), None, P(U), 3, P(V), 3, None) == -4
    assert lib.tinv_bdsvd(3, P(a), P(b), P(s), None, 3, P(V), 3, None) == -5
    assert lib.tinv_bdsvd(3, P(a), P(b), P(s), P(U), 2, P(V), 3, None) == -6
    assert lib.tinv_bdsvd(3, P(a), P(b), P(s), P(U), 3, None, 3, None) == -7
    assert lib.tinv_bdsvd(3, P(a), P(b), P(s), P(U), 3, P(V), 2, None) == -8
    assert lib.tinv_bdsvd(3, P(np.array([1.0, np.nan, 1.0])), P(b), P(s), P(U), 3, P(V), 3,
                          None) == -2
    o = binding.Opts()
    lib.tinv_opts_default(ctypes.byref(o))
    o.method = 5
    assert lib.tinv_bdsvd(3, P(a), P(b), P(s), P(U), 3, P(V), 3, ctypes.byref(o)) == -9


def test_tune_argument_checks(lib):
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    d, e, w = np.zeros(4), np.ones(3), np.array([-1.5, -0.5, 0.5, 1.5])
    mt, ms, cached = ctypes.c_int32(7), ctypes.c_float(1.0), ctypes.c_int32(7)
    R = (ctypes.byref(mt), ctypes.byref(ms), ctypes.byref(cached))
    assert lib.tinv_tune(-1, None, None, 0, None, None, 1, *R) == -1
    assert lib.tinv_tune(4, None, P(e), 4, P(w), None, 1, *R) == -2
    assert lib.tinv_tune(4, P(d), None, 4, P(w), None, 1, *R) == -3
    assert lib.tinv_tune(4, P(d), P(e), 5, P(w), None, 1, *R) == -4
    assert lib.tinv_tune(4, P(d), P(e), 4, None, None, 1, *R) == -5
    assert lib.tinv_tune(4, P(d), P(e), 4, P(w[::-1].copy()), None, 1, *R) == -5
    assert lib.tinv_tune(4, P(np.array([0.0, np.inf, 0.0, 0.0])), P(e), 4, P(w), None, 1, *R) == -2
    o = binding.Opts()
    lib.tinv_opts_default(ctypes.byref(o))
    o.method = 3
    assert lib.tinv_tune(4, P(d), P(e), 4, P(w), ctypes.byref(o), 1, *R) == -6
    assert lib.tinv_tune(4, P(d), P(e), 4, P(w), None, 0, *R) == -7
    assert lib.tinv_tune(4, P(d), P(e), 4, P(w), None, 1, None, None, None) == -8
    # nothing to tune: order 0 or 1, or no eigenvalues; the outputs are reset
    assert lib.tinv_tune(0, None, None, 0, None, None, 1, *R) == 0
    assert (mt.value, ms.value, cached.value) == (0, 0.0, 0)
    assert lib.tinv_tune(1, P(np.array([2.0])), None, 1, P(np.array([2.0])), None, 1, *R) == 0
    assert lib.tinv_tune(4, P(d), P(e), 0, None, None, 1, *R) == 0
    lib.tinv_tune_clear()


def test_tune_cache_file_round_trip(lib, tmp_path):
    # the tune cache's file form needs no device: load, save, reload give the same entries
    tag = "# tinv tune cache v2\n"
    rows = ["0\tNVIDIA GB300\t152\t0\t0\t0\t4200\t4200\t14\t400\t0\t0\t171.894\n",
            "1\tNVIDIA GB300\t152\t0\t0\t0\t2100\t2100\t14\t200\t16\t8\t43.15\n",
            "0\tNVIDIA GB300\t152\t1\t0\t0\t210\t210\t14\t20\t0\t0\t3.5\n",
            "2\tNVIDIA GB300\t152\t0\t0\t0\t560000\t512\t123456789\t4096\t0\t8\t2100.5\n"]
    src, out, out2 = tmp_path / "a.txt", tmp_path / "b.txt", tmp_path / "c.txt"
    src.write_text(tag + "".join(rows))
    lib.tinv_tune_clear()
    assert lib.tinv_tune_load(str(src).encode()) == 4
    assert lib.tinv_tune_save(str(out).encode()) == 0
    text = out.read_text()
    assert text.startswith(tag) and sorted(text[len(tag):].splitlines()) == sorted(
        r.rstrip("\n") for r in rows)
    # the same entries again replace, they do not duplicate
    assert binding.tune_load(str(out)) == 4
    binding.tune_save(str(out2))
    assert out2.read_text() == text
    # a v1 file (no kind, no blocks) reads as tinv_tune entries with block 0
    v1 = tmp_path / "v1.txt"
    v1.write_text("# tinv tune cache v1\nNVIDIA GB300\t152\t0\t0\t4200\t4200\t14\t400\t4\t160.5\n")
    lib.tinv_tune_clear()
    assert lib.tinv_tune_load(str(v1).encode()) == 1
    assert lib.tinv_tune_save(str(out).encode()) == 0
    assert out.read_text() == tag + "0\tNVIDIA GB300\t152\t0\t0\t0\t4200\t4200\t14\t400\t4\t0\t160.5\n"
    # errors: NULL path, missing file, no tag line, a malformed entry (earlier entries kept)
    assert lib.tinv_tune_save(None) == -1 and lib.tinv_tune_load(None) == -1
    assert lib.tinv_tune_load(str(tmp_path / "missing.txt").encode()) == -2
    (tmp_path / "notag.txt").write_text("".join(rows))
    assert lib.tinv_tune_load(str(tmp_path / "notag.txt").encode()) == -2
    lib.tinv_tune_clear()
    bad = tmp_path / "bad.txt"
    for wrong in ("0\tNVIDIA GB300\t152\t0\t0\t0\t10\t20\t1\t2\t0\t0\t1.0\n",   # m > n
                  "0\tNVIDIA GB300\t152\t0\t0\t0\t10\t10\t1\t2\t0\t17\t1.0\n",  # block > 16
                  "3\tNVIDIA GB300\t152\t0\t0\t0\t10\t10\t1\t2\t0\t0\t1.0\n",   # unknown kind
                  "0\tNVIDIA GB300\t152\t0\t0\t0\t10\t10\t1\t2\t0\t0\n"):         # a field short
        bad.write_text(tag + rows[0] + wrong + rows[1])
        lib.tinv_tune_clear()
        assert lib.tinv_tune_load(str(bad).encode()) == -3, wrong
        assert lib.tinv_tune_save(str(out).encode()) == 0
        assert out.read_text() == tag + rows[0]
    lib.tinv_tune_clear()
    assert lib.tinv_tune_save(str(out).encode()) == 0 and out.read_text() == tag
    assert lib.tinv_tune_save(str(tmp_path / "no" / "such" / "dir.txt").encode()) == -2


def test_tune_auto_and_batch_argument_checks(lib):
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    t = binding.Tuning()
    d, e, w = np.zeros(4), np.ones(3), np.arange(4.0)
    T = ctypes.byref(t)
    assert lib.tinv_tune_auto(-1, None, None, 0, None, None, 1, T) == -1
    assert lib.tinv_tune_auto(4, None, P(e), 4, P(w), None, 1, T) == -2
    assert lib.tinv_tune_auto(4, P(d), P(e), 5, P(w), None, 1, T) == -4
    assert lib.tinv_tune_auto(4, P(d), P(e), 4, P(w[::-1].copy()), None, 1, T) == -5
    assert lib.tinv_tune_auto(4, P(d), P(e), 4, P(w), None, 0, T) == -7
    assert lib.tinv_tune_auto(4, P(d), P(e), 4, P(w), None, 1, None) == -8
    assert lib.tinv_tune_auto(0, None, None, 0, None, None, 1, T) == 0 and t.max_team == 0 and t.block == 0
    ns, off_de, off_z = binding.pack_offsets([4, 3])
    D, E, W = np.zeros(7), np.ones(7), np.r_[np.arange(4.0), np.arange(3.0)]
    args = lambda: [2, P(ns), P(off_de), P(off_z), P(D), P(E), P(W), None, 1, T]
    assert lib.tinv_tune_batch(-1, *args()[1:]) == -1
    a = args(); a[1] = None
    assert lib.tinv_tune_batch(*a) == -2
    a = args(); a[4] = None
    assert lib.tinv_tune_batch(*a) == -5
    W2 = W.copy(); W2[1] = -1.0  # problem 0 not ascending
    a = args(); a[6] = P(W2)
    assert lib.tinv_tune_batch(*a) == -7
    a = args(); a[8] = 0
    assert lib.tinv_tune_batch(*a) == -9
    a = args(); a[9] = None
    assert lib.tinv_tune_batch(*a) == -10
    assert lib.tinv_tune_batch(0, None, None, None, None, None, None, None, 1, T) == 0


def test_server_config_and_null_checks(lib):
    c = binding.ServerCfg()
    lib.tinv_server_cfg_default(ctypes.byref(c))
    assert (c.max_slots, c.max_inflight, c.hbm_fraction, c.method, c.max_pending) == \
        (4096, 4, 0.5, binding.TINV_CWY, 65536)
    assert ctypes.sizeof(binding.ServerCfg) == 64 and ctypes.sizeof(binding.Stats) == 184
    t = ctypes.c_uint64()
    d = np.zeros(3)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.tinv_submit(None, 3, P(d), P(d), None, P(d), 0, ctypes.byref(t)) == -1
    assert lib.tinv_poll(None, 1, None) == -1
    assert lib.tinv_wait(None, 1, 0, None) == -1
    assert lib.tinv_cancel(None, 1) == -1
    assert lib.tinv_server_destroy(None) == -1
    h = ctypes.c_void_p()
    assert lib.tinv_server_create(None, None) == -2
    bad = binding.ServerCfg()
    lib.tinv_server_cfg_default(ctypes.byref(bad))
    bad.hbm_fraction = 0.99
    assert lib.tinv_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1


def test_binding_refuses_missing_library(tmp_path):
    saved = binding._lib
    try:
        binding._lib = None
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "nope.so"))
    finally:
        binding._lib = saved
