"""Failure detection without a GPU (CPU only): on a machine with no CUDA device every compute entry
point of the C ABI returns TINV_ENODEV after its argument checks -- no crash, no hang, no partial
write to the caller's outputs -- and the Python binding raises it as a TinvError.  Skipped where a
device is present, since the calls would then do real work."""
import ctypes

import numpy as np
import pytest

from paper_1209_1910_gb300 import binding, build

ENODEV = -107


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    build.build()
    return binding.load()


def test_every_compute_entry_point_reports_no_device(lib):
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    n, m = 8, 2
    d = np.linspace(-1.0, 1.0, n)
    e = np.full(n - 1, 0.3)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    w = np.linalg.eigvalsh(T)
    s = w[:m].copy()
    Z = np.full(n * n, 7.0)
    isp = np.zeros(n, dtype=np.int64)
    ib = np.zeros(n, dtype=np.int64)
    nb = ctypes.c_int64(-1)
    ns = np.array([n], dtype=np.int64)
    off = np.zeros(1, dtype=np.int64)
    info = np.zeros(1, dtype=np.int64)
    f = [np.zeros(m * n) for _ in range(4)]
    piv = np.zeros(m * n, dtype=np.uint8)
    X = np.ones(n * m)
    V = np.random.default_rng(0).standard_normal(n * m)
    mt = ctypes.c_int32(5)
    calls = {
        "tinv": lambda: lib.tinv(n, P(d), P(e), P(w), P(Z)),
        "tinv_ex": lambda: lib.tinv_ex(n, P(d), P(e), n, P(w), P(Z), n, None, None),
        "tinv_batch": lambda: lib.tinv_batch(1, P(ns), P(off), P(off), P(d), P(e), P(w), P(Z),
                                             P(info), None),
        "tinv_bisect": lambda: lib.tinv_bisect(n, P(d), P(e), P(np.zeros(n)), None),
        "tinv_bisect_batch": lambda: lib.tinv_bisect_batch(1, P(ns), P(off), P(d), P(e),
                                                           P(np.zeros(n)), None),
        "tinv_split": lambda: lib.tinv_split(n, P(d), P(e), P(isp), ctypes.byref(nb), None),
        "tinv_eig": lambda: lib.tinv_eig(n, P(d), P(e), P(np.zeros(n)), P(Z), n, P(ib), P(isp),
                                         ctypes.byref(nb), None),
        "tinv_bdsvd": lambda: lib.tinv_bdsvd(n, P(d), P(e), P(np.zeros(n)), P(Z), n,
                                             P(np.zeros(n * n)), n, None),
        "tinv_plan": lambda: lib.tinv_plan(n, P(d), P(e), n, P(w), P(np.zeros(n)),
                                           P(np.zeros(n, dtype=np.int32)), P(np.zeros(3)), None),
        "tinv_lu": lambda: lib.tinv_lu(n, P(d), P(e), m, P(s), *[P(x) for x in f], P(piv), None),
        "tinv_solve": lambda: lib.tinv_solve(n, P(d), P(e), m, P(s), P(X), n, 0, None),
        "tinv_solve_noalloc": lambda: lib.tinv_solve_noalloc(n, P(d), P(e), m, P(s), P(X), n, 0,
                                                             None),
        "tinv_orth": lambda: lib.tinv_orth(n, m, P(V), n, P(np.zeros(n * m)), n, None, None,
                                           None),
        "tinv_tune": lambda: lib.tinv_tune(n, P(d), P(e), n, P(w), None, 1, ctypes.byref(mt),
                                           None, None),
        "tinv_tune_auto": lambda: lib.tinv_tune_auto(n, P(d), P(e), n, P(w), None, 1,
                                                     ctypes.byref(binding.Tuning())),
        "tinv_tune_batch": lambda: lib.tinv_tune_batch(
            1, P(np.array([n], dtype=np.int64)), P(np.zeros(1, dtype=np.int64)),
            P(np.zeros(1, dtype=np.int64)), P(d), P(e), P(w), None, 1, ctypes.byref(binding.Tuning())),
    }
    for name, call in calls.items():
        assert call() == ENODEV, name
    assert np.all(Z == 7.0)  # nothing written
    h = ctypes.c_void_p()
    cfg = binding.ServerCfg()
    lib.tinv_server_cfg_default(ctypes.byref(cfg))
    assert lib.tinv_server_create(ctypes.byref(cfg), ctypes.byref(h)) == ENODEV
    assert not h.value
    assert b"device" in lib.tinv_strerror(ENODEV)
    # the workspace query is host arithmetic and needs no device
    assert lib.tinv_workspace_size(n, n, None) > 0


def test_binding_raises_the_code(lib):
    d = np.linspace(-1.0, 1.0, 6)
    e = np.full(5, 0.3)
    with pytest.raises(binding.TinvError) as ex:
        binding.tinv(d, e, np.linspace(-1.0, 1.0, 6))
    assert ex.value.code == ENODEV
