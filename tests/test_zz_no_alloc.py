"""tinv_solve_noalloc: the shifted solve for callers that cannot have the library allocate
device memory (its scratch is a fixed device array inside the library).  Checked against
tinv_solve through the C ABI, on two calls in a row: the second call finds the first call's
contents in the scratch.  The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

from helpers import EPS
from paper_1209_1910_gb300 import inputs

pytestmark = pytest.mark.gpu

P = ctypes.c_void_p


def _cases():
    # (n, seed, shifts): a ragged size, the largest square case the scratch takes, a tiny one
    for n, seed, m in [(700, 3, 19), (512, 5, 512), (97, 7, 60)]:
        d, e = inputs.uniform(n, seed=seed)
        A = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        lam = np.linalg.eigvalsh(A)
        idx = np.linspace(0, n - 2, m).astype(int)
        shifts = 0.5 * (lam[idx] + lam[idx + 1])  # between neighbouring eigenvalues
        Y = np.random.default_rng(seed).uniform(-1, 1, (m, n))  # row j = right-hand side j
        check = list(range(0, m, max(1, m // 7)))
        cond = {j: np.linalg.cond(A - shifts[j] * np.eye(n)) for j in check}
        yield n, m, d, e, shifts, Y, cond


def test_solve_noalloc_matches_solve_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_1910_gb300 import binding, build

    build.build()
    lib = binding.load()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    for n, m, d, e, shifts, Y, cond in _cases():
        td, te, ts = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (d, e, shifts))
        for scale in (0, 1):
            ref = torch.from_numpy(Y).to(dev)
            o = binding._opts(device=True, stream=stream.cuda_stream)
            rc = lib.tinv_solve(n, P(td.data_ptr()), P(te.data_ptr()), m, P(ts.data_ptr()),
                                P(ref.data_ptr()), n, scale, ctypes.byref(o))
            assert rc == 0
            b = ref.cpu().numpy()
            for call in range(2):
                X = torch.from_numpy(Y).to(dev)
                rc = lib.tinv_solve_noalloc(n, P(td.data_ptr()), P(te.data_ptr()), m,
                                            P(ts.data_ptr()), P(X.data_ptr()), n, scale,
                                            P(stream.cuda_stream))
                assert rc == 0
                torch.cuda.synchronize()
                a = X.cpu().numpy()
                assert np.isfinite(a).all()
                # the bar of the solve parity tests: 50 cond(T - sI) eps max|x|
                for j, c in cond.items():
                    err = np.abs(a[j] - b[j]).max()
                    assert err <= 50 * c * EPS * np.abs(b[j]).max(), (n, scale, call, j)


def test_solve_noalloc_rejects_sizes_beyond_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_1910_gb300 import binding

    lib = binding.load()
    # m * n = 4096 * 128 exceeds the 262144 elements of the static scratch: refused with
    # TINV_ENOTSUP before any pointer is touched or any work is enqueued
    assert lib.tinv_solve_noalloc(4096, P(16), P(16), 128, P(16), P(16), 4096, 0, None) == -106


def test_solve_noalloc_padded_leading_dimension():
    # X with ldx > n: each column's rows n..ldx-1 hold a sentinel that must survive both calls,
    # and rows 0..n-1 must match tinv_solve on the unpadded right-hand sides
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_1910_gb300 import binding, build

    build.build()
    lib = binding.load()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    n, m, ldx, seed = 301, 40, 301 + 13, 11
    d, e = inputs.uniform(n, seed=seed)
    A = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    lam = np.linalg.eigvalsh(A)
    idx = np.linspace(0, n - 2, m).astype(int)
    shifts = 0.5 * (lam[idx] + lam[idx + 1])
    Y = np.random.default_rng(seed).uniform(-1, 1, (m, n))
    td, te, ts = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (d, e, shifts))
    ref = torch.from_numpy(Y).to(dev)
    o = binding._opts(device=True, stream=stream.cuda_stream)
    assert lib.tinv_solve(n, P(td.data_ptr()), P(te.data_ptr()), m, P(ts.data_ptr()),
                          P(ref.data_ptr()), n, 1, ctypes.byref(o)) == 0
    b = ref.cpu().numpy()
    sentinel = -7.25e33
    for call in range(2):
        Xp = np.full((m, ldx), sentinel)
        Xp[:, :n] = Y
        X = torch.from_numpy(Xp).to(dev)
        assert lib.tinv_solve_noalloc(n, P(td.data_ptr()), P(te.data_ptr()), m, P(ts.data_ptr()),
                                      P(X.data_ptr()), ldx, 1, P(stream.cuda_stream)) == 0
        torch.cuda.synchronize()
        a = X.cpu().numpy()
        assert np.all(a[:, n:] == sentinel), call
        for j in range(0, m, 5):
            c = np.linalg.cond(A - shifts[j] * np.eye(n))
            assert np.abs(a[j, :n] - b[j]).max() <= 50 * c * EPS * np.abs(b[j]).max(), (call, j)
