"""GPU Sturm bisection (tinv_bisect, tinv_bisect_batch) against the oracle's bisection.

Both sides evaluate the same sequence of IEEE round-to-nearest operations (Sturm pivots, bracket
test, midpoint), so the eigenvalue approximations must agree bit for bit."""
import numpy as np
import pytest

from paper_1209_1910_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_1910_gb300 import binding, build

    build.build()
    binding.load()
    return binding


def _cases():
    out = []
    out.append(inputs.uniform(1000, seed=1))
    out.append(inputs.glued_wilkinson(20, 1e-10))
    out.append(inputs.toeplitz(500, 2.0, 1.0))
    out.append(inputs.toeplitz(300, 0.0, 1.0))
    out.append((np.array([3.0]), np.zeros(0)))
    out.append((np.array([1.0, 1.0]), np.array([1.0])))
    out.append((np.zeros(5), np.zeros(4)))  # T = 0
    d, e = inputs.uniform(200, seed=5)
    e[[10, 50, 51, 120]] = 0.0  # exact splits
    out.append((d, e))
    d, e = inputs.uniform(150, seed=6)
    out.append((d * 1e150, e * 1e-150))  # tiny off-diagonal against a huge diagonal
    out.append((d * 1e-300, e * 1e-300))  # subnormal range
    return out


def test_bisect_bit_exact(gpu, orc):
    for d, e in _cases():
        w = gpu.bisect(d, e)
        wo = orc.bisect(d, e)
        assert np.array_equal(w, wo), len(d)
        assert np.all(np.diff(w) >= 0)


def test_bisect_toeplitz_closed_form(gpu):
    n = 500
    d, e = inputs.toeplitz(n, 2.0, 1.0)
    lam = inputs.toeplitz_eigenpairs(n, 2.0, 1.0)[0]
    w = gpu.bisect(d, e)
    assert np.abs(w - lam).max() <= 4 * np.finfo(float).eps * 4.0


def test_bisect_batch_device_matches_single(gpu, orc):
    import torch

    sizes = [64, 0, 1, 333, 21 * 7, 1000]
    probs = []
    for q, n in enumerate(sizes):
        if q == 4:
            probs.append(inputs.glued_wilkinson(7, 1e-10))
        else:
            probs.append(inputs.uniform(n, seed=40 + q))
    ns = np.array([len(p[0]) for p in probs], dtype=np.int64)
    off = np.zeros(len(ns), dtype=np.int64)
    a = 2
    for q, n in enumerate(ns):
        off[q] = a
        a += n + 3
    D = np.zeros(a)
    E = np.zeros(a)
    for q, (d, e) in enumerate(probs):
        D[off[q]:off[q] + len(d)] = d
        E[off[q]:off[q] + len(e)] = e
    dev = torch.device("cuda:0")
    td, te = torch.from_numpy(D).to(dev), torch.from_numpy(E).to(dev)
    tw = torch.full((a,), 5.0, dtype=torch.float64, device=dev)
    gpu.bisect_batch_device(ns, off, td, te, tw)
    torch.cuda.synchronize()
    W = tw.cpu().numpy()
    for q, (d, e) in enumerate(probs):
        n = len(d)
        if n == 0:
            continue
        assert np.array_equal(W[off[q]:off[q] + n], orc.bisect(d, e)), q
