"""Full-size single problems of order 10^4 (one Peters-Wilkinson cluster of nearly all vectors):
the residual and orthogonality bounds on the whole result (products formed on the GPU), the closed form per
sampled vector for d=0, e=1, and the singletons of the uniform matrix against the oracle; one
member at a time and in blocks of 16 (the cluster on the whole grid, its staged vectors read from
the team's buffers in L2)."""
import math

import numpy as np
import pytest

from helpers import EPS, clusters_from_heads, singleton_equal
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


def _solve_on_device(gpu, d, e, w, block=0):
    import torch

    dev = torch.device("cuda:0")
    n = len(d)
    td, te, tw = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (d, e, w))
    Zt = torch.zeros((n, n), dtype=torch.float64, device=dev)  # row j = eigenvector j
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    gpu.tinv_device(td, te, tw, Zt, info=info, block=block)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    Z = Zt.T
    R = td[:, None] * Z
    R[:-1] += te[:, None] * Z[1:]
    R[1:] += te[:, None] * Z[:-1]
    R -= Z * tw[None, :]
    nrm = float(np.max(np.abs(d) + np.r_[0, np.abs(e)] + np.r_[np.abs(e), 0]))
    res = float(R.abs().max()) / (n * EPS * nrm)
    del R
    G = Zt @ Zt.T
    G.diagonal().sub_(1.0)
    orth = float(G.abs().max()) / (n * EPS)
    del G
    return Zt, res, orth


@pytest.mark.parametrize("block", [0, 16])
def test_toeplitz_zero_diagonal_10000_closed_form(gpu, block):
    n = 10000
    d, e = inputs.toeplitz(n, 0.0, 1.0)
    lam = np.sort(2.0 * np.cos(np.arange(1, n + 1) * math.pi / (n + 1)))
    Zt, res, orth = _solve_on_device(gpu, d, e, lam, block)
    assert res <= 10 and orth <= 10
    # sampled vectors against sin(i k pi / (n+1)), within the Davis-Kahan bound 4 |r| / gap
    i = np.arange(1, n + 1)
    for j in list(range(0, n, 997)) + [n - 1]:
        k = n - j  # ascending order: lambda_j = 2 cos(k pi / (n+1)) with k = n - j
        v = math.sqrt(2.0 / (n + 1)) * np.sin(i * k * math.pi / (n + 1))
        z = Zt[j].cpu().numpy()
        r = d * z
        r[:-1] += e * z[1:]
        r[1:] += e * z[:-1]
        r -= lam[j] * z
        gap = min(lam[j] - lam[j - 1] if j > 0 else np.inf, lam[j + 1] - lam[j] if j < n - 1 else np.inf)
        ang = np.linalg.norm(z - v * np.sign(z @ v))
        assert ang <= 4 * np.linalg.norm(r) / gap + 1e-13, j


@pytest.mark.parametrize("block", [0, 16])
def test_uniform_10000_invariants_and_singletons(gpu, orc, block):
    from scipy.linalg import eigvalsh_tridiagonal

    d, e = inputs.uniform(10000, seed=1)
    w = eigvalsh_tridiagonal(d, e)  # LAPACK's MRRR eigenvalues: any accurate w will do here
    Zt, res, orth = _solve_on_device(gpu, d, e, w, block)
    assert res <= 10 and orth <= 10
    head = orc.plan(d, e, w)[1]
    cl = clusters_from_heads(head)
    assert max(len(c) for c in cl) > 5000  # one giant cluster
    singles = [c[0] for c in cl if len(c) == 1][:8]
    assert singles
    for j in singles:
        zo, oinfo, *_ = orc.tinv(d, e, w[j:j + 1], "cwy", j0=j)
        assert oinfo == 0
        z = Zt[j].cpu().numpy()[:, None]
        assert singleton_equal(z, zo, 1e-10), j
