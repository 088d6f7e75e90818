"""Parity of tinv_bdsvd (singular triplets of a bidiagonal matrix through its Golub-Kahan form,
through the C ABI) with the oracle's bdsvd: bit-identical singular values (bisection of the
same T_GK), and the same singular vectors (per vector within 1e-10 where T_GK's plan gives a
singleton, by the largest principal angle <= 1e-10 inside clusters)."""
import numpy as np
import pytest

from helpers import EPS, clusters_from_heads, sin_angle

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


def _rand(n, seed):
    g = np.random.default_rng(seed)
    return g.uniform(0.5, 2.0, n) * g.choice([-1.0, 1.0], n), g.uniform(-1.0, 1.0, n - 1)


def _coupled(copies, blk, coupling, seed):
    a0, b0 = _rand(blk, seed)
    a = np.tile(a0, copies)
    b = np.concatenate([np.r_[b0, coupling]] * (copies - 1) + [b0])
    return a, b


def _cases():
    return {
        "random60": _rand(60, 7),
        "random500": _rand(500, 8),
        "coupled40": _coupled(4, 10, 1e-6, 11),
        "coupled400": _coupled(40, 10, 1e-6, 12),
        "diagonal8": (np.array([3.0, -1.0, 2.0, 0.5, -4.0, 1.5, 2.5, -0.25]), np.zeros(7)),
        "order1": (np.array([-2.5]), np.zeros(0)),
    }


def _check(orc, a, b, s, U, V, info, method="cwy"):
    so, Uo, Vo, oinfo = orc.bdsvd(a, b, method=method)
    assert info == 0 and oinfo == 0
    assert np.array_equal(s, so)
    d2, e2 = orc.golub_kahan(a, b)
    head = orc.plan(d2, e2, s)[1]
    for idx in clusters_from_heads(head):
        if len(idx) == 1:
            assert np.abs(U[:, idx] - Uo[:, idx]).max() <= 1e-10, idx
            assert np.abs(V[:, idx] - Vo[:, idx]).max() <= 1e-10, idx
        else:
            assert sin_angle(Uo[:, idx], U[:, idx]) <= 1e-10, (idx[0], len(idx))
            assert sin_angle(Vo[:, idx], V[:, idx]) <= 1e-10, (idx[0], len(idx))
    n = len(a)
    B = np.diag(a) + np.diag(b, 1)
    nrm = np.abs(B).sum(axis=0).max()
    assert np.abs(B @ V - U * s).max() <= 10 * n * EPS * nrm
    assert np.abs(B.T @ U - V * s).max() <= 10 * n * EPS * nrm
    assert np.abs(U.T @ U - np.eye(n)).max() <= 10 * n * EPS
    assert np.abs(V.T @ V - np.eye(n)).max() <= 10 * n * EPS


@pytest.mark.parametrize("case", sorted(_cases()))
def test_bdsvd_matches_oracle(gpu, orc, case):
    a, b = _cases()[case]
    s, U, V, info = gpu.bdsvd(a, b)
    _check(orc, a, b, s, U, V, info)


def test_bdsvd_mgs_and_device_pointers(gpu, orc):
    torch = pytest.importorskip("torch")
    a, b = _cases()["coupled40"]
    s, U, V, info = gpu.bdsvd(a, b, method="mgs")
    _check(orc, a, b, s, U, V, info, method="mgs")
    n = len(a)
    dev = torch.device("cuda:0")
    ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    ts = torch.zeros(n, dtype=torch.float64, device=dev)
    tU = torch.zeros((n, n), dtype=torch.float64, device=dev)
    tV = torch.zeros((n, n), dtype=torch.float64, device=dev)
    assert gpu.bdsvd_device(ta, tb, ts, tU, tV, method="mgs") == 0
    assert np.array_equal(ts.cpu().numpy(), s)
    assert np.array_equal(tU.cpu().numpy().T, U) and np.array_equal(tV.cpu().numpy().T, V)
