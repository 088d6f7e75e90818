"""Parity of the split driver (tinv_split / tinv_eig through the C ABI) with the oracle's
split driver: the same blocks, bit-identical eigenvalues and block indices (bisection is
bit-exact), eigenvectors exactly zero outside their blocks and, inside each block, the same
vectors as the oracle's per-block inverse iteration (singletons within 1e-10 after the sign
convention, clusters by the largest principal angle <= 1e-10)."""
import numpy as np
import pytest

from helpers import clusters_from_heads, orth_ratio, residual_ratio, sin_angle, singleton_equal
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
    out = {}
    out["glued210_zero_glue"] = inputs.glued_wilkinson(10, 0.0)
    out["glued420_tiny_glue"] = inputs.glued_wilkinson(20, 1e-17)
    d, e = inputs.uniform(300, seed=5)
    e[[0, 30, 31, 150, 298]] = 0.0
    out["uniform300_cut"] = (d, e)
    out["uniform200_unsplit"] = inputs.uniform(200, seed=6)
    g = np.random.default_rng(3)
    out["diagonal64"] = (np.round(g.uniform(-4, 4, 64), 1), np.zeros(63))
    out["order1"] = (np.array([2.5]), np.zeros(0))
    out["order2_split"] = (np.array([1.0, -1.0]), np.zeros(1))
    return out


def _check(orc, d, e, w, Z, ib, isp, info, method="cwy"):
    wo, Zo, ibo, ispo, oinfo = orc.eig_split(d, e, method=method)
    assert info == 0 and oinfo == 0
    assert np.array_equal(isp, ispo)
    assert np.array_equal(w, wo)
    assert np.array_equal(ib, ibo)
    starts = np.r_[0, isp[:-1]]
    for b, (s, t) in enumerate(zip(starts, isp)):
        cols = np.nonzero(ib == b)[0]
        assert len(cols) == t - s
        assert np.all(Z[:s, cols] == 0.0) and np.all(Z[t:, cols] == 0.0)
        head = orc.plan(d[s:t], e[s:t - 1], w[cols])[1]
        for idx in clusters_from_heads(head):
            c = cols[idx]
            if len(idx) == 1:
                assert singleton_equal(Z[s:t, c], Zo[s:t, c], 1e-10), (b, c)
            else:
                assert sin_angle(Zo[s:t, c], Z[s:t, c]) <= 1e-10, (b, len(idx))


@pytest.mark.parametrize("case", sorted(_cases()))
def test_eig_matches_oracle(gpu, orc, case):
    d, e = _cases()[case]
    isp = gpu.split(d, e)
    assert np.array_equal(isp, orc.split(d, e))
    w, Z, ib, isp2, info = gpu.eig(d, e)
    assert np.array_equal(isp2, isp)
    _check(orc, d, e, w, Z, ib, isp2, info)
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10


def test_diagonal_is_an_exact_permutation(gpu):
    d, e = _cases()["diagonal64"]
    w, Z, ib, isp, info = gpu.eig(d, e)
    order = np.argsort(d, kind="stable")
    assert info == 0 and len(isp) == 64
    assert np.array_equal(ib, order)
    assert np.array_equal(Z, np.eye(64)[:, order])


def test_eig_mgs_and_iters(gpu, orc):
    d, e = inputs.glued_wilkinson(10, 0.0)
    iters = np.zeros(len(d), dtype=np.int32)
    w, Z, ib, isp, info = gpu.eig(d, e, method="mgs", iters=iters)
    _check(orc, d, e, w, Z, ib, isp, info, method="mgs")
    assert np.all((iters >= 1) & (iters <= 5))


def test_eig_leading_dimension_and_device_pointers(gpu):
    torch = pytest.importorskip("torch")
    d, e = _cases()["uniform300_cut"]
    n = len(d)
    w, Z, ib, isp, info = gpu.eig(d, e)
    w2, Z2, ib2, isp2, info2 = gpu.eig(d, e, ldz=n + 5)
    assert np.array_equal(w2, w) and np.array_equal(Z2, Z) and np.array_equal(ib2, ib)
    dev = torch.device("cuda:0")
    dd = torch.from_numpy(d).to(dev)
    de = torch.from_numpy(e).to(dev)
    dw = torch.zeros(n, dtype=torch.float64, device=dev)
    dZ = torch.zeros((n, n), dtype=torch.float64, device=dev)
    dib = torch.zeros(n, dtype=torch.int64, device=dev)
    info3, isp3 = gpu.eig_device(dd, de, dw, dZ, dib)
    assert info3 == 0 and np.array_equal(isp3, isp)
    assert np.array_equal(dw.cpu().numpy(), w)
    assert np.array_equal(dZ.cpu().numpy().T, Z)
    assert np.array_equal(dib.cpu().numpy(), ib)


def test_eig_full_size_zero_glue(gpu, orc):
    # the benchmark matrix with exactly zero glue: 200 independent W21+ blocks, no cluster spans
    # two blocks (unsplit, the same matrix has clusters of 200 and 400 members)
    d, e = inputs.glued_wilkinson(200, 0.0)
    w, Z, ib, isp, info = gpu.eig(d, e)
    assert len(isp) == 200
    _check(orc, d, e, w, Z, ib, isp, info)
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10


def test_split_device_pointers(gpu, orc):
    torch = pytest.importorskip("torch")
    d, e = _cases()["uniform300_cut"]
    dev = torch.device("cuda:0")
    isp = gpu.split_device(torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev))
    assert np.array_equal(isp, orc.split(d, e))


def test_eig_more_blocks_than_one_bisection_launch(gpu):
    # n = 70000 with every off-diagonal zero: 70000 blocks of order 1, more than one bisection
    # launch takes (65535 problems), and a 39 GB Z; the result must be the sorted diagonal and an
    # exact permutation matrix
    torch = pytest.importorskip("torch")
    n = 70000
    dev = torch.device("cuda:0")
    free, _ = torch.cuda.mem_get_info(dev)
    if free < 48 * 2**30:
        pytest.skip("needs ~40 GB of free device memory")
    g = np.random.default_rng(9)
    d = np.round(g.uniform(-50.0, 50.0, n), 3)
    td = torch.from_numpy(d).to(dev)
    te = torch.zeros(n - 1, dtype=torch.float64, device=dev)
    tw = torch.zeros(n, dtype=torch.float64, device=dev)
    tZ = torch.empty((n, n), dtype=torch.float64, device=dev)  # row j = eigenvector j
    tib = torch.zeros(n, dtype=torch.int64, device=dev)
    info, isp = gpu.eig_device(td, te, tw, tZ, tib)
    assert info == 0 and len(isp) == n
    order = np.argsort(d, kind="stable")
    assert np.array_equal(tib.cpu().numpy(), order)
    w = tw.cpu().numpy()
    assert np.abs(w - d[order]).max() <= 2 * np.finfo(float).eps * 50.0
    # each eigenvector is the unit vector of its block's row: one entry 1, all others 0
    assert torch.equal(tZ.argmax(dim=1).cpu(), torch.from_numpy(order))
    assert float(tZ.sum()) == float(n) and float(tZ.abs().max()) == 1.0
    del tZ
