"""Batched path (tinv_batch): many independent problems of uneven order in one launch sequence.

Each problem of a batch must meet the same bars as a single call (residual and orthogonality
invariants, singletons per vector and clusters by subspace angle against the oracle), and must
be the same alone and in the mix: with one CTA per cluster (MGS, or compact WY without teams)
the arithmetic of every cluster is the same in both, so the vectors are bit-identical; with CTA
teams the reduction shapes differ and the subspaces agree within 1e-10.
"""
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


def _problems(sizes, seed=11):
    probs = []
    for q, n in enumerate(sizes):
        if n == 0:
            probs.append((np.zeros(0), np.zeros(0), np.zeros(0)))
            continue
        if q % 2 == 1 and n % 21 == 0:
            d, e = inputs.glued_wilkinson(n // 21, 1e-10)
        else:
            d, e = inputs.uniform(n, seed=seed * 1000 + q)
        probs.append((d, e, inputs.eigenvalues(d, e)))
    return probs


SIZES = [1, 2, 7, 21, 64, 105, 200, 420, 333, 63, 1000, 210]


def _compare(Z, Zo, head, tol=1e-10):
    for idx in clusters_from_heads(head):
        if len(idx) == 1:
            assert singleton_equal(Z[:, idx[0]], Zo[:, idx[0]], tol), idx[0]
        else:
            assert sin_angle(Zo[:, idx], Z[:, idx]) <= tol, (idx[0], len(idx))


@pytest.mark.parametrize("method", ["cwy", "mgs"])
def test_batch_matches_oracle(gpu, orc, method):
    probs = _problems(SIZES)
    Zs, rc, info, iters = gpu.tinv_batch([p[0] for p in probs], [p[1] for p in probs],
                                         [p[2] for p in probs], method=method, return_info=True)
    assert rc == 0 and np.all(info == 0)
    assert np.all((iters >= 1) & (iters <= 5))
    for (d, e, w), Z in zip(probs, Zs):
        n = len(d)
        if n == 1:
            assert Z.tolist() == [[1.0]]
            continue
        assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10, n
        Zo, oinfo, *_ = orc.tinv(d, e, w, method)
        assert oinfo == 0
        _compare(Z, Zo, orc.plan(d, e, w)[1])


@pytest.mark.parametrize("method,max_team", [("mgs", 0), ("cwy", 1)])
def test_batch_bit_identical_to_single_calls(gpu, method, max_team):
    probs = _problems(SIZES, seed=12)
    Zs = gpu.tinv_batch([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                        method=method, max_team=max_team)
    for (d, e, w), Z in zip(probs, Zs):
        Z1 = gpu.tinv(d, e, w, method=method, max_team=max_team)
        assert np.array_equal(Z, Z1), len(d)


def test_batch_with_teams_matches_single_calls(gpu):
    # one large glued problem (teams) among small ones
    probs = _problems([64, 2100, 97, 420], seed=13)
    Zs = gpu.tinv_batch([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs])
    for (d, e, w), Z in zip(probs, Zs):
        Z1 = gpu.tinv(d, e, w)
        assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
        wp, head, _ = gpu.plan(d, e, w)  # clusters of the single call's plan
        for idx in clusters_from_heads(head):
            if len(idx) == 1:
                assert singleton_equal(Z[:, idx[0]], Z1[:, idx[0]], 1e-10)
            else:
                assert sin_angle(Z1[:, idx], Z[:, idx]) <= 1e-10


def test_batch_device_pointers_with_gaps(gpu):
    import torch

    probs = _problems([50, 0, 126, 1, 300], seed=14)
    ns = np.array([len(p[0]) for p in probs], dtype=np.int64)
    # packed with gaps between problems; Z regions padded too
    off_de = np.zeros(len(ns), dtype=np.int64)
    off_z = np.zeros(len(ns), dtype=np.int64)
    a = z = 3
    for q, n in enumerate(ns):
        off_de[q], off_z[q] = a, z
        a += n + 5
        z += n * n + 7
    dev = torch.device("cuda:0")
    D = np.full(a, 99.0)
    E = np.full(a, 99.0)
    W = np.full(a, 99.0)
    for q, (d, e, w) in enumerate(probs):
        k = len(d)
        D[off_de[q]:off_de[q] + k] = d
        E[off_de[q]:off_de[q] + max(k - 1, 0)] = e
        W[off_de[q]:off_de[q] + k] = w
    td, te, tw = (torch.from_numpy(x).to(dev) for x in (D, E, W))
    tz = torch.full((z,), -7.0, dtype=torch.float64, device=dev)
    info = torch.full((len(ns),), -1, dtype=torch.int64, device=dev)
    gpu.tinv_batch_device(ns, off_de, off_z, td, te, tw, tz, info=info)
    torch.cuda.synchronize()
    Zall = tz.cpu().numpy()
    assert info.cpu().numpy().tolist() == [0] * len(ns)
    for q, (d, e, w) in enumerate(probs):
        k = len(d)
        Z = Zall[off_z[q]:off_z[q] + k * k].reshape((k, k), order="F")
        if k > 1:
            assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
            Z1 = gpu.tinv(d, e, w)
            wp, head, _ = gpu.plan(d, e, w)
            for idx in clusters_from_heads(head):
                assert sin_angle(Z1[:, idx], Z[:, idx]) <= 1e-10
        elif k == 1:
            assert Z.tolist() == [[1.0]]
    # the gaps are untouched
    mask = np.ones(z, dtype=bool)
    for q, n in enumerate(ns):
        mask[off_z[q]:off_z[q] + n * n] = False
    assert np.all(Zall[mask] == -7.0)


def test_batch_empty_and_workspace(gpu):
    assert gpu.tinv_batch([], [], []) == []
    assert gpu.batch_workspace_size([100, 200]) >= gpu.workspace_size(200, 200)
