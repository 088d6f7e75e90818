"""Parity of the blocked compact-WY path (tinv_opts.block; Sec. 3.2's block form, Eqs.
cwy1/cwy2) with the oracle, through the C ABI.

* Stand-alone orthogonalization: the GPU block step equals the oracle's (orc_orth_cwy_block)
  within 10 n eps kappa(V) for Q, Y and T, whatever the block size.
* Inverse iteration: the invariants at 10 n eps, every cluster's invariant subspace equal to
  the oracle's blocked iteration (and to the one-member iteration) by principal angle <= 1e-10,
  DSTEIN's sweep counts, the sign convention on every column, and bit-identical repeats.
* block <= 1 is exactly the one-member path."""
import numpy as np
import pytest

from helpers import EPS, check_sign_convention, clusters_from_heads, orth_ratio, residual_ratio, sin_angle

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


def _graded(n, m, kappa, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    W, _ = np.linalg.qr(rng.standard_normal((m, m)))
    return (U * np.logspace(0, -np.log10(kappa), m)) @ W.T


@pytest.mark.parametrize("block", [2, 5, 8, 16])
@pytest.mark.parametrize("n,m,kappa", [(700, 80, 1.0), (1500, 200, 1e8), (97, 97, 1e3), (1500, 600, 1e4)])
def test_orth_block_matches_oracle(gpu, orc, n, m, kappa, block):
    V = np.random.default_rng(5).standard_normal((n, m)) if kappa == 1.0 else _graded(n, m, kappa)
    kap = np.linalg.cond(V)
    Q, Y, T = gpu.orth(V, "cwy", want_yt=True, block=block)
    Qo, Yo, To, _ = orc.orth(V, "cwy_block", block=block)
    tol = 10 * n * EPS * kap
    assert np.abs(Q - Qo).max() <= tol
    assert np.abs(np.tril(Y) - np.tril(Yo)).max() <= tol * np.abs(Yo).max()
    assert np.abs(np.triu(T) - np.triu(To)).max() <= tol * np.abs(To).max()
    assert np.abs(Q.T @ Q - np.eye(m)).max() <= 10 * n * EPS


def _check_blocked(gpu, orc, d, e, w, block, oracle_clusters=None):
    Z, info, ifail, iters = gpu.tinv(d, e, w, block=block, return_info=True)
    assert info == 0
    assert np.all(iters == 3)
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    head = orc.plan(d, e, w)[1]
    cl = clusters_from_heads(head)
    picks = [c for c in cl if len(c) > 1] if oracle_clusters is None else oracle_clusters(cl)
    for idx in picks:
        s, t = int(idx[0]), int(idx[-1]) + 1
        Zo, oinfo, *_ = orc.tinv(d, e, w[s:t], "cwy", j0=s, block=block)
        assert oinfo == 0
        assert sin_angle(Zo, Z[:, s:t]) <= 1e-10, (s, t)
    assert check_sign_convention(Z) > 0
    return Z


@pytest.mark.parametrize("block", [2, 4, 8, 16])
def test_blocked_glued2100_every_cluster(gpu, orc, block):
    d, e = inputs.glued_wilkinson(100, 1e-10)
    w = inputs.eigenvalues(d, e)
    cnt = np.zeros(4, dtype=np.int64)
    gpu.tinv(d, e, w, block=block, counters=cnt.ctypes.data)
    assert cnt[2] > 0  # clusters on CTA teams: the blocked path ran
    _check_blocked(gpu, orc, d, e, w, block)


@pytest.mark.parametrize("block", [8, 16])
def test_blocked_glued4200_full_size(gpu, orc, block):
    d, e, w = inputs.workload("glued4200")
    Z = _check_blocked(gpu, orc, d, e, w, block,
                       oracle_clusters=lambda cl: [c for c in cl if len(c) == 200][:1] +
                                                  [c for c in cl if len(c) == 400][:1])
    # the one-member iteration spans the same invariant subspaces
    Z1 = gpu.tinv(d, e, w)
    for idx in clusters_from_heads(orc.plan(d, e, w)[1]):
        assert sin_angle(Z1[:, idx], Z[:, idx]) <= 1e-10


@pytest.mark.parametrize("case", ["uniform1000", "glued3108"])
def test_blocked_other_workloads(gpu, orc, case):
    if case == "glued3108":
        d, e = inputs.glued_wilkinson(148, 1e-10)
        w = orc.bisect(d, e)
        pick = lambda cl: [c for c in cl if c[0] == 1924]
    else:
        d, e, w = inputs.workload(case)
        pick = None
    _check_blocked(gpu, orc, d, e, w, 8, oracle_clusters=pick)


@pytest.mark.parametrize("block", [8, 16])
def test_blocked_toeplitz4200_closed_form(gpu, block):
    # one cluster of 4200 members on a team of the whole grid: too large for the shared-memory
    # block staging, so the team reads its staged vectors from its buffers in L2; the closed
    # form holds
    n = 4200
    d, e = inputs.toeplitz(n, 2.0, 1.0)
    lam, V = inputs.toeplitz_eigenpairs(n, 2.0, 1.0)
    cnt = np.zeros(4, dtype=np.int64)
    Z, info, *_ = gpu.tinv(d, e, lam, block=block, return_info=True, counters=cnt.ctypes.data)
    assert cnt[2] > 0  # the cluster ran on a CTA team
    assert info == 0 and residual_ratio(d, e, lam, Z) <= 10 and orth_ratio(Z) <= 10
    from helpers import tri_matvec

    R = tri_matvec(d, e, Z) - Z * lam
    gaps = np.minimum(np.r_[np.inf, np.diff(lam)], np.r_[np.diff(lam), np.inf])
    ang = np.linalg.norm(Z - V * np.sign(np.sum(Z * V, axis=0)), axis=0)
    assert np.all(ang <= 4 * np.linalg.norm(R, axis=0) / gaps + 1e-13)


def test_blocked_deterministic_and_block_one_is_the_member_path(gpu):
    d, e = inputs.glued_wilkinson(60, 1e-10)
    w = inputs.eigenvalues(d, e)
    assert np.array_equal(gpu.tinv(d, e, w, block=6), gpu.tinv(d, e, w, block=6))
    Z0 = gpu.tinv(d, e, w)
    assert np.array_equal(gpu.tinv(d, e, w, block=1), Z0)
    assert np.array_equal(gpu.tinv(d, e, w, block=0), Z0)


@pytest.mark.parametrize("block", [8, 16])
def test_blocked_single_cta(gpu, orc, block):
    # every cluster on one CTA (max_team = 1): the blocked form there holds the block's panel in
    # the CTA's q-vector buffer; every cluster against the oracle's blocked iteration
    d, e = inputs.glued_wilkinson(100, 1e-10)
    w = inputs.eigenvalues(d, e)
    Z, info, ifail, iters = gpu.tinv(d, e, w, block=block, max_team=1, return_info=True)
    assert info == 0 and np.all(iters == 3)
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    for idx in clusters_from_heads(orc.plan(d, e, w)[1]):
        if len(idx) > 1:
            s, t = int(idx[0]), int(idx[-1]) + 1
            Zo, oinfo, *_ = orc.tinv(d, e, w[s:t], "cwy", j0=s, block=block)
            assert oinfo == 0
            assert sin_angle(Zo, Z[:, s:t]) <= 1e-10, (s, t)
    assert check_sign_convention(Z) > 0
    # a uniform matrix's clusters of all sizes, and repeats bit for bit
    d, e, w = inputs.workload("uniform1000")
    Z = gpu.tinv(d, e, w, block=block, max_team=1)
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    assert np.array_equal(Z, gpu.tinv(d, e, w, block=block, max_team=1))


def test_blocked_batch(gpu, orc):
    probs = []
    for q, n in enumerate([64, 2100, 97, 420, 1000]):
        if q % 2:
            d, e = inputs.glued_wilkinson(n // 21, 1e-10)
        else:
            d, e = inputs.uniform(n, seed=q)
        probs.append((d, e, inputs.eigenvalues(d, e)))
    Zs, rc, info, iters = gpu.tinv_batch([p[0] for p in probs], [p[1] for p in probs],
                                         [p[2] for p in probs], block=8, return_info=True)
    assert rc == 0 and np.all(info == 0)
    for (d, e, w), Z in zip(probs, Zs):
        assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
        Z1 = gpu.tinv(d, e, w)
        for idx in clusters_from_heads(orc.plan(d, e, w)[1]):
            if len(idx) > 1:
                assert sin_angle(Z1[:, idx], Z[:, idx]) <= 1e-10
