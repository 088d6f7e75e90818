"""Parity of the CUDA path (through the C ABI) with the oracle.

Bars:
  * plan and LU factors: bit-exact (integer decisions and un-contracted FP64 on both sides);
  * solve: |x_gpu - x_orc| <= 50 cond eps |x| for shifts away from the spectrum; for shifts at
    eigenvalues the normalized directions agree to 1e-12;
  * stand-alone orthogonalization: |Q_gpu - Q_orc|_max <= 10 n eps kappa(V);
  * inverse iteration: residual <= 10 n eps ||T||_1, orthogonality <= 10 n eps (the invariants
    of a correct eigenvector set); singletons agree with the oracle per vector within 1e-10 (after DSTEIN's sign
    convention); clusters agree by the largest principal angle <= 1e-10.
"""
import math

import numpy as np
import pytest

from helpers import (EPS, check_sign_convention, clusters_from_heads, orth_ratio, residual_ratio,
                     sin_angle, singleton_equal)
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


# ---------------------------------------------------------------------------------------------
# a1-a2: plan
# ---------------------------------------------------------------------------------------------
def _plan_cases(orc):
    cases = []
    d, e = inputs.uniform(1000, seed=1)
    cases.append(("uniform1000", d, e, orc.bisect(d, e)))
    for g in (20, 200):
        d, e = inputs.glued_wilkinson(g, 1e-10)
        cases.append(("glued%d" % (21 * g), d, e, inputs.eigenvalues(d, e)))
    d, e = inputs.toeplitz(500, 2.0, 1.0)
    cases.append(("toeplitz500", d, e, inputs.toeplitz_eigenpairs(500, 2.0, 1.0)[0]))
    cases.append(("coincident", np.zeros(3), np.ones(2), np.array([1.0, 1.0, 1.0])))
    cases.append(("tie", np.array([998.0, 0, 0, 0]), np.array([2.0, 0, 0]),
                  np.array([0.0, 1.0, 2.5, 3.5])))
    return cases


def test_plan_bit_exact(gpu, orc):
    for name, d, e, w in _plan_cases(orc):
        wp, head, scal = gpu.plan(d, e, w)
        owp, ohead, on, ot, odt = orc.plan(d, e, w)
        assert np.array_equal(wp, owp), name
        assert np.array_equal(head, ohead), name
        assert scal.tolist() == [on, ot, odt], name


# ---------------------------------------------------------------------------------------------
# a3: LU
# ---------------------------------------------------------------------------------------------
def _near_tie(scale):
    """First pivot step near the tie |c| (|a| + |b|) = |a| (|c| + |a1| + |b1|) of the scaled
    pivoting rule (a = d0 - s = 1, b = c = e0 = 2, a1 + b1 = 4): shifts a few units in the last
    place either side of s = 0 put the cross products inside, at and outside the band that
    integer compares of their bit patterns cannot decide; `scale` (a power of two) moves the
    products below the normal range or above 1e300."""
    d = np.array([1.0, 3.0, 2.0, 5.0]) * scale
    e = np.array([2.0, 1.0, 0.5]) * scale
    shifts = np.arange(-24, 25) * 2.0 ** -52 * scale
    return d, e, shifts


@pytest.mark.parametrize("case", ["uniform1000", "glued4200", "hand3", "near_tie",
                                  "near_tie_tiny", "near_tie_huge"])
def test_lu_bit_exact(gpu, orc, case):
    if case == "hand3":
        d, e, shifts = np.array([1.0, 4.0, 1.0]), np.array([2.0, 1.0]), np.array([0.0, 0.5, 5.0])
    elif case.startswith("near_tie"):
        d, e, shifts = _near_tie({"near_tie": 1.0, "near_tie_tiny": 2.0 ** -520,
                                  "near_tie_huge": 2.0 ** 500}[case])
    else:
        d, e, w = inputs.workload(case)
        rng = np.random.default_rng(0)
        idx = np.sort(rng.choice(len(w), 24, replace=False))
        wp = orc.plan(d, e, w)[0]
        shifts = np.r_[wp[idx], [0.0, d[3] + 1e-3, -5.0]]
    l, u0, u1, u2, piv = gpu.lu(d, e, shifts)
    for j, s in enumerate(shifts):
        ou0, ou1, ou2, ol, opiv = orc.lagtf(d, e, s)
        assert np.array_equal(l[j], ol), (case, j)
        assert np.array_equal(u0[j], ou0), (case, j)
        assert np.array_equal(u1[j], ou1), (case, j)
        assert np.array_equal(u2[j], ou2), (case, j)
        assert np.array_equal(piv[j], opiv), (case, j)


# ---------------------------------------------------------------------------------------------
# a5: solve
# ---------------------------------------------------------------------------------------------
def test_solve_away_from_spectrum(gpu, orc):
    d, e = inputs.uniform(700, seed=3)
    lam = orc.bisect(d, e)
    idx = np.arange(5, 690, 37)
    shifts = 0.5 * (lam[idx] + lam[idx + 1])
    Y = np.random.default_rng(1).uniform(-1, 1, (700, len(idx)))
    X = gpu.solve(d, e, shifts, Y)
    A = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    for j, s in enumerate(shifts):
        x, _ = orc.lagts(orc.lagtf(d, e, s), Y[:, j])
        cond = np.linalg.cond(A - s * np.eye(700))
        assert np.abs(X[:, j] - x).max() <= 50 * cond * EPS * np.abs(x).max(), j


@pytest.mark.parametrize("case", ["uniform1000", "glued4200"])
def test_solve_at_eigenvalues_direction(gpu, orc, case):
    d, e, w = inputs.workload(case)
    wp = orc.plan(d, e, w)[0]
    idx = np.arange(0, len(w), len(w) // 17)
    rng = np.random.default_rng(2)
    Y = rng.uniform(-1, 1, (len(d), len(idx)))
    X = gpu.solve(d, e, wp[idx], Y)
    for j, i in enumerate(idx):
        x, _ = orc.lagts(orc.lagtf(d, e, wp[i]), Y[:, j])
        a = X[:, j] / np.linalg.norm(X[:, j])
        b = x / np.linalg.norm(x)
        assert np.linalg.norm(a - b * np.sign(a @ b)) < 1e-12, (case, i)


# ---------------------------------------------------------------------------------------------
# a6: stand-alone orthogonalization (same V on both sides)
# ---------------------------------------------------------------------------------------------
def _graded(n, m, kappa, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    W, _ = np.linalg.qr(rng.standard_normal((m, m)))
    return (U * np.logspace(0, -np.log10(kappa), m)) @ W.T


@pytest.mark.parametrize("max_team", [0, 1, 3])
@pytest.mark.parametrize("n,m,kappa", [(700, 80, 1.0), (1500, 200, 1e8), (97, 97, 1e3)])
def test_orth_cwy_matches_oracle(gpu, orc, n, m, kappa, max_team):
    V = np.random.default_rng(5).standard_normal((n, m)) if kappa == 1.0 else _graded(n, m, kappa)
    kap = np.linalg.cond(V)
    Q, Y, T = gpu.orth(V, "cwy", want_yt=True, max_team=max_team)
    Qo, Yo, To, _ = orc.orth(V, "cwy_new")
    tol = 10 * n * EPS * kap
    assert np.abs(Q - Qo).max() <= tol
    assert np.abs(np.tril(Y) - np.tril(Yo)).max() <= tol * np.abs(Yo).max()
    # T grows with the conditioning of Y; compare it relative to its size
    assert np.abs(np.triu(T) - np.triu(To)).max() <= tol * np.abs(To).max()
    assert np.abs(Q.T @ Q - np.eye(m)).max() <= 10 * n * EPS


def test_orth_cwy_stays_orthogonal_when_mgs_does_not(gpu):
    # Table 1: compact WY O(eps) whatever kappa(V); MGS O(eps kappa(V))
    V = _graded(600, 60, 1e14, seed=3)
    Qc = gpu.orth(V, "cwy")
    Qm = gpu.orth(V, "mgs")
    assert np.abs(Qc.T @ Qc - np.eye(60)).max() < 100 * EPS
    assert np.abs(Qm.T @ Qm - np.eye(60)).max() > 1e-6


def test_orth_mgs_matches_oracle(gpu, orc):
    V = np.random.default_rng(6).standard_normal((800, 50))
    Q = gpu.orth(V, "mgs")
    Qo, *_ = orc.orth(V, "mgs")
    assert np.abs(Q - Qo).max() <= 10 * 800 * EPS * np.linalg.cond(V)


# ---------------------------------------------------------------------------------------------
# the whole path
# ---------------------------------------------------------------------------------------------
def _compare(d, e, w, Z, Zo, head, tol_vec=1e-10, tol_sub=1e-10):
    """Singletons equal the oracle's vectors as computed (the sign convention of Alg. 4's final
    normalization, reading c12, is compared, not re-applied); clusters by principal angle; the
    sign convention holds on every column."""
    for idx in clusters_from_heads(head):
        if len(idx) == 1:
            assert singleton_equal(Z[:, idx[0]], Zo[:, idx[0]], tol_vec), idx[0]
        else:
            assert sin_angle(Zo[:, idx], Z[:, idx]) <= tol_sub, (idx[0], len(idx))
    check_sign_convention(Z)


@pytest.mark.parametrize("method", ["cwy", "mgs"])
def test_tinv_uniform1000(gpu, orc, method):
    d, e = inputs.uniform(1000, seed=1)
    w = orc.bisect(d, e)
    Z, info, ifail, iters = gpu.tinv(d, e, w, method=method, return_info=True)
    Zo, oinfo, *_ = orc.tinv(d, e, w, method)
    assert info == 0 and oinfo == 0
    assert np.all((iters >= 3) & (iters <= 5))
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    head = orc.plan(d, e, w)[1]
    _compare(d, e, w, Z, Zo, head)


@pytest.mark.parametrize("method", ["cwy", "mgs"])
@pytest.mark.parametrize("max_team", [0, 1])
def test_tinv_glued420(gpu, orc, method, max_team):
    d, e = inputs.glued_wilkinson(20, 1e-10)
    w = orc.bisect(d, e)
    Z, info, *_ = gpu.tinv(d, e, w, method=method, max_team=max_team, return_info=True)
    Zo, oinfo, *_ = orc.tinv(d, e, w, method)
    assert info == 0 and oinfo == 0
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    _compare(d, e, w, Z, Zo, orc.plan(d, e, w)[1])


def _within_cluster_orth(Z, head):
    worst = 0.0
    for idx in clusters_from_heads(head):
        G = Z[:, idx].T @ Z[:, idx] - np.eye(len(idx))
        worst = max(worst, float(np.abs(G).max()))
    return worst / (Z.shape[0] * EPS)


def _oracle_clusters(orc, d, e, w, method, clusters):
    """The oracle on each cluster's own sub-range of the spectrum (the j0 offset reproduces its
    start vectors), clusters in threads (the oracle's C calls release the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    def run(idx):
        s, t = int(idx[0]), int(idx[-1]) + 1
        Zo, oinfo, *_ = orc.tinv(d, e, w[s:t], method, j0=s)
        return s, t, Zo, oinfo

    with ThreadPoolExecutor(min(16, max(1, len(clusters)))) as ex:
        return list(ex.map(run, clusters))


@pytest.mark.parametrize("method", ["cwy", "mgs"])
def test_tinv_glued2100_every_cluster(gpu, orc, method):
    # 100 copies of W_21^+ glued by 1e-10: 14 clusters (7 of 200, 7 of 100 members), every one
    # compared with the oracle by principal angle; the whole-matrix invariants at 10 n eps
    d, e = inputs.glued_wilkinson(100, 1e-10)
    w = inputs.eigenvalues(d, e)
    Z, info, *_ = gpu.tinv(d, e, w, method=method, return_info=True)
    assert info == 0
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    head = orc.plan(d, e, w)[1]
    cl = clusters_from_heads(head)
    assert sorted(len(c) for c in cl) == [100] * 7 + [200] * 7
    for s, t, Zo, oinfo in _oracle_clusters(orc, d, e, w, method, cl):
        assert oinfo == 0
        assert sin_angle(Zo, Z[:, s:t]) <= 1e-10, (s, t)
    assert check_sign_convention(Z) > 0


@pytest.mark.parametrize("method", ["cwy", "mgs"])
def test_tinv_glued4200_full_size(gpu, orc, method):
    # The benchmark workload: 200 copies of W_21^+ glued by 1e-10, n = 4200.  Its 400-member
    # clusters hold eigenvalues that coincide in FP64 (389 distinct of 400).  The invariants are
    # held to 10 n eps (LAPACK's DSTEIN meets them on this matrix too), orthogonality inside
    # every cluster as well, and all 14 clusters are compared with the oracle by principal angle.
    d, e, w = inputs.workload("glued4200")
    Z, info, *_ = gpu.tinv(d, e, w, method=method, return_info=True)
    assert info == 0
    head = orc.plan(d, e, w)[1]
    assert _within_cluster_orth(Z, head) <= 10
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    cl = clusters_from_heads(head)
    sizes = sorted(len(c) for c in cl)
    assert sizes == [200] * 7 + [400] * 7
    for s, t, Zo, oinfo in _oracle_clusters(orc, d, e, w, method, cl):
        assert oinfo == 0
        assert sin_angle(Zo, Z[:, s:t]) <= 1e-10, (s, t)


def test_tinv_glued3108_near_singular_solves(gpu, orc):
    # 148 copies of W_21^+: the shifts of the 296-member clusters leave one small pivot per
    # block in U, and for late members the chunked back substitution folds maps that grew
    # across two of them (a boundary error of ~1e-5 relative).  The solves' consistency check
    # must catch that and redo those solves sequentially.
    d, e = inputs.glued_wilkinson(148, 1e-10)
    w = orc.bisect(d, e)
    head = orc.plan(d, e, w)[1]
    Zs = {}
    for name, kw in (("cwy", {}), ("cwy1", {"max_team": 1}), ("mgs", {"method": "mgs"})):
        Z, info, *_ = gpu.tinv(d, e, w, return_info=True, **kw)
        assert info == 0
        assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10, name
        Zs[name] = Z
    assert _within_cluster_orth(Zs["cwy"], head) <= 10
    s, t = 1924, 2220
    Zo, oinfo, *_ = orc.tinv(d, e, w[s:t], "cwy", j0=s)
    assert oinfo == 0
    assert sin_angle(Zo, Zs["cwy"][:, s:t]) <= 1e-10


def test_tinv_toeplitz4200_closed_form(gpu):
    n = 4200
    d, e = inputs.toeplitz(n, 2.0, 1.0)
    lam, V = inputs.toeplitz_eigenpairs(n, 2.0, 1.0)
    Z, info, *_ = gpu.tinv(d, e, lam, return_info=True)
    assert info == 0
    assert residual_ratio(d, e, lam, Z) <= 10 and orth_ratio(Z) <= 10
    from helpers import tri_matvec

    R = tri_matvec(d, e, Z) - Z * lam
    gaps = np.minimum(np.r_[np.inf, np.diff(lam)], np.r_[np.diff(lam), np.inf])
    ang = np.linalg.norm(Z - V * np.sign(np.sum(Z * V, axis=0)), axis=0)
    assert np.all(ang <= 4 * np.linalg.norm(R, axis=0) / gaps + 1e-13)


def test_tinv_edge_cases(gpu, orc):
    # n = 2
    Z = gpu.tinv(np.array([1.0, 1.0]), np.array([1.0]), np.array([0.0, 2.0]))
    s = 1 / math.sqrt(2)
    assert np.allclose(Z, [[s, s], [-s, s]], atol=1e-15)
    # exact zeros in e, coinciding eigenvalues of decoupled blocks
    d = np.array([0.5, 0.5, 0.5, -0.2, 0.1, 0.3])
    e = np.array([0.0, 0.0, 0.3, 0.0, 0.2])
    w = np.sort(np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1)))
    for method in ("cwy", "mgs"):
        Z = gpu.tinv(d, e, w, method=method)
        assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    # a sub-range of the spectrum, ragged sizes around the chunking
    for n in (33, 64, 65, 127, 257, 1031):
        d, e = inputs.uniform(n, seed=n)
        w = orc.bisect(d, e)
        Z, info, *_ = gpu.tinv(d, e, w[n // 4: n // 2], j0=n // 4, return_info=True)
        assert info == 0 and residual_ratio(d, e, w[n // 4: n // 2], Z) <= 10
        Zo = orc.tinv(d, e, w[n // 4: n // 2], "cwy", j0=n // 4)[0]
        head = orc.plan(d, e, w[n // 4: n // 2])[1]
        _compare(d, e, w, Z, Zo, head)


def test_tinv_deterministic(gpu):
    d, e, w = inputs.workload("uniform1000")
    Z1 = gpu.tinv(d, e, w)
    Z2 = gpu.tinv(d, e, w)
    assert np.array_equal(Z1, Z2)
    d, e = inputs.glued_wilkinson(30, 1e-10)
    w = inputs.eigenvalues(d, e)
    assert np.array_equal(gpu.tinv(d, e, w), gpu.tinv(d, e, w))


def test_tinv_device_pointers(gpu, orc):
    import torch

    d, e, w = inputs.workload("uniform1000")
    dev = torch.device("cuda:0")
    td, te, tw = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (d, e, w))
    Zt = torch.zeros((len(w), len(d)), dtype=torch.float64, device=dev)
    iters = torch.zeros(len(w), dtype=torch.int32, device=dev)
    info = torch.full((1,), -7, dtype=torch.int64, device=dev)
    ws = torch.empty(gpu.workspace_size(len(d), len(w)), dtype=torch.uint8, device=dev)
    gpu.tinv_device(td, te, tw, Zt, workspace=ws, iters=iters, info=info)
    torch.cuda.synchronize()
    Z = Zt.cpu().numpy().T
    assert int(info.item()) == 0
    assert int(iters.min()) >= 3
    assert np.array_equal(Z, gpu.tinv(d, e, w))
