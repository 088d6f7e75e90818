"""Pins of the oracle's blocked compact WY (Sec. 3.2: the compact-WY form of a product of
Householder reflectors, Eqs. cwy1/cwy2, applied to a block of columns at once) and of inverse
iteration with each cluster's members orthogonalized in blocks.

Stand-alone, a block step is the Householder QR of the block's columns after the reflectors
before it, so it yields the same Q, Y and T as the column-at-a-time form of Sec. 3.3.2 and the
QR factor of a library QR.  In inverse iteration a block's members are orthogonalized against
each other's current iterates rather than finished vectors, which changes the iteration; it is
held to the invariants, to each cluster's invariant subspace as found by the one-column form
and by LAPACK's DSTEIN (a black box), to the closed form of the Toeplitz matrix, to a dense
Jacobi brute force, and to DSTEIN's sweep counts."""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack

from helpers import EPS, clusters_from_heads, dense, orth_ratio, residual_ratio, sin_angle
from paper_1209_1910_gb300 import inputs

BLOCKS = [1, 2, 4, 8]  # the library's blocks hold at most 8 members


def _graded(n, m, kappa, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    W, _ = np.linalg.qr(rng.standard_normal((m, m)))
    return (U * np.logspace(0, -np.log10(kappa), m)) @ W.T


@pytest.mark.parametrize("block", [1, 3, 8, 50])
@pytest.mark.parametrize("kappa", [1.0, 1e8])
def test_block_step_is_the_householder_qr(orc, block, kappa):
    n, m = 300, 50
    V = np.random.default_rng(1).standard_normal((n, m)) if kappa == 1.0 else _graded(n, m, kappa)
    Qb, Yb, Tb, _ = orc.orth(V, "cwy_block", block=block)
    Qn, Yn, Tn, _ = orc.orth(V, "cwy_new")
    tol = 10 * n * EPS * np.linalg.cond(V)
    assert np.abs(Qb - Qn).max() <= tol
    assert np.abs(np.tril(Yb) - np.tril(Yn)).max() <= tol * np.abs(Yn).max()
    assert np.abs(np.triu(Tb) - np.triu(Tn)).max() <= tol * np.abs(Tn).max()
    # the QR factor of a library QR (up to column signs); Q orthonormal to O(eps) whatever
    # kappa(V) (Table 1's property of compact WY)
    Ql = np.linalg.qr(V)[0]
    s = np.sign(np.sum(Qb * Ql, axis=0))
    assert np.abs(-Qb - Ql * s).max() <= tol or np.abs(Qb - Ql * s).max() <= tol
    assert np.abs(Qb.T @ Qb - np.eye(m)).max() <= 10 * n * EPS


def test_block_step_eq_cwy2_product_identity(orc):
    # Q = I - Y T Y^T equals the product H_1 ... H_m of the reflectors (Eq. cwy2)
    n, m = 80, 20
    V = np.random.default_rng(3).standard_normal((n, m))
    _, Y, T, _ = orc.orth(V, "cwy_block", block=6)
    Y = np.tril(Y)
    T = np.triu(T)
    P = np.eye(n)
    for j in range(m):
        y = Y[:, j]
        P = P @ (np.eye(n) - T[j, j] * np.outer(y, y))
    assert np.abs(P - (np.eye(n) - Y @ T @ Y.T)).max() <= 100 * n * EPS


def _cases():
    return {"uniform1000": inputs.uniform(1000, seed=1),
            "glued420": inputs.glued_wilkinson(20, 1e-10),
            "glued2100": inputs.glued_wilkinson(100, 1e-10),
            "zero301": inputs.toeplitz(301, 0.0, 1.0)}


CASES = _cases()


@pytest.mark.parametrize("case", list(CASES))
def test_blocked_invariants_subspaces_and_sweeps(orc, case):
    d, e = CASES[case]
    w = inputs.eigenvalues(d, e)
    Z1, info1, _, it1, _ = orc.tinv(d, e, w, "cwy")
    head = orc.plan(d, e, w)[1]
    cl = [c for c in clusters_from_heads(head) if len(c) > 1]
    for b in BLOCKS:
        Z, info, _, it, _ = orc.tinv(d, e, w, "cwy", block=b)
        assert info == 0 and info1 == 0
        assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10, b
        # every member of these inputs needs exactly 1 + EXTRA sweeps, blocked or not
        assert np.array_equal(it, it1) and np.all(it == 3), b
        for c in cl:
            assert sin_angle(Z1[:, c], Z[:, c]) <= 1e-10, (b, c[0], len(c))


def test_block_of_one_is_the_one_column_iteration(orc):
    # block = 1 runs Alg. 4's CWY iteration through the block step: the same vectors to rounding
    d, e = inputs.uniform(400, seed=5)
    w = inputs.eigenvalues(d, e)
    Z1 = orc.tinv(d, e, w, "cwy")[0]
    Zb = orc.tinv(d, e, w, "cwy", block=1)[0]
    assert np.abs(Zb - Z1).max() <= 1e-11


def test_blocked_agrees_with_lapack_dstein_subspaces(orc):
    d, e = inputs.glued_wilkinson(20, 1e-10)
    n = len(d)
    w = orc.bisect(d, e)
    Zl, info = lapack.dstein(d, e, w, np.ones(n, dtype=np.int32), np.full(n, n, dtype=np.int32))
    assert info == 0
    head = orc.plan(d, e, w)[1]
    for b in (4, 16):
        Z = orc.tinv(d, e, w, "cwy", block=b)[0]
        for idx in clusters_from_heads(head):
            assert sin_angle(Zl[:, idx], Z[:, idx]) < 1e-10, (b, idx[0])


def test_blocked_toeplitz_closed_form(orc):
    n = 200
    d, e = inputs.toeplitz(n, 2.0, 1.0)
    lam, V = inputs.toeplitz_eigenpairs(n, 2.0, 1.0)
    for b in (4, 16):
        Z, info, *_ = orc.tinv(d, e, lam, "cwy", block=b)
        assert info == 0
        R = dense(d, e) @ Z - Z * lam
        gaps = np.minimum(np.r_[np.inf, np.diff(lam)], np.r_[np.diff(lam), np.inf])
        bound = 4 * np.linalg.norm(R, axis=0) / gaps + 1e-14
        ang = np.linalg.norm(Z - V * np.sign(np.sum(Z * V, axis=0)), axis=0)
        assert np.all(ang <= bound), b


def test_blocked_jacobi_brute_force(orc):
    d, e = inputs.uniform(48, seed=9)
    lam, V = orc.jacobi(dense(d, e))
    w = orc.bisect(d, e)
    assert np.abs(lam - w).max() <= 10 * 48 * EPS * np.abs(dense(d, e)).sum(0).max()
    head = orc.plan(d, e, w)[1]
    for b in (2, 8):
        Z = orc.tinv(d, e, w, "cwy", block=b)[0]
        for idx in clusters_from_heads(head):
            assert sin_angle(V[:, idx], Z[:, idx]) <= 1e-10, (b, idx[0])


def test_blocked_repeated_simple_eigenvalue_reports_ifail(orc):
    # a simple eigenvalue asked for three times: the block holds the two later copies, whose
    # remainders never grow (no second eigenvector within the cluster tolerance), so they run
    # MAXITS sweeps and are reported as not converged; the first copy converges in 3 sweeps
    d, e = inputs.uniform(50, seed=4)
    w = orc.bisect(d, e)
    ww = np.full(3, w[10])
    Z, info, ifail, iters, _ = orc.tinv(d, e, ww, "cwy", block=4)
    assert info == 2 and ifail.tolist() == [1, 2]
    assert iters[0] == 3 and np.all(iters[1:] == 5)
    assert np.allclose(np.linalg.norm(Z, axis=0), 1.0, atol=1e-14)
