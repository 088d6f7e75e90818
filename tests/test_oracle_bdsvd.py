"""Oracle pins for singular triplets of an upper bidiagonal B by inverse iteration on its
Golub-Kahan tridiagonal form (a further use of the method named in the paper's Sec. 6).
CPU only."""
import math

import numpy as np

import oracle
from helpers import EPS, dense, sin_angle


def _bidiag(a, b):
    return np.diag(a) + np.diag(b, 1)


def _rand(n, seed):
    g = np.random.default_rng(seed)
    return g.uniform(0.5, 2.0, n) * g.choice([-1.0, 1.0], n), g.uniform(-1.0, 1.0, n - 1)


def test_golub_kahan_form_has_the_interleaved_singular_vectors():
    # closed form of the construction: with B = U S V^T (numpy), z = (v1, u1, v2, u2, ...)/sqrt 2
    # is an eigenvector of T_GK for +sigma and (v1, -u1, ...)/sqrt 2 for -sigma
    a, b = _rand(12, 3)
    d2, e2 = oracle.golub_kahan(a, b)
    assert np.all(d2 == 0.0) and np.array_equal(e2[0::2], a) and np.array_equal(e2[1::2], b)
    T = dense(d2, e2)
    Uu, S, Vt = np.linalg.svd(_bidiag(a, b))
    for j in range(12):
        z = np.zeros(24)
        z[0::2], z[1::2] = Vt[j], Uu[:, j]
        z /= math.sqrt(2.0)
        assert np.abs(T @ z - S[j] * z).max() < 1e-14
        z[1::2] *= -1.0
        assert np.abs(T @ z + S[j] * z).max() < 1e-14


def test_random_bidiagonal_against_numpy_svd():
    n = 60
    a, b = _rand(n, 7)
    s, U, V, info = oracle.bdsvd(a, b)
    assert info == 0
    B = _bidiag(a, b)
    Uu, S, Vt = np.linalg.svd(B)
    nrm = np.abs(B).sum(axis=0).max()
    assert np.all(np.diff(s) >= 0)
    assert np.abs(s - S[::-1]).max() <= 4 * n * EPS * nrm
    assert np.abs(B @ V - U * s).max() <= 10 * n * EPS * nrm
    assert np.abs(B.T @ U - V * s).max() <= 10 * n * EPS * nrm
    assert np.abs(U.T @ U - np.eye(n)).max() <= 10 * n * EPS
    assert np.abs(V.T @ V - np.eye(n)).max() <= 10 * n * EPS
    gaps = np.diff(S[::-1])
    for j in range(n):
        sep = min(gaps[j - 1] if j > 0 else np.inf, gaps[j] if j < n - 1 else np.inf)
        if sep < 1e-6:
            continue
        k = n - 1 - j
        assert abs(abs(V[:, j] @ Vt[k]) - 1.0) < 1e-10
        assert abs(abs(U[:, j] @ Uu[:, k]) - 1.0) < 1e-10
        assert (V[:, j] @ Vt[k]) * (U[:, j] @ Uu[:, k]) > 0  # u and v carry the same sign


def test_diagonal_bidiagonal_gives_signed_permutations():
    a = np.array([3.0, -1.0, 2.0, 0.5])
    s, U, V, info = oracle.bdsvd(a, np.zeros(3))
    order = np.argsort(np.abs(a), kind="stable")
    assert np.abs(s - np.abs(a)[order]).max() <= 4 * EPS * 3.0
    for j, i in enumerate(order):
        assert abs(abs(V[i, j]) - 1.0) < 1e-15 and abs(abs(U[i, j]) - 1.0) < 1e-15
        assert np.sum(np.abs(V[:, j])) == abs(V[i, j]) and np.sum(np.abs(U[:, j])) == abs(U[i, j])
        assert U[i, j] * V[i, j] * a[i] > 0


def test_order_one():
    s, U, V, info = oracle.bdsvd(np.array([-2.5]), np.zeros(0))
    assert info == 0 and abs(s[0] - 2.5) <= 4 * EPS * 2.5
    assert abs(abs(V[0, 0]) - 1.0) < 1e-15 and U[0, 0] * V[0, 0] < 0


def test_clustered_singular_values():
    # four copies of one random bidiagonal block coupled by 1e-6: clusters of 4 singular values
    # (one Peters-Wilkinson cluster each in T_GK); inside each cluster the vectors span the
    # cluster's singular subspaces.  (With a coupling of 1e-10 the oracle's own inverse iteration
    # on T_GK loses orthogonality to about 1e-10 for some seeds: the reorthogonalization of
    # nearly coincident iterates cancels, as on glued Wilkinson matrices.)
    a0, b0 = _rand(10, 11)
    a = np.tile(a0, 4)
    b = np.concatenate([np.r_[b0, 1e-6], np.r_[b0, 1e-6], np.r_[b0, 1e-6], b0])
    s, U, V, info = oracle.bdsvd(a, b)
    assert info == 0
    d2, e2 = oracle.golub_kahan(a, b)
    head = oracle.plan(d2, e2, s)[1]
    assert np.array_equal(head, np.repeat(np.arange(0, 40, 4), 4))
    B = _bidiag(a, b)
    n = 40
    nrm = np.abs(B).sum(axis=0).max()
    assert np.abs(B @ V - U * s).max() <= 10 * n * EPS * nrm
    assert np.abs(U.T @ U - np.eye(n)).max() <= 10 * n * EPS
    assert np.abs(V.T @ V - np.eye(n)).max() <= 10 * n * EPS
    Uu, S, Vt = np.linalg.svd(B)
    for c in range(10):
        idx = np.arange(4 * c, 4 * c + 4)
        k = n - 1 - idx
        assert np.ptp(s[idx]) < 1e-5
        assert sin_angle(V[:, idx], Vt[k].T) < 1e-6
        assert sin_angle(U[:, idx], Uu[:, k]) < 1e-6
