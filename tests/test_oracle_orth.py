"""Pins of the oracle's orthogonalizers (Sec. 3): compact-WY identities (Eqs. cwy1, cwy2,
Eq. yt and the t_j identity of Sec. 3.3.2), agreement with a library QR, and Table 1's
computation and orthogonality rows."""
import numpy as np
import pytest

from helpers import EPS

METHODS = ["mgs", "house", "cwy_ordinary", "cwy_new"]


def graded(n, m, kappa, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    W, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = np.logspace(0, -np.log10(kappa), m)
    return (U * s) @ W.T


@pytest.mark.parametrize("method", METHODS)
def test_matches_library_qr_up_to_column_signs(orc, method):
    V = np.random.default_rng(3).standard_normal((90, 25))
    Q, *_ = orc.orth(V, method)
    Qr, _ = np.linalg.qr(V)
    s = np.sign(np.sum(Q * Qr, axis=0))
    assert np.all(s != 0)
    assert np.abs(Q - Qr * s).max() < 1e-13


@pytest.mark.parametrize("method", ["cwy_ordinary", "cwy_new"])
def test_cwy_product_identity(orc, method):
    # Eq. cwy2: H_1 ... H_j = I - Y_j T_j Y_j^T, with H_i = I - t_i y_i y_i^T, t_i = 2/||y_i||^2
    V = np.random.default_rng(4).standard_normal((30, 9))
    Q, Y, T, _ = orc.orth(V, method)
    n, m = Y.shape
    P = np.eye(n)
    for i in range(m):
        y = Y[:, i]
        P = P @ (np.eye(n) - (2.0 / (y @ y)) * np.outer(y, y))
        Ti = T[: i + 1, : i + 1]
        assert np.abs(P - (np.eye(n) - Y[:, : i + 1] @ Ti @ Y[:, : i + 1].T)).max() < 1e-14
    assert np.allclose(np.triu(T), T)


def test_cwy_new_t_identity_and_structure(orc):
    # t_j = 2/||y_j||^2 = 1/(c_j^2 - u_jj c_j) (Sec. 3.3.2); y_j = [0_{j-1}; y_hat_j] (Eq. yt)
    V = np.random.default_rng(5).standard_normal((25, 8))
    Q, Y, T, _ = orc.orth(V, "cwy_new")
    for j in range(8):
        assert np.all(Y[:j, j] == 0.0)
        assert T[j, j] == pytest.approx(2.0 / (Y[:, j] @ Y[:, j]), rel=1e-14)
    # the new form and Alg. 2 produce the same reflectors
    _, Yh, th, _ = orc.orth(V, "house")
    assert np.abs(Yh - Y).max() < 1e-13
    assert np.abs(th - np.diag(T)).max() < 1e-13


def test_q_from_T_not_T_transpose(orc):
    # Reading of Sec. 3.3.1/3.3.2: q_j = (I - Y_j T_j Y_j^T) e_j at step j.  Formed with the
    # printed T_j^T, the q_j are neither orthonormal nor a basis of span(v_1..v_j).
    V = np.random.default_rng(6).standard_normal((40, 10))
    Q, Y, T, _ = orc.orth(V, "cwy_ordinary")
    n, m = Y.shape
    Qt = np.zeros((n, m))
    for j in range(m):
        Yj, Tj = Y[:, : j + 1], T[: j + 1, : j + 1]
        Qt[:, j] = np.eye(n)[:, j] - Yj @ (Tj.T @ Yj[j, :])
    assert np.abs(Q.T @ Q - np.eye(m)).max() < 1e-14
    assert np.abs(Qt.T @ Qt - np.eye(m)).max() > 1e-2
    # span(q_1..q_j) = span(v_1..v_j) holds for T_j only
    for j in range(1, m + 1):
        P = Q[:, :j] @ Q[:, :j].T
        assert np.abs(V[:, :j] - P @ V[:, :j]).max() < 1e-12


def test_table1_orthogonality_vs_condition(orc):
    # Table 1: MGS orthogonality O(eps kappa(V)); Householder and compact WY O(eps)
    m = 40
    for kappa in (1e2, 1e6, 1e10, 1e14):
        V = graded(200, m, kappa)
        err = {}
        for method in METHODS:
            Q, *_ = orc.orth(V, method)
            err[method] = np.abs(Q.T @ Q - np.eye(m)).max()
        for method in ("house", "cwy_ordinary", "cwy_new"):
            assert err[method] < 100 * EPS
        assert err["mgs"] > 1e-3 * EPS * kappa
        assert err["mgs"] < 100 * EPS * kappa
    assert err["mgs"] > 1e-4  # at kappa = 1e14 MGS has lost orthogonality


def test_table1_computation_counts(orc):
    # Table 1: MGS 2m^2n, compact WY 4m^2n + m^3, new compact WY 4m^2n - m^3 (leading terms)
    n, m = 2000, 400
    V = np.random.default_rng(7).standard_normal((n, m))
    f = {meth: orc.orth(V, meth)[3] for meth in ("mgs", "cwy_ordinary", "cwy_new")}
    assert f["mgs"] / (2 * m * m * n) == pytest.approx(1.0, abs=0.01)
    assert f["cwy_ordinary"] / (4 * m * m * n + m ** 3) == pytest.approx(1.0, abs=0.01)
    assert f["cwy_new"] / (4 * m * m * n - m ** 3) == pytest.approx(1.0, abs=0.01)
    assert f["cwy_new"] < f["cwy_ordinary"]


def test_rank_deficient_input_breakdown(orc):
    # v_3 in span(v_1, v_2): the remainder is exactly zero in exact arithmetic; all
    # Householder-based forms must still return an orthonormal Q.
    V = np.zeros((6, 3))
    V[:, 0] = [1, 0, 0, 0, 0, 0]
    V[:, 1] = [0, 1, 0, 0, 0, 0]
    V[:, 2] = [2, 3, 0, 0, 0, 0]
    for method in ("house", "cwy_ordinary", "cwy_new"):
        Q, *_ = orc.orth(V, method)
        assert np.abs(Q.T @ Q - np.eye(3)).max() < 1e-15
