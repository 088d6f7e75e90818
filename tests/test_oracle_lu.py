"""Pins of the oracle's shifted tridiagonal LU with scaled partial pivoting and its solve
(the linear system of Eq. 1)."""
import numpy as np
import pytest

from helpers import EPS, dense
from paper_1209_1910_gb300 import inputs


def test_pivot_choices_hand_computed_3x3(orc):
    # T = [[1,2,0],[2,4,1],[0,1,1]], lambda = 0.
    # step 0: |a|/(|a|+|b|) = 1/3 > |c|/(|c|+|a1|+|b1|) = 2/7 -> keep row 0, l0 = 2,
    #         new a1 = 4 - 2*2 = 0.
    # step 1: pivot row is [0, 1]: scaled pivot 0 < 1/2 -> interchange, l1 = 0/1 = 0.
    u0, u1, u2, l, piv = orc.lagtf([1.0, 4.0, 1.0], [2.0, 1.0], 0.0)
    assert u0.tolist() == [1.0, 1.0, 1.0]
    assert u1[:2].tolist() == [2.0, 1.0]
    assert u2[:2].tolist() == [0.0, 0.0]
    assert l[:2].tolist() == [2.0, 0.0]
    assert piv[:2].tolist() == [0, 1]


def test_pivot_scale_of_the_current_row_and_a_tie(orc):
    # T = [[1,1,0],[1,1.5,1],[0,1,2]], lambda = 0.
    # step 0: 1/2 > 1/3.5 -> keep row 0, l0 = 1, current pivot row [0.5, 1].
    # step 1: the current row scaled by its own 1-norm: 0.5/1.5 = 1/3 against 1/(1+2) = 1/3, a
    #         tie -> keep it, l1 = 1/0.5 = 2 (scaled pivoting admits |l| > 1), u0[2] = 2 - 2*1.
    u0, u1, u2, l, piv = orc.lagtf([1.0, 1.5, 2.0], [1.0, 1.0], 0.0)
    assert piv[:2].tolist() == [0, 0]
    assert u0.tolist() == [1.0, 0.5, 0.0]
    assert u1[:2].tolist() == [1.0, 1.0]
    assert u2[:2].tolist() == [0.0, 0.0]
    assert l[:2].tolist() == [1.0, 2.0]


def test_scaled_pivoting_differs_from_magnitude_pivoting(orc):
    # |c| = 2 > |a| = 1, but scaled: 1/3 > 2/12 -> no interchange
    u0, u1, u2, l, piv = orc.lagtf([1.0, 10.0], [2.0], 0.0)
    assert piv[0] == 0 and l[0] == 2.0 and u0.tolist() == [1.0, 6.0]
    # a tie keeps the current row
    u0, u1, u2, l, piv = orc.lagtf([1.0, 1.0], [1.0], 0.0)
    assert piv[0] == 0 and u0.tolist() == [1.0, 0.0]


def test_tiny_pivot_replaced_by_tolerance(orc):
    # DLAGTS, job -1: a diagonal entry of U is perturbed (by tol = eps max|U|) only where a
    # quotient by it could overflow.  T = [[1,1],[1,1]] is singular: u0 = [1, 0].
    f = orc.lagtf([1.0, 1.0], [1.0], 0.0)
    x, tol = orc.lagts(f, [0.0, 1.0])
    assert tol == EPS
    assert x.tolist() == [-1.0 / EPS, 1.0 / EPS]
    x, _ = orc.lagts(f, [1.0, 1.0])
    assert x.tolist() == [1.0, 0.0]
    # a subnormal pivot: its reciprocal overflows, so it is replaced by tol
    f = orc.lagtf([1.0, 1e-310], [0.0], 0.0)
    x, tol = orc.lagts(f, [0.0, 1.0])
    assert tol == EPS and x.tolist() == [0.0, 1.0 / EPS]


def test_small_normal_pivot_is_not_perturbed(orc):
    # a pivot far below eps max|U| but in the normal range is used as it is (no overflow can
    # occur): x_2 = 1 / 1e-20 exactly, as DLAGTS gives; the inverse iteration's amplification
    # near an eigenvalue comes from exactly such pivots
    f = orc.lagtf([1.0, 1e-20], [0.0], 0.0)
    x, tol = orc.lagts(f, [0.0, 1.0])
    assert tol == EPS and x.tolist() == [0.0, 1e20]
    # the same at the threshold scale: a pivot just above DBL_MIN * max(1, |u1|) is kept
    f = orc.lagtf([1.0, 1e-300], [0.0], 0.0)
    x, _ = orc.lagts(f, [0.0, 1e-10])
    assert x[1] == 1e-10 / 1e-300


@pytest.mark.parametrize("seed", range(4))
def test_solve_residual_random_shift(orc, seed):
    d, e = inputs.uniform(60, seed=seed)
    A = dense(d, e)
    lam = np.linalg.eigvalsh(A)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        i = rng.integers(0, len(lam) - 1)
        sigma = 0.5 * (lam[i] + lam[i + 1])  # well away from the spectrum
        f = orc.lagtf(d, e, sigma)
        y = rng.uniform(-1, 1, len(d))
        x, _ = orc.lagts(f, y)
        ref = np.linalg.solve(A - sigma * np.eye(len(d)), y)
        cond = np.linalg.cond(A - sigma * np.eye(len(d)))
        assert np.abs(x - ref).max() <= 50 * cond * EPS * np.abs(ref).max()
        r = (A - sigma * np.eye(len(d))) @ x - y
        assert np.abs(r).max() <= 50 * EPS * np.abs(A - sigma * np.eye(len(d))).sum(0).max() * np.abs(x).max()


def test_solve_with_zero_offdiagonal(orc):
    # an exact zero in e splits T; pivoting must cope
    d = np.array([0.3, -0.2, 0.7, 0.1, -0.5])
    e = np.array([0.4, 0.0, -0.6, 0.2])
    A = dense(d, e)
    f = orc.lagtf(d, e, 0.05)
    y = np.arange(1.0, 6.0)
    x, _ = orc.lagts(f, y)
    assert np.allclose((A - 0.05 * np.eye(5)) @ x, y, rtol=0, atol=1e-13)


def test_solve_at_eigenvalue_gives_eigenvector_direction(orc):
    # one solve at a computed eigenvalue already points along the eigenvector
    d, e = inputs.uniform(40, seed=11)
    A = dense(d, e)
    lam, V = np.linalg.eigh(A)
    f = orc.lagtf(d, e, lam[17])
    x, _ = orc.lagts(f, np.random.default_rng(1).uniform(-1, 1, 40))
    x /= np.linalg.norm(x)
    assert abs(abs(x @ V[:, 17]) - 1.0) < 1e-12
