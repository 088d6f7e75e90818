"""Oracle pins for splitting T into unreduced blocks (the IBLOCK/ISPLIT convention DSTEIN takes
from LAPACK's bisection, Sec. 5.1) and for the split driver (bisection + inverse iteration per
block, merged in ascending order).  CPU only."""
import numpy as np

import oracle
from paper_1209_1910_gb300 import inputs
from helpers import EPS, dense, orth_ratio, residual_ratio


def test_split_threshold_is_eps_times_onenorm_inclusive():
    # ||T||_1 = 4 (row 1: |2| + |1| + |1|); the entry equal to eps*4 splits, the next
    # representable value above does not
    d = np.array([1.0, 2.0, 1.0, 1.0, 1.0, 1.0])
    tol = EPS * 4.0
    e = np.array([1.0, 1.0, tol, np.nextafter(tol, 1.0), 0.0])
    assert oracle.onenorm(d, e) == 4.0
    assert list(oracle.split(d, e)) == [3, 5, 6]
    # signs do not matter (||T||_1 is then about 3, so 2 eps is below the threshold), an exact
    # zero always splits, no entry means one block
    e2 = np.array([1.0, -2.0 * EPS, 1.0, 1.0, 1.0])
    assert list(oracle.split(d, e2)) == [2, 6]
    assert list(oracle.split(d, np.ones(5))) == [6]
    assert list(oracle.split(np.array([5.0]), np.zeros(0))) == [1]
    assert len(oracle.split(np.zeros(0), np.zeros(0))) == 0


def test_diagonal_matrix_gives_sorted_diagonal_and_a_permutation():
    # every e_i = 0: n blocks of order 1, each eigenvector is e_i exactly; ties keep row order
    d = np.array([3.0, -1.0, 2.0, -1.0, 0.5, 3.0])
    w, Z, iblock, isplit, info = oracle.eig_split(d, np.zeros(5))
    assert info == 0
    assert list(isplit) == [1, 2, 3, 4, 5, 6]
    order = np.argsort(d, kind="stable")
    # bisection of a 1 x 1 block returns the midpoint of a bracket of width <= 2 eps |d_i|
    assert np.abs(w - d[order]).max() <= 2 * EPS * 3.0
    assert np.array_equal(iblock, order)
    assert np.array_equal(Z, np.eye(6)[:, order])


def test_repeated_identical_blocks():
    # three W21+ blocks with exactly zero glue: every eigenvalue of W21+ three times, one vector
    # per block, each zero outside its block and equal (up to sign) to the block's own vector
    d, e = inputs.glued_wilkinson(3, delta=0.0)
    w, Z, iblock, isplit, info = oracle.eig_split(d, e)
    assert info == 0 and list(isplit) == [21, 42, 63]
    db, eb = d[:21], e[:20]
    wb = oracle.bisect(db, eb)
    assert np.array_equal(w, np.repeat(wb, 3))
    assert np.array_equal(iblock, np.tile([0, 1, 2], 21))
    lam = np.linalg.eigvalsh(dense(db, eb))
    assert np.abs(w - np.repeat(lam, 3)).max() <= 1e-13 * 11
    Zb, _, _, _, _ = oracle.tinv(db, eb, wb)
    for j in range(63):
        b = iblock[j]
        col = Z[:, j]
        outside = np.r_[col[:21 * b], col[21 * (b + 1):]]
        assert np.all(outside == 0.0)
        assert np.array_equal(col[21 * b:21 * (b + 1)], Zb[:, j // 3])
    assert orth_ratio(Z) < 1.0
    assert residual_ratio(d, e, w, Z) < 1.0


def test_random_blocks_against_jacobi():
    # a random T with three entries set to zero: eigenpairs against brute-force Jacobi on the
    # dense matrix (the spectrum is simple and well separated at this seed)
    d, e = inputs.uniform(40, seed=11)
    e[[7, 19, 20]] = 0.0
    w, Z, iblock, isplit, info = oracle.eig_split(d, e)
    assert info == 0 and list(isplit) == [8, 20, 21, 40]
    lam, V = oracle.jacobi(dense(d, e))
    nrm = oracle.onenorm(d, e)
    assert np.abs(w - lam).max() <= 40 * EPS * nrm
    gaps = np.diff(lam)
    assert gaps.min() > 1e-3
    for j in range(40):
        assert abs(abs(Z[:, j] @ V[:, j]) - 1.0) < 1e-10
        b0 = 0 if iblock[j] == 0 else isplit[iblock[j] - 1]
        b1 = isplit[iblock[j]]
        assert np.all(Z[:b0, j] == 0.0) and np.all(Z[b1:, j] == 0.0)
    assert residual_ratio(d, e, w, Z) < 1.0
    assert orth_ratio(Z) < 1.0


def test_unsplit_matrix_is_one_block():
    d, e = inputs.uniform(30, seed=4)
    w, Z, iblock, isplit, info = oracle.eig_split(d, e)
    assert list(isplit) == [30] and np.all(iblock == 0)
    assert np.array_equal(w, oracle.bisect(d, e))
    lam = np.linalg.eigvalsh(dense(d, e))
    assert np.abs(w - lam).max() <= 30 * EPS * oracle.onenorm(d, e)
    assert residual_ratio(d, e, w, Z) < 1.0 and orth_ratio(Z) < 1.0


def test_tiny_glue_splits_and_stays_accurate():
    # glue far below eps ||T||_1 (= 11 eps): the split result is still an eigen-decomposition of
    # the unsplit T within the method's bounds
    d, e = inputs.glued_wilkinson(4, delta=1e-17)
    w, Z, iblock, isplit, info = oracle.eig_split(d, e)
    assert list(isplit) == [21, 42, 63, 84]
    assert residual_ratio(d, e, w, Z) < 1.0
    assert orth_ratio(Z) < 1.0
