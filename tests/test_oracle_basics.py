"""Pins of the oracle's start vectors, norm, Sturm bisection and cluster plan.

Each check compares the oracle with something other than itself: published generator
outputs, closed forms, a dense library eigensolver, brute force, or hand-computed cases.
"""
import math
import os

import numpy as np
import pytest

from helpers import EPS, dense, onenorm_dense
from paper_1209_1910_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs(orc):
    vals = [int(x) for x in open(os.path.join(GOLD, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    M = (1 << 64) - 1
    got = [orc.sm64_mix((1234567 + (i + 1) * gamma) & M) for i in range(len(vals))]
    assert got == vals


def test_start_values_range_and_grid(orc):
    v = orc.start_vector(seed=7, j=3, n=4000)
    assert v.min() >= -1.0 and v.max() < 1.0
    # exact multiples of 2^-52 (2*(k*2^-53) - 1)
    assert np.all(np.ldexp(v + 1.0, 52) == np.round(np.ldexp(v + 1.0, 52)))
    assert abs(v.mean()) < 0.05 and abs(v.var() - 1.0 / 3.0) < 0.03
    # distinct streams per vector index and per restart
    w = orc.start_vector(seed=7, j=4, n=4000)
    x = orc.start_vector(seed=7, j=3, n=4000, attempt=1)
    assert abs(np.corrcoef(v, w)[0, 1]) < 0.05 and abs(np.corrcoef(v, x)[0, 1]) < 0.05


def test_onenorm_matches_dense(orc):
    for seed in range(5):
        d, e = inputs.uniform(57, seed=seed)
        assert orc.onenorm(d, e) == onenorm_dense(d, e)
    d, e = inputs.glued_wilkinson(3)
    assert orc.onenorm(d, e) == 11.0 + 1e-10  # row end of a block: 10 + 1 + delta


@pytest.mark.parametrize("a,b,n", [(2.0, 1.0, 100), (0.0, 1.0, 101), (1.0, 1.0, 64)])
def test_bisect_toeplitz_closed_form(orc, a, b, n):
    d, e = inputs.toeplitz(n, a, b)
    w = orc.bisect(d, e)
    lam, _ = inputs.toeplitz_eigenpairs(n, a, b)
    nrm = abs(a) + 2 * abs(b)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(w - lam).max() <= 4 * EPS * nrm


def test_bisect_vs_dense_eigensolver(orc):
    for seed in range(3):
        d, e = inputs.uniform(80, seed=seed)
        w = orc.bisect(d, e)
        ref = np.linalg.eigvalsh(dense(d, e))
        # both sides carry O(eps ||T||) error of their own
        assert np.abs(w - ref).max() <= 16 * EPS * onenorm_dense(d, e)


def test_sturm_count_brute_force(orc):
    d, e = inputs.uniform(40, seed=5)
    lam = np.linalg.eigvalsh(dense(d, e))
    for x in np.linspace(lam[0] - 0.5, lam[-1] + 0.5, 57):
        if np.min(np.abs(lam - x)) < 1e-8:
            continue
        assert orc.sturm_count(d, e, x, 1e-300) == int(np.sum(lam < x))


def test_jacobi_vs_closed_form_and_eigh(orc):
    d, e = inputs.toeplitz(24, 2.0, 1.0)
    lam, V = orc.jacobi(dense(d, e))
    lc, Vc = inputs.toeplitz_eigenpairs(24, 2.0, 1.0)
    assert np.abs(lam - lc).max() < 50 * EPS * 4.0
    assert np.abs(np.abs(np.sum(V * Vc, axis=0)) - 1).max() < 1e-13
    A = np.random.default_rng(0).standard_normal((30, 30))
    A = A + A.T
    lam, V = orc.jacobi(A)
    assert np.abs(lam - np.linalg.eigvalsh(A)).max() < 1e-12
    assert np.abs(A @ V - V * lam).max() < 1e-12


def test_plan_glued_wilkinson_cluster_structure(orc):
    # 2*g-member clusters from the 7 near-coincident eigenvalue pairs of W_21^+ and g-member
    # clusters from the other 7 eigenvalues: 14 clusters (7 x 2g, 7 x g).
    for g in (20, 200):
        d, e = inputs.glued_wilkinson(g, 1e-10)
        w = inputs.eigenvalues(d, e)
        wp, head, onenrm, ortol, dtpcrt = orc.plan(d, e, w)
        assert onenrm == pytest.approx(11.0, abs=1e-9) and ortol == 1e-3 * onenrm
        assert dtpcrt == math.sqrt(0.1 / len(d))
        sizes = np.bincount(head)
        sizes = sorted(sizes[sizes > 0].tolist())
        assert sizes == [g] * 7 + [2 * g] * 7
        assert np.all(np.diff(wp) > 0)


def test_plan_perturbs_coincident_shifts(orc):
    # three equal approximations: w'_j = w'_{j-1} + 10 eps |w_j|
    d, e = np.array([0.0, 0.0, 0.0]), np.array([1.0, 1.0])
    wp, head, *_ = orc.plan(d, e, np.array([1.0, 1.0, 1.0]))
    assert wp.tolist() == [1.0, 1.0 + 10 * EPS, 1.0 + 20 * EPS]
    assert head.tolist() == [0, 0, 0]
    # well separated: untouched
    wp, head, *_ = orc.plan(d, e, np.array([-1.0, 0.25, 1.0]))
    assert wp.tolist() == [-1.0, 0.25, 1.0]


def test_plan_gap_equal_to_tolerance_stays_in_cluster(orc):
    # ||T||_1 = 1000 so ortol = 1.0 exactly; a gap of exactly 1.0 continues the cluster,
    # a larger gap starts a new one (Alg. 1 / Alg. 4 use "<=").
    d = np.array([998.0, 0.0, 0.0, 0.0])
    e = np.array([2.0, 0.0, 0.0])
    wp, head, onenrm, ortol, _ = orc.plan(d, e, np.array([0.0, 1.0, 2.5, 3.5]))
    assert onenrm == 1000.0 and ortol == 1.0
    assert head.tolist() == [0, 0, 2, 2]
