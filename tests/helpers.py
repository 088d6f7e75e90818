"""Test-side checks: invariants and subspace comparisons (plain numpy)."""
import numpy as np

EPS = np.finfo(np.float64).eps


def dense(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def onenorm_dense(d, e):
    return float(np.abs(dense(d, e)).sum(axis=0).max())


def tri_matvec(d, e, Z):
    """T @ Z for tridiagonal T without forming T."""
    Z = np.asarray(Z)
    out = d[:, None] * Z
    out[:-1] += e[:, None] * Z[1:]
    out[1:] += e[:, None] * Z[:-1]
    return out


def residual_ratio(d, e, w, Z):
    """max|T Z - Z diag(w)| / (n eps ||T||_1)."""
    n = len(d)
    R = tri_matvec(d, e, Z) - Z * np.asarray(w)[None, :]
    nrm = float(np.max(np.abs(d) + np.r_[0, np.abs(e)] + np.r_[np.abs(e), 0]))
    return float(np.abs(R).max() / (n * EPS * nrm))


def orth_ratio(Z):
    """max|Z^T Z - I| / (n eps)."""
    n = Z.shape[0]
    G = Z.T @ Z
    return float(np.abs(G - np.eye(Z.shape[1])).max() / (n * EPS))


def sin_angle(A, B):
    """sin of the largest principal angle between span(A) and span(B).  Both bases are
    orthonormalized first (QR), so a basis whose columns are orthogonal only to O(eps kappa), as
    MGS gives, is compared by the subspace it spans."""
    if A.shape[1] == 0:
        return 0.0
    Qa = np.linalg.qr(A)[0]
    Qb = np.linalg.qr(B)[0]
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2))


def clusters_from_heads(head):
    """List of index arrays, one per cluster, from the head array of a plan."""
    head = np.asarray(head)
    starts = np.flatnonzero(head == np.arange(len(head)))
    ends = np.r_[starts[1:], len(head)]
    return [np.arange(s, t) for s, t in zip(starts, ends)]


def sign_fix(Z):
    """Make the first entry of largest magnitude of each column positive (DSTEIN convention)."""
    Z = np.array(Z, copy=True)
    idx = np.argmax(np.abs(Z), axis=0)
    s = np.sign(Z[idx, np.arange(Z.shape[1])])
    s[s == 0] = 1
    return Z * s


def first_max_ties(z, rel=1e-8):
    """True when the first entry of largest magnitude of z is not clear-cut: another entry's
    magnitude is within a relative `rel` of the largest (rounding can then pick either)."""
    a = np.abs(np.asarray(z))
    top = a.max()
    return int(np.sum(a >= top * (1.0 - rel))) > 1


def check_sign_convention(Z):
    """DSTEIN's convention on every column that has a clear-cut first entry of largest
    magnitude: that entry is positive.  Returns the number of columns checked."""
    Z = np.asarray(Z)
    checked = 0
    for j in range(Z.shape[1]):
        z = Z[:, j]
        if first_max_ties(z):
            continue
        assert z[int(np.argmax(np.abs(z)))] > 0.0, j
        checked += 1
    return checked


def singleton_equal(zg, zo, tol):
    """A singleton's vector against the oracle's, WITHOUT re-applying the sign convention:
    equal within tol when the oracle's first largest entry is clear-cut (so both sides must have
    chosen the same sign), equal up to sign otherwise."""
    zg, zo = np.asarray(zg).ravel(), np.asarray(zo).ravel()
    if first_max_ties(zo):
        return min(np.abs(zg - zo).max(), np.abs(zg + zo).max()) <= tol
    return np.abs(zg - zo).max() <= tol
