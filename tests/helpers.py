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
    """sin of the largest principal angle between span(A) and span(B) (orthonormal columns)."""
    if A.shape[1] == 0:
        return 0.0
    return float(np.linalg.norm(B - A @ (A.T @ B), 2))


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
