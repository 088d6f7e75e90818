"""Seeded synthetic tridiagonal workloads.

This module holds no arithmetic of the inverse-iteration method: it only draws or writes down
the matrices (diagonal ``d``, off-diagonal ``e``) of the paper's experiments (Sec. 5.1) and of
the derived benchmark configurations, and obtains eigenvalue approximations ``w`` from a
library bisection routine (LAPACK ``dstebz`` through SciPy, the same routine the paper uses
to produce its eigenvalues in Sec. 5.1) or from the closed form of the tridiagonal Toeplitz
spectrum.  It imports nothing else from this package, so tests and benchmarks can share it.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, seed: int = 1, lo: float = -1.0, hi: float = 1.0):
    """Random tridiagonal matrix, d and e i.i.d. U[lo, hi) (Type 1 of Sec. 5.1 uses [0, 1))."""
    g = rng(seed)
    d = g.uniform(lo, hi, n)
    e = g.uniform(lo, hi, max(n - 1, 0))
    return d, e


def wilkinson_block() -> np.ndarray:
    """Diagonal of W_21^+: 10, 9, ..., 1, 0, 1, ..., 10 (Sec. 5.1)."""
    return np.abs(11.0 - np.arange(1, 22, dtype=np.float64))


def glued_wilkinson(g: int, delta: float = 1e-10):
    """g copies of W_21^+ (unit off-diagonal) glued by off-diagonal entries delta (Type 3)."""
    d = np.tile(wilkinson_block(), g)
    e = np.ones(21 * g - 1)
    e[20::21] = delta
    return d, e


def bidiagonal(n: int, seed: int = 1):
    """Upper bidiagonal B for the singular-vector workload: diagonal a_i = +-U[1, 2) (random
    sign), superdiagonal b_i ~ U[-1/2, 1/2) (|b_i / a_{i+1}| <= 1/2 keeps B well conditioned)."""
    g = rng(seed)
    a = g.uniform(1.0, 2.0, n) * g.choice([-1.0, 1.0], n)
    b = g.uniform(-0.5, 0.5, max(n - 1, 0))
    return a, b


def toeplitz(n: int, a: float, b: float):
    """Tridiagonal Toeplitz matrix: diagonal a, off-diagonal b (Type 2 has a = b = 1)."""
    return np.full(n, float(a)), np.full(max(n - 1, 0), float(b))


def toeplitz_eigenpairs(n: int, a: float, b: float, k=None):
    """Closed form (textbook): lambda_k = a + 2b cos(k pi/(n+1)), v_ik = sqrt(2/(n+1)) sin(ik pi/(n+1)),
    k = 1..n.  Returned in ascending eigenvalue order (for b > 0 that is k = n..1)."""
    ks = np.arange(n, 0, -1) if b > 0 else np.arange(1, n + 1)
    if k is not None:
        ks = ks[np.asarray(k)]
    lam = a + 2.0 * b * np.cos(ks * math.pi / (n + 1))
    i = np.arange(1, n + 1)[:, None]
    V = math.sqrt(2.0 / (n + 1)) * np.sin(i * ks[None, :] * math.pi / (n + 1))
    return lam, V


def eigenvalues(d, e) -> np.ndarray:
    """Ascending eigenvalues by LAPACK dstebz bisection (SciPy), the paper's eigenvalue step."""
    from scipy.linalg import eigvalsh_tridiagonal

    d = np.asarray(d, dtype=np.float64)
    if len(d) == 1:
        return d.copy()
    return eigvalsh_tridiagonal(d, np.asarray(e, dtype=np.float64), lapack_driver="stebz")


def workload(name: str):
    """Named single-problem workloads: returns (d, e, w)."""
    if name == "uniform1000":
        d, e = uniform(1000, seed=1)
    elif name == "glued4200":
        d, e = glued_wilkinson(200, 1e-10)
    elif name == "glued2100":
        d, e = glued_wilkinson(100, 1e-10)
    elif name == "toeplitz4200":
        d, e = toeplitz(4200, 2.0, 1.0)
        return d, e, toeplitz_eigenpairs(4200, 2.0, 1.0)[0]
    elif name == "toeplitz6000":
        d, e = toeplitz(6000, 2.0, 1.0)
        return d, e, toeplitz_eigenpairs(6000, 2.0, 1.0)[0]
    elif name == "uniform10000":
        d, e = uniform(10000, seed=1)
    elif name == "zero10000":
        d, e = toeplitz(10000, 0.0, 1.0)
        return d, e, toeplitz_eigenpairs(10000, 0.0, 1.0)[0]
    else:
        raise KeyError(name)
    return d, e, eigenvalues(d, e)


def batch_sizes(count: int = 512, seed: int = 2, lo: int = 64, hi: int = 4096):
    """n log-uniform in [lo, hi]; odd entries are glued W_21^+ so n is rounded to 21*g."""
    g = rng(seed)
    ns = np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    out = []
    for p, n in enumerate(ns):
        if p % 2 == 1:
            gg = max(1, int(round(n / 21)))
            out.append(21 * gg)
        else:
            out.append(int(n))
    return out


def batch_matrices(count: int = 512, seed: int = 2, lo: int = 64, hi: int = 4096):
    """The batched workload's matrices: list of (d, e); even problems U[-1,1], odd glued
    W_21^+ (glue 1e-10)."""
    probs = []
    for p, n in enumerate(batch_sizes(count, seed, lo, hi)):
        if p % 2 == 1:
            d, e = glued_wilkinson(n // 21, 1e-10)
        else:
            d, e = uniform(n, seed=seed * 1000003 + p)
        probs.append((d, e))
    return probs


def batch(count: int = 512, seed: int = 2, lo: int = 64, hi: int = 4096):
    """The batched workload with eigenvalues: list of (d, e, w)."""
    return [(d, e, eigenvalues(d, e)) for d, e in batch_matrices(count, seed, lo, hi)]


def request_stream(count: int, rate_hz: float, seed: int = 3, lo: int = 128, hi: int = 16384,
                   glued_frac: float = 0.3):
    """Serving workload: Poisson arrivals (exponential gaps at rate_hz) of problems with n
    log-uniform in [lo, hi]; a fraction glued_frac are glued W_21^+, the rest U[-1,1].
    Returns a list of (arrival_s, d, e, w)."""
    g = rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += g.exponential(1.0 / rate_hz)
        n = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        if g.uniform() < glued_frac:
            gg = max(1, int(round(n / 21)))
            d, e = glued_wilkinson(gg, 1e-10)
        else:
            d, e = uniform(n, seed=seed * 7919 + r)
        out.append((t, d, e, eigenvalues(d, e)))
    return out
