"""Seeded synthetic inputs: symmetric tridiagonal matrices of the paper's workloads.

This module holds none of the eigensolver's arithmetic; it only produces the
diagonal ``a`` and off-diagonal ``b`` (numpy float64) that both the CUDA path
and the CPU oracle are fed.  Generators use ``numpy.random.default_rng(seed)``.

Families:
  * ``uniform``   : a ~ U[lo_a, hi_a], b ~ U[lo_b, hi_b] (i.i.d.)
  * ``toeplitz``  : a_i = alpha, b_i = beta (Sec. 5, Example 3; closed-form spectrum)
  * ``clement``   : zero diagonal, b_i = sqrt(i (n + 1 - i)), dimension n + 1 (eq. Clement-Tri)
  * ``legendre``  : zero diagonal, b_i = i / sqrt((2i - 1)(2i + 1)), i = 2..n (eq. Legendre-Tri)
  * ``laguerre``  : a_i = 2i + 1, b_i = i + 1 (eq. Laguerre-Tri)
  * ``hermite``   : zero diagonal, b_i = sqrt(i) (eq. Hermite-Tri)
  * ``glued_wilkinson``: copies of the Wilkinson matrix W+_{2m+1} (diagonal |i - m|,
    off-diagonal 1) glued by off-diagonal ``glue`` and truncated to n (heavy deflation)
  * ``example1``  : the rank-one problem of Example 1: d_i = i (hi - lo) / N and a
    random unit vector u.
"""
import numpy as np


def uniform(n, seed, lo_a=-1.0, hi_a=1.0, lo_b=-1.0, hi_b=1.0):
    rng = np.random.default_rng(seed)
    a = rng.uniform(lo_a, hi_a, n)
    b = rng.uniform(lo_b, hi_b, max(n - 1, 0))
    return a, b


def toeplitz(n, alpha=2.0, beta=1.0):
    return np.full(n, float(alpha)), np.full(max(n - 1, 0), float(beta))


def clement(n_plus_1):
    n = n_plus_1 - 1
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.zeros(n_plus_1), np.sqrt(i * (n + 1 - i))


def legendre(n):
    i = np.arange(2, n + 1, dtype=np.float64)
    return np.zeros(n), i / np.sqrt((2 * i - 1) * (2 * i + 1))


def laguerre(n):
    i = np.arange(1, n + 1, dtype=np.float64)
    return 2 * i + 1, np.arange(2, n + 1, dtype=np.float64)


def hermite(n):
    return np.zeros(n), np.sqrt(np.arange(1, n, dtype=np.float64))


def glued_wilkinson(n, m=10, glue=1e-8):
    w = 2 * m + 1
    reps = (n + w - 1) // w
    blk_a = np.abs(np.arange(w) - m).astype(np.float64)
    a = np.tile(blk_a, reps)[:n]
    b = np.ones(reps * w - 1)
    b[w - 1::w] = glue
    return a, b[: max(n - 1, 0)]


def example1(N, seed, lo=1.0, hi=9.0):
    rng = np.random.default_rng(seed)
    d = np.arange(1, N + 1, dtype=np.float64) * (hi - lo) / N
    u = rng.standard_normal(N)
    u /= np.linalg.norm(u)
    return d, u


def batch_sizes(count, seed, lo=64, hi=2048):
    """Sizes of the batched workload: N_b uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count)


def batch(count, seed, lo=64, hi=2048):
    """Uneven batch: even members uniform U[-1, 1], odd members glued Wilkinson."""
    sizes = batch_sizes(count, seed, lo, hi)
    out = []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            out.append(uniform(int(n), seed * 100003 + i))
        else:
            out.append(glued_wilkinson(int(n)))
    return out
