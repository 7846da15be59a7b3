"""Seeded synthetic inputs shaped like the paper's workloads.

The paper inverts "random generated matrices" (Sec. 5, performance
discussion) and, in its motivating physics use, many small covariance-like
systematics matrices (Sec. 2). No dataset is public or needed; every input
here comes from numpy's PCG64 generator with an explicit seed, row-major
FP64, and the same bytes go to the CPU oracle and to the GPU library.

This module holds no arithmetic of the inversion method. It is shared by the
oracle's tests and by the GPU path's tests and benchmark, and imports
nothing from either.
"""
import math

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def diag_dominant_uniform(n, seed, shift=None):
    """Entries iid U[-1, 1], plus `shift` on the diagonal (default n)."""
    g = rng(seed)
    a = g.uniform(-1.0, 1.0, size=(n, n))
    a[np.diag_indices(n)] += float(n if shift is None else shift)
    return a


def gaussian_shifted(n, seed, sigma=1.5):
    """Entries iid N(0, 1)/sqrt(n), plus sigma * I (well conditioned for sigma > 1)."""
    g = rng(seed)
    a = g.standard_normal(size=(n, n)) / math.sqrt(n)
    a[np.diag_indices(n)] += sigma
    return a


def spd_covariance(n, seed, ridge=0.1):
    """B B^T + ridge * I with B iid N(0, 1): symmetric positive definite."""
    g = rng(seed)
    b = g.standard_normal(size=(n, n))
    return b @ b.T + ridge * np.eye(n)


def spd_covariance_batch(count, n, seed, ridge=0.1):
    """count matrices B B^T + ridge * I, batch-major (count, n, n)."""
    g = rng(seed)
    b = g.standard_normal(size=(count, n, n))
    return np.einsum("bij,bkj->bik", b, b) + ridge * np.eye(n)[None]


def log_uniform_sizes(count, lo, hi, seed):
    """count integer orders round(exp(U(ln lo, ln hi)))."""
    g = rng(seed)
    v = np.exp(g.uniform(math.log(lo), math.log(hi), size=count))
    return np.clip(np.rint(v).astype(np.int64), lo, hi)


def uneven_batch(count, lo, hi, seed):
    """count diagonally dominant matrices (U[-1,1] + n I) of log-uniform order."""
    sizes = log_uniform_sizes(count, lo, hi, seed)
    g = rng(seed + 1_000_003)
    mats = []
    for n in sizes:
        a = g.uniform(-1.0, 1.0, size=(int(n), int(n)))
        a[np.diag_indices(int(n))] += float(n)
        mats.append(a)
    return mats


def unimodular_block_lu(sizes, seed, lower_density=0.5):
    """Integer matrix A = L U whose blockwise inversion is exact in FP64.

    L is block-unit-lower for the partition `sizes` (identity diagonal blocks,
    random entries in {-1, 0, 1} strictly below them); U is unit upper
    triangular with entries in {-1, 0, 1} above the diagonal. Every pivot
    block and Schur complement met by a blockwise elimination over `sizes` is
    then a diagonal block of U (unit upper triangular), so partial pivoting
    always selects a diagonal 1 and every intermediate is an integer.
    Returns (A, L, U) as float64 arrays of small integers.
    """
    g = rng(seed)
    n = int(sum(sizes))
    L = np.eye(n)
    U = np.eye(n)
    off = 0
    for m in sizes:
        below = slice(off + m, n)
        blk = g.integers(-1, 2, size=(n - off - m, m)).astype(np.float64)
        mask = g.random(size=blk.shape) < lower_density
        L[below, off:off + m] = blk * mask
        off += m
    iu = np.triu_indices(n, 1)
    U[iu] = g.integers(-1, 2, size=len(iu[0])).astype(np.float64)
    return L @ U, L, U


def poisson_arrivals(rate_per_s, duration_s, seed):
    """Arrival times (seconds) of a Poisson process."""
    g = rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return np.array(out)
        out.append(t)
