"""The seeded input generators shared by the oracle's tests and the GPU path.

Each generator is checked against the recipe it states (value bounds, the
diagonal shift, symmetry and positive definiteness, the log-uniform order
law, the unit-triangular factors of the exact pins, Poisson statistics) and
for determinism: the same seed gives the same bytes, so the oracle and the
GPU library see identical inputs.
"""
import math

import numpy as np
import pytest

from paper_2305_11103_gb300 import inputs


@pytest.mark.parametrize("make", [
    lambda s: inputs.diag_dominant_uniform(64, s),
    lambda s: inputs.gaussian_shifted(64, s),
    lambda s: inputs.spd_covariance(32, s),
    lambda s: inputs.spd_covariance_batch(8, 5, s),
    lambda s: inputs.log_uniform_sizes(100, 8, 512, s),
    lambda s: inputs.unimodular_block_lu([3, 5, 4], s)[0],
    lambda s: inputs.poisson_arrivals(100.0, 1.0, s),
])
def test_same_seed_same_bytes(make):
    a, b, c = make(11), make(11), make(12)
    assert a.tobytes() == b.tobytes()
    assert a.shape != c.shape or a.tobytes() != c.tobytes()


def test_diag_dominant_uniform_bounds():
    n = 200
    a = inputs.diag_dominant_uniform(n, 1)
    off = a[~np.eye(n, dtype=bool)]
    assert off.min() >= -1.0 and off.max() <= 1.0
    d = np.diag(a)
    assert d.min() >= n - 1.0 and d.max() <= n + 1.0
    # every row strictly diagonally dominant: n - 1 entries of magnitude below 1
    # against a diagonal of at least n - 1
    assert np.all(np.abs(a).sum(axis=1) - np.abs(d) < d)
    b = inputs.diag_dominant_uniform(n, 1, shift=3.0)
    assert np.array_equal(b - np.diag(np.diag(b)), a - np.diag(np.diag(a)))
    assert np.allclose(np.diag(a) - np.diag(b), n - 3.0)


def test_gaussian_shifted_moments_and_conditioning():
    n = 512
    a = inputs.gaussian_shifted(n, 3, sigma=1.5)
    g = a - 1.5 * np.eye(n)
    # entries N(0, 1/n): the sample variance of n^2 entries is within a few % of 1/n
    assert abs(g.mean()) < 5.0 / n
    assert abs(g.var() * n - 1.0) < 0.02
    # the spectrum of N(0,1)/sqrt(n) fills the unit disc, so sigma = 1.5 keeps A well
    # away from singular; sigma = 1.05 (the harder headline case) is worse but finite
    s = np.linalg.svd(a, compute_uv=False)
    assert s[-1] > 0.1 and s[0] / s[-1] < 100.0
    s2 = np.linalg.svd(inputs.gaussian_shifted(n, 4, sigma=1.05), compute_uv=False)
    assert s2[0] / s2[-1] > s[0] / s[-1]


def test_spd_covariance_is_spd():
    for n, seed in ((5, 5), (11, 5), (64, 9)):
        a = inputs.spd_covariance(n, seed)
        assert np.allclose(a, a.T, rtol=0, atol=1e-12 * np.abs(a).max())
        w = np.linalg.eigvalsh((a + a.T) / 2)
        assert w.min() >= 0.1 * (1 - 1e-9)


def test_spd_covariance_batch_is_spd_and_batch_major():
    c = inputs.spd_covariance_batch(50, 5, 5)
    assert c.shape == (50, 5, 5)
    assert np.allclose(c, np.transpose(c, (0, 2, 1)), rtol=0, atol=1e-12)
    w = np.linalg.eigvalsh(c)
    assert w.min() >= 0.1 * (1 - 1e-9)
    # each matrix is B B^T + 0.1 I for its own B: they differ
    assert not np.allclose(c[0], c[1])


def test_log_uniform_sizes_law():
    lo, hi = 8, 512
    v = inputs.log_uniform_sizes(20000, lo, hi, 6)
    assert v.dtype == np.int64 and v.min() >= lo and v.max() <= hi
    # half the mass lies below the geometric mean; a quarter below lo^(3/4) hi^(1/4)
    gm = math.sqrt(lo * hi)
    assert abs(np.mean(v < gm) - 0.5) < 0.02
    q1 = lo ** 0.75 * hi ** 0.25
    assert abs(np.mean(v < q1) - 0.25) < 0.02


def test_uneven_batch_orders_and_shift():
    mats = inputs.uneven_batch(40, 8, 64, 6)
    sizes = inputs.log_uniform_sizes(40, 8, 64, 6)
    assert [m.shape[0] for m in mats] == list(sizes)
    for m in mats:
        n = m.shape[0]
        assert m.shape == (n, n)
        d = np.diag(m)
        assert d.min() >= n - 1.0 and d.max() <= n + 1.0
        assert np.abs(m - np.diag(d)).max() <= 1.0


@pytest.mark.parametrize("sizes", [[3, 5, 4], [1, 1, 1, 1], [7], [2, 6, 1, 5]])
def test_unimodular_block_lu_structure(sizes):
    a, L, U = inputs.unimodular_block_lu(sizes, 13)
    n = sum(sizes)
    assert a.shape == (n, n)
    assert np.array_equal(a, L @ U)
    assert np.array_equal(a, np.rint(a))
    # U unit upper triangular, L unit lower with identity diagonal blocks
    assert np.array_equal(np.tril(U), np.eye(n))
    assert np.array_equal(np.triu(L), np.eye(n))
    off = 0
    for m in sizes:
        assert np.array_equal(L[off:off + m, off:off + m], np.eye(m))
        off += m
    assert set(np.unique(L)) <= {-1.0, 0.0, 1.0}
    assert set(np.unique(U)) <= {-1.0, 0.0, 1.0}
    # det A = det L det U = 1, so A^-1 is an integer matrix
    assert round(np.linalg.det(a)) == 1


def test_poisson_arrivals_statistics():
    rate, dur = 2000.0, 5.0
    t = inputs.poisson_arrivals(rate, dur, 7)
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < dur
    # count ~ Poisson(rate * dur): within 5 standard deviations
    mean = rate * dur
    assert abs(len(t) - mean) < 5 * math.sqrt(mean)
    gaps = np.diff(t)
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1.0) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
