"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

None of these re-types the oracle's formula. They use exact rational
arithmetic, closed forms of special structure, a different identity of the
paper (Eq. (d)), invariants of the inverse, LAPACK as a third opinion, and the
paper's partition table. The last test builds oracle variants with planted
mistakes and shows that each one fails at least one pin.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.oracle import OracleError
from paper_2305_11103_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers ---
def rational_inverse(M):
    """Exact inverse of an integer (or rational) matrix by fraction Gauss-Jordan."""
    n = len(M)
    a = [[Fraction(int(v)) if float(v).is_integer() else Fraction(v) for v in row] + [Fraction(int(i == j)) for j in range(n)]
         for i, row in enumerate(np.asarray(M).tolist())]
    for c in range(n):
        r = next(i for i in range(c, n) if a[i][c] != 0)
        a[c], a[r] = a[r], a[c]
        piv = a[c][c]
        a[c] = [v / piv for v in a[c]]
        for i in range(n):
            if i != c and a[i][c] != 0:
                f = a[i][c]
                a[i] = [vi - f * vc for vi, vc in zip(a[i], a[c])]
    return [row[n:] for row in a]


def read_table(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":")
            rows[int(k)] = [int(t) for t in v.split()]
    return rows


def rel_err(X, Y):
    return np.linalg.norm(X - Y) / np.linalg.norm(Y)


PARTITIONS = [[1, 1], [2, 3], [3, 2], [1, 2, 3, 4], [4, 4, 4, 4], [5, 7, 1, 3, 8], [8, 8, 8, 8], [3] * 10 + [2]]


# ------------------------------------------------------- partition rules ---
def test_paper_partition_table():
    for m, sizes in read_table("paper_partition_table.txt").items():
        assert oracle.paper_partition(m) == sizes, m


def test_paper_block_counts():
    for m, (nk,) in read_table("paper_block_counts.txt").items():
        s = oracle.paper_partition(m)
        assert len(s) == nk and sum(s) == m and set(s) <= {2, 3, 4}


def test_paper_partition_all_orders():
    for m in range(2, 600):
        s = oracle.paper_partition(m)
        assert sum(s) == m and set(s) <= {2, 3, 4}
        assert s == sorted(s)                       # remainder sits in the last blocks
        assert len(s) & (len(s) - 1) == 0           # a power of two


def test_quarter_partition():
    for m in range(4, 300):
        s = oracle.quarter_partition(m)
        assert len(s) == 4 and sum(s) == m
        assert s == sorted(s) and s[-1] - s[0] <= 1 and s[0] == m // 4


# ---------------------------------------------------- exact integer pins ---
@pytest.mark.parametrize("sizes", PARTITIONS)
@pytest.mark.parametrize("seed", [11, 12])
def test_unimodular_exact(sizes, seed):
    """A = L U (block-unit-lower times unit-upper, integer): the blockwise
    inverse is an integer matrix and every step is exact in FP64."""
    A, L, U = inputs.unimodular_block_lu(sizes, seed)
    exact = rational_inverse(A)
    assert all(abs(v) < 2**53 for row in exact for v in row)
    assert all(v.denominator == 1 for row in exact for v in row)
    X = oracle.block_inverse(A, sizes)
    assert np.array_equal(X, np.array([[float(v) for v in row] for row in exact]))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_rational_bruteforce(n):
    g = inputs.rng(100 + n)
    for trial in range(6):
        A = g.integers(-5, 6, size=(n, n)).astype(np.float64)
        if abs(np.linalg.det(A)) < 0.5:
            A += 7 * np.eye(n)
        cuts = sorted(g.choice(np.arange(1, n), size=min(n - 1, trial % 3), replace=False)) if n > 1 else []
        sizes = list(np.diff([0, *cuts, n]))
        try:
            X = oracle.block_inverse(A, sizes)
        except OracleError:
            # a leading block or a Schur complement is singular for this partition
            continue
        exact = np.array([[float(v) for v in row] for row in rational_inverse(A)])
        assert rel_err(X, exact) <= 1e-13 * max(1.0, np.linalg.cond(A))


# --------------------------------------------------------- closed forms ---
def test_scalar_2x2_closed_form():
    g = inputs.rng(3)
    for _ in range(20):
        a, b, c, d = g.uniform(-2, 2, size=4)
        det = a * d - b * c
        if abs(det) < 1e-3 or abs(a) < 1e-3:
            continue
        expect = np.array([[d, -b], [-c, a]]) / det
        X = oracle.block_inverse(np.array([[a, b], [c, d]]), [1, 1])
        assert np.allclose(X, expect, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("sizes", [[3, 5], [4, 4, 2], [6, 1, 7]])
def test_block_triangular_and_diagonal(sizes):
    n = sum(sizes)
    g = inputs.rng(4)
    A = g.uniform(-1, 1, (n, n)) + n * np.eye(n)
    m0 = sizes[0]
    Aup = A.copy()
    Aup[m0:, :m0] = 0.0                              # C = 0: block upper triangular
    Ai = np.linalg.inv(Aup[:m0, :m0])
    Di = np.linalg.inv(Aup[m0:, m0:])
    expect = np.zeros_like(A)
    expect[:m0, :m0] = Ai
    expect[:m0, m0:] = -Ai @ Aup[:m0, m0:] @ Di
    expect[m0:, m0:] = Di
    assert rel_err(oracle.block_inverse(Aup, sizes), expect) < 1e-14
    Adiag = np.zeros_like(A)
    off = 0
    for m in sizes:
        Adiag[off:off + m, off:off + m] = A[off:off + m, off:off + m]
        off += m
    X = oracle.block_inverse(Adiag, sizes)
    off = 0
    for m in sizes:
        blk = X[off:off + m, off:off + m]
        assert rel_err(blk, np.linalg.inv(Adiag[off:off + m, off:off + m])) < 1e-14
        off += m
    assert np.count_nonzero(X) == sum(m * m for m in sizes)


def test_small_inverse_closed_form_vs_exact():
    g = inputs.rng(5)
    for m in (1, 2, 3):
        for _ in range(10):
            A = g.integers(-9, 10, size=(m, m)).astype(np.float64)
            if round(np.linalg.det(A)) == 0:
                continue
            exact = np.array([[float(v) for v in row] for row in rational_inverse(A)])
            assert np.allclose(oracle.small_inverse(A), exact, rtol=4e-16 * 8, atol=0)
            assert np.allclose(oracle.gj_inverse(A), exact, rtol=4e-16 * 8 * m, atol=1e-15)


# -------------------------------------------- a different identity: Eq. (d) ---
@pytest.mark.parametrize("sizes", [[5, 9], [8, 8], [12, 3]])
def test_eq_d_cross_check(sizes):
    """Eq. (d) gives the top-left block as S_D^-1 with S_D = A - B D^-1 C and
    the bottom-left as -D^-1 C S_D^-1; Eq. (ad) combines S_D^-1 with S_A^-1."""
    n = sum(sizes)
    A = inputs.gaussian_shifted(n, 21, sigma=2.0)
    m0 = sizes[0]
    a, b, c, d = A[:m0, :m0], A[:m0, m0:], A[m0:, :m0], A[m0:, m0:]
    Di = np.linalg.inv(d)
    SDi = np.linalg.inv(a - b @ Di @ c)
    SAi = np.linalg.inv(d - c @ np.linalg.inv(a) @ b)
    X = oracle.block_inverse(A, sizes)
    assert rel_err(X[:m0, :m0], SDi) < 1e-13
    assert rel_err(X[m0:, :m0], -Di @ c @ SDi) < 1e-13
    assert rel_err(X[m0:, m0:], SAi) < 1e-13


# ------------------------------------------------------------ invariants ---
@pytest.mark.parametrize("sizes", [[64] * 4, [16, 48, 7, 33], [2, 3] * 6])
def test_invariants(sizes):
    n = sum(sizes)
    A = inputs.diag_dominant_uniform(n, 31, shift=n)
    X = oracle.block_inverse(A, sizes)
    eye = np.eye(n)
    assert np.linalg.norm(A @ X - eye) / (np.linalg.norm(A) * np.linalg.norm(X)) < 1e-15
    assert np.linalg.norm(X @ A - eye) / (np.linalg.norm(A) * np.linalg.norm(X)) < 1e-15
    assert oracle.residual(A, X) < 1e-15
    # inverse of the inverse
    assert rel_err(oracle.block_inverse(X, sizes), A) < 1e-13
    # transpose: the same partition applies to A^T
    assert rel_err(oracle.block_inverse(A.T.copy(), sizes), X.T) < 1e-13
    # power-of-two scaling is exact
    assert np.array_equal(oracle.block_inverse(A * 8.0, sizes), X / 8.0)
    # LAPACK as a third opinion
    assert rel_err(X, np.linalg.inv(A)) < 1e-14


def test_spd_gives_symmetric():
    A = inputs.spd_covariance(24, 41)
    X = oracle.block_inverse(A, [6, 6, 6, 6])
    assert np.linalg.norm(X - X.T) / np.linalg.norm(X) < 24 * 2.0**-52 * np.linalg.cond(A)


def test_block_permutation():
    """Permuting whole blocks of equal order: (P A P^T)^-1 = P A^-1 P^T."""
    sizes = [5] * 4
    A = inputs.diag_dominant_uniform(20, 42, shift=20)
    perm_blocks = [2, 0, 3, 1]
    perm = np.concatenate([np.arange(5 * b, 5 * b + 5) for b in perm_blocks])
    P = np.eye(20)[perm]
    X = oracle.block_inverse(A, sizes)
    Xp = oracle.block_inverse(P @ A @ P.T, sizes)
    assert rel_err(Xp, P @ X @ P.T) < 1e-14


def test_singular_detection():
    # permutation matrix: every leading block is singular (Sec. 3, counter-diagonal case)
    J = np.fliplr(np.eye(6))
    with pytest.raises(OracleError) as e:
        oracle.block_inverse(J, [3, 3])
    assert e.value.status == -2 and e.value.failing_block == 0
    # non-singular leading block, singular Schur complement in block 2
    A = np.eye(6)
    A[4, 5] = A[5, 4] = 1.0                   # last 2x2 block [[1,1],[1,1]] is singular
    with pytest.raises(OracleError) as e:
        oracle.block_inverse(A, [2, 2, 2])
    assert e.value.failing_block == 2
    with pytest.raises(OracleError) as e:
        oracle.block_inverse(np.full((4, 4), np.nan), [2, 2])
    assert e.value.status == -2


def test_bad_arguments():
    with pytest.raises(OracleError):
        oracle.block_inverse(np.eye(4), [2, 1])
    with pytest.raises(OracleError):
        oracle.block_inverse(np.eye(4), [4, 0])


# ---------------------------------------------- residual and Newton-Schulz ---
def test_residual_closed_form():
    A, _, _ = inputs.unimodular_block_lu([4, 4, 4], 7)
    X = np.array([[float(v) for v in row] for row in rational_inverse(A)])
    assert oracle.residual(A, X) == 0.0
    # X = 2 A^-1 gives ||2I - I||_F / (||A||_F ||2 A^-1||_F)
    expect = np.sqrt(12) / (np.linalg.norm(A) * np.linalg.norm(2 * X))
    assert abs(oracle.residual(A, 2 * X) - expect) <= 1e-14 * expect


def test_ns_step_quadratic():
    n = 48
    A = inputs.gaussian_shifted(n, 51, sigma=1.5)
    Xe = np.linalg.inv(A)
    g = inputs.rng(52)
    X0 = Xe @ (np.eye(n) + 1e-3 * g.standard_normal((n, n)))
    e0 = np.linalg.norm(np.eye(n) - A @ X0, 2)
    X1 = oracle.ns_step(A, X0)
    e1 = np.linalg.norm(np.eye(n) - A @ X1, 2)
    assert e1 <= 1.01 * e0 ** 2 + 1e-14
    # the exact inverse is a fixed point (up to rounding)
    assert rel_err(oracle.ns_step(A, Xe), Xe) < 1e-14


# ------------------------------------------------- the pins catch mistakes ---
def _pin_suite(mutant):
    """Run a compact pin subset against one oracle build; return the failures."""
    fails = []
    for sizes in ([2, 3], [4, 4, 4], [1, 2, 3, 4]):
        A, _, _ = inputs.unimodular_block_lu(sizes, 13)
        exact = np.array([[float(v) for v in row] for row in rational_inverse(A)])
        try:
            if not np.array_equal(oracle.block_inverse(A, sizes, mutant=mutant), exact):
                fails.append(("unimodular", sizes))
        except OracleError:
            fails.append(("unimodular-raise", sizes))
    A = inputs.diag_dominant_uniform(12, 3)
    B = A.copy()
    B[[0, 5]] = B[[5, 0]]                        # forces a row swap inside a block
    try:
        X = oracle.block_inverse(B, [6, 6], mutant=mutant)
        if rel_err(X, np.linalg.inv(B)) > 1e-12:
            fails.append(("lapack", "swap"))
    except OracleError:
        fails.append(("lapack-raise", "swap"))
    # closed forms of orders 2 and 3 against exact rationals
    g = inputs.rng(5)
    for m in (2, 3):
        A = g.integers(-9, 10, size=(m, m)).astype(np.float64)
        while round(np.linalg.det(A)) == 0:
            A = g.integers(-9, 10, size=(m, m)).astype(np.float64)
        exact = np.array([[float(v) for v in row] for row in rational_inverse(A)])
        if not np.allclose(oracle.small_inverse(A, mutant=mutant), exact, rtol=4e-16 * 8, atol=0):
            fails.append(("closed form", m))
    # the paper's partition table
    for m, sizes in read_table("paper_partition_table.txt").items():
        if oracle.paper_partition(m, mutant=mutant) != sizes:
            fails.append(("table 2", m))
            break
    # four near-equal blocks, the larger ones last
    for m in (9, 10, 11):
        q = oracle.quarter_partition(m, mutant=mutant)
        if sum(q) != m or q != sorted(q) or q[0] != m // 4:
            fails.append(("quarters", m))
            break
    # rho of the exact inverse and of twice it
    A, _, _ = inputs.unimodular_block_lu([4, 4, 4], 7)
    X = np.array([[float(v) for v in row] for row in rational_inverse(A)])
    expect = np.sqrt(12) / (np.linalg.norm(A) * np.linalg.norm(2 * X))
    if oracle.residual(A, X, mutant=mutant) != 0.0 or \
            abs(oracle.residual(A, 2 * X, mutant=mutant) - expect) > 1e-14 * expect:
        fails.append(("rho", "closed form"))
    # one Newton-Schulz step squares the right residual
    n = 24
    A = inputs.gaussian_shifted(n, 51, sigma=1.5)
    X0 = np.linalg.inv(A) @ (np.eye(n) + 1e-3 * inputs.rng(52).standard_normal((n, n)))
    e0 = np.linalg.norm(np.eye(n) - A @ X0, 2)
    e1 = np.linalg.norm(np.eye(n) - A @ oracle.ns_step(A, X0, mutant=mutant), 2)
    if e1 > 1.01 * e0 ** 2 + 1e-14:
        fails.append(("newton-schulz", "quadratic"))
    return fails


def test_pins_pass_on_real_oracle():
    assert _pin_suite(0) == []


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_pins_catch_planted_mistakes(mutant):
    oracle.build_oracle(mutant=mutant)
    assert _pin_suite(mutant), f"mutant {mutant} passed every pin"
