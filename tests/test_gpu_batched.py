"""Batched small-matrix inversion (orders 1..8, one thread per matrix) through
the C ABI, against the oracle with the same partition (the paper's Table 2
rule) and against the residual gate rho <= 1e-12 per matrix."""
import numpy as np
import pytest

import oracle
from paper_2305_11103_gb300 import inputs
from tolerance import eps_max, eps_norm, fwd_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def bi(cuda_device):
    from paper_2305_11103_gb300 import build as libbuild
    libbuild.build()
    from paper_2305_11103_gb300 import blockinv
    blockinv.lib()
    return blockinv


def close_to_oracle(A, X, Xo, tag=""):
    """Normwise and elementwise error against the oracle within
    16 sqrt(n) kappa_2 u (see tests/tolerance.py)."""
    b = fwd_bound(A, Xo)
    assert eps_norm(X, Xo) <= b, (tag, eps_norm(X, Xo), b)
    assert eps_max(X, Xo) <= b, (tag, eps_max(X, Xo), b)


def batched_rho(A, X):
    n = A.shape[-1]
    R = np.einsum("bij,bjk->bik", A, X) - np.eye(n)[None]
    return np.linalg.norm(R, axis=(1, 2)) / (np.linalg.norm(A, axis=(1, 2)) * np.linalg.norm(X, axis=(1, 2)))


def run(bi, A):
    count, n, _ = A.shape
    d = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    st = torch.full((count,), 99, dtype=torch.int32, device="cuda")
    assert bi.blockinv_invert_batched_small(count, n, d.data_ptr(), st.data_ptr(), None) == bi.OK
    torch.cuda.synchronize()
    return d.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("count", [1, 127, 1000])
def test_small_orders_vs_oracle(bi, n, count):
    g = inputs.rng(500 + 10 * n + count)
    A = g.uniform(-1, 1, size=(count, n, n)) + n * np.eye(n)[None]
    X, st = run(bi, A)
    assert np.all(st == 0)
    sizes = oracle.paper_partition(n) if n >= 2 else [1]
    assert np.all(batched_rho(A, X) <= 1e-12)
    for m in range(0, count, max(1, count // 25)):
        Xo = oracle.block_inverse(A[m], sizes)
        close_to_oracle(A[m], X[m], Xo)


def test_spd_5x5_full_batch(bi):
    """200 000 SPD 5 x 5 matrices B B^T + 0.1 I, B iid N(0, 1), seed 5."""
    A = inputs.spd_covariance_batch(200_000, 5, 5)
    X, st = run(bi, A)
    assert np.all(st == 0)
    assert np.all(batched_rho(A, X) <= 1e-12)
    g = inputs.rng(55)
    for m in g.choice(200_000, size=50, replace=False):
        Xo = oracle.block_inverse(A[m], [2, 3])
        close_to_oracle(A[m], X[m], Xo)
    # SPD input: symmetric inverse up to rounding
    assert np.max(np.abs(X - X.transpose(0, 2, 1)) / np.abs(X).max(axis=(1, 2))[:, None, None]) < 1e-9


def test_exact_unimodular_batch(bi):
    mats = [inputs.unimodular_block_lu([2, 3], 900 + k)[0] for k in range(64)]
    A = np.stack(mats)
    X, st = run(bi, A)
    assert np.all(st == 0)
    for m in range(64):
        assert np.array_equal(X[m], oracle.block_inverse(A[m], [2, 3]))


def test_per_matrix_status(bi):
    g = inputs.rng(77)
    A = g.uniform(-1, 1, size=(300, 5, 5)) + 5 * np.eye(5)[None]
    A[10] = np.fliplr(np.eye(5))            # leading 2 x 2 block singular
    A[20, :2, :2] = [[1.0, 2.0], [2.0, 4.0]]  # singular leading block again
    A[30, 3, 3] = np.nan
    keep = A.copy()
    X, st = run(bi, A)
    assert st[10] == bi.ERR_SINGULAR and st[20] == bi.ERR_SINGULAR and st[30] == bi.ERR_NONFINITE
    ok = np.ones(300, bool)
    ok[[10, 20, 30]] = False
    assert np.all(st[ok] == 0)
    assert np.array_equal(X[10], keep[10]) and np.array_equal(X[20], keep[20])
    assert np.all(batched_rho(A[ok], X[ok]) <= 1e-12)


def test_argument_errors(bi):
    assert bi.blockinv_invert_batched_small(10, 9, 0x1000, None, None) == bi.ERR_INVALID
    assert bi.blockinv_invert_batched_small(10, 0, 0x1000, None, None) == bi.ERR_INVALID
    assert bi.blockinv_invert_batched_small(0, 5, None, None, None) == bi.OK


# ------------------------------------------------- uneven (grouped) batches ---
def device_batch(mats):
    ts = [torch.from_numpy(np.ascontiguousarray(A)).cuda() for A in mats]
    return ts, [t.data_ptr() for t in ts], [t.shape[0] for t in ts]


def quarter(n):
    if n < 8:
        return oracle.paper_partition(n) if n >= 2 else [1]
    return oracle.quarter_partition(n)


def test_uneven_default_partition_vs_oracle(bi):
    mats = inputs.uneven_batch(60, 8, 300, 61)
    ts, ptrs, ns = device_batch(mats)
    st = torch.full((60,), 7, dtype=torch.int32, device="cuda")
    assert bi.blockinv_invert_batched(ns, None, ptrs, ns, bi.F64, None, st.data_ptr()) == bi.OK
    assert torch.all(st == 0)
    for A, t in zip(mats, ts):
        X = t.cpu().numpy()
        n = A.shape[0]
        Xo = oracle.block_inverse(A, quarter(n))
        assert np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e-12
        close_to_oracle(A, X, Xo)


def test_uneven_explicit_partitions_and_large_block(bi):
    parts = [[3, 4], [100, 157], [1, 1, 1], [200, 200], [64] * 5 + [3], [129]]
    mats = [inputs.gaussian_shifted(sum(q), 62 + i, sigma=1.5) for i, q in enumerate(parts)]
    ts, ptrs, ns = device_batch(mats)
    st = torch.full((len(mats),), 7, dtype=torch.int32, device="cuda")
    assert bi.blockinv_invert_batched(ns, parts, ptrs, ns, bi.F64, None, st.data_ptr()) == bi.OK
    assert torch.all(st == 0)
    for A, t, q in zip(mats, ts, parts):
        X = t.cpu().numpy()
        Xo = oracle.block_inverse(A, q)
        close_to_oracle(A, X, Xo)


def test_uneven_status_and_plan_replay(bi):
    mats = inputs.uneven_batch(40, 8, 200, 63)
    mats[5] = np.fliplr(np.eye(mats[5].shape[0])).copy()   # singular leading block
    ts, ptrs, ns = device_batch(mats)
    plan = bi.BatchPlan(ns, None, ptrs, ns)
    st = torch.full((40,), 7, dtype=torch.int32, device="cuda")
    first = None
    for rep in range(3):     # the first run captures the graph, the others replay it
        for A, t in zip(mats, ts):
            t.copy_(torch.from_numpy(A))
        assert plan.run(None, st.data_ptr()) == bi.OK
        torch.cuda.synchronize()
        assert st[5].item() == bi.ERR_SINGULAR
        ok = [i for i in range(40) if i != 5]
        assert all(st[i].item() == 0 for i in ok)
        res = [ts[i].cpu().numpy() for i in ok]
        if first is None:
            first = res
        else:
            assert all(np.array_equal(a, b) for a, b in zip(first, res))
    plan.close()


def test_uneven_full_config(bi):
    """2000 matrices, n = round(exp(U(ln 8, ln 512))), U[-1,1] + n I, seed 6."""
    mats = inputs.uneven_batch(2000, 8, 512, 6)
    ts, ptrs, ns = device_batch(mats)
    st = torch.full((2000,), 7, dtype=torch.int32, device="cuda")
    assert bi.blockinv_invert_batched(ns, None, ptrs, ns, bi.F64, None, st.data_ptr()) == bi.OK
    assert torch.all(st == 0)
    g = inputs.rng(66)
    for i in g.choice(2000, size=25, replace=False):
        A, X = mats[i], ts[i].cpu().numpy()
        n = A.shape[0]
        assert np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e-12
        Xo = oracle.block_inverse(A, quarter(n))
        close_to_oracle(A, X, Xo)


def test_batched_argument_errors(bi):
    t = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    assert bi.blockinv_invert_batched([8], [[4, 3]], [t.data_ptr()], [8]) == bi.ERR_INVALID
    assert bi.blockinv_invert_batched([8], None, [t.data_ptr()], [7]) == bi.ERR_INVALID
    assert bi.blockinv_invert_batched([8], None, [t.data_ptr()], [8], mode="tf32") == bi.ERR_INVALID


def _check_batch(mats, ts, parts=None, sample=None):
    idx = range(len(mats)) if sample is None else sample
    for i in idx:
        A, X = mats[i], ts[i].cpu().numpy()
        n = A.shape[0]
        assert np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e-12
        Xo = oracle.block_inverse(A, parts[i] if parts else quarter(n))
        close_to_oracle(A, X, Xo)


def _size_class(n):
    return int(np.floor(np.log2(n)))


def test_table_single_block_classes_vs_oracle(bi):
    """Size classes given one block: their matrices have no Schur tiles at all
    (the Schur launches count tiles over the rows outside the pivot block)
    and are inverted by the pivot kernels and the row panel alone."""
    mats = inputs.uneven_batch(60, 8, 200, 69)
    ns = [A.shape[0] for A in mats]
    assert bi.blockinv_batch_tuning_clear() == bi.OK
    for c in range(3, 8):
        assert bi.blockinv_batch_tuning_set(c, 1 if c % 2 else 3, 32) == bi.OK
    try:
        ts, ptrs, _ = device_batch(mats)
        st = torch.full((60,), 7, dtype=torch.int32, device="cuda")
        assert bi.blockinv_invert_batched(ns, None, ptrs, ns, bi.F64, None, st.data_ptr()) == bi.OK
        torch.cuda.synchronize()
        assert torch.all(st == 0)
        parts = []
        for n in ns:
            p = 1 if _size_class(n) % 2 else 3
            q, r = divmod(n, p)
            parts.append([q + (1 if i >= p - r else 0) for i in range(p)])
        _check_batch(mats, ts, parts)
    finally:
        bi.blockinv_batch_tuning_clear()


def test_table_partition_and_32_tiles_vs_oracle(bi):
    """Table entries set by hand: p near-equal blocks and 32 x 32 Schur tiles."""
    mats = inputs.uneven_batch(80, 8, 300, 65)
    ns = [A.shape[0] for A in mats]
    assert bi.blockinv_batch_tuning_clear() == bi.OK
    for c in range(3, 9):
        assert bi.blockinv_batch_tuning_set(c, 2 if c < 5 else 5, 32 if c % 2 else 64) == bi.OK
    try:
        ts, ptrs, _ = device_batch(mats)
        st = torch.full((80,), 7, dtype=torch.int32, device="cuda")
        assert bi.blockinv_invert_batched(ns, None, ptrs, ns, bi.F64, None, st.data_ptr()) == bi.OK
        assert torch.all(st == 0)
        parts = []
        for n in ns:
            p = 2 if _size_class(n) < 5 else 5
            q, r = divmod(n, p)
            parts.append([q + (1 if i >= p - r else 0) for i in range(p)])
        _check_batch(mats, ts, parts)
    finally:
        bi.blockinv_batch_tuning_clear()


def test_autotuner_choices_are_valid_and_exact(bi):
    mats = inputs.uneven_batch(300, 8, 520, 64)
    ns = [A.shape[0] for A in mats]
    assert bi.blockinv_batch_tuning_clear() == bi.OK
    try:
        assert bi.blockinv_batch_tune(ns, 2) == bi.OK
        for c in sorted({_size_class(n) for n in ns}):
            st, p, tile = bi.blockinv_batch_tuning(c)
            members = [n for n in ns if _size_class(n) == c]
            assert st == bi.OK and tile in (32, 64) and 0 <= p <= min(members)   # 0: the default stays
            assert p == 0 or p == 1 or (-(-max(members) // p) <= 128 and min(members) // p >= 4)
        ts, ptrs, _ = device_batch(mats)
        st = torch.full((300,), 7, dtype=torch.int32, device="cuda")
        plan = bi.BatchPlan(ns, None, ptrs, ns)
        assert plan.run(None, st.data_ptr()) == bi.OK
        torch.cuda.synchronize()
        plan.close()
        assert torch.all(st == 0)
        parts = []
        for n in ns:
            p = bi.blockinv_batch_tuning(_size_class(n))[1]
            if p == 0:
                parts.append(quarter(n))
                continue
            q, r = divmod(n, p)
            parts.append([q + (1 if i >= p - r else 0) for i in range(p)])
        _check_batch(mats, ts, parts, sample=inputs.rng(67).choice(300, size=40, replace=False))
    finally:
        bi.blockinv_batch_tuning_clear()


# ------------------------------------- one order <= 32, one partition ---
def run_fixed(bi, A, sizes, flags=0):
    count, n, _ = A.shape
    d = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    st = torch.full((count,), 99, dtype=torch.int32, device="cuda")
    assert bi.blockinv_invert_batched_fixed(count, n, sizes, d.data_ptr(), flags, st.data_ptr()) == bi.OK
    torch.cuda.synchronize()
    return d.cpu().numpy(), st.cpu().numpy()


def _vs_oracle(A, X, sizes, idx):
    for i in idx:
        n = A.shape[1]
        Xo = oracle.block_inverse(A[i], sizes)
        close_to_oracle(A[i], X[i], Xo, i)


def test_tau_11x11_spd_blocks_5_6(bi):
    """The paper's 11 x 11 systematics matrices with blocks of 5 and 6 (Sec. 2):
    SPD B B^T + 0.1 I; exact symmetry of the result."""
    g = inputs.rng(80)
    B = g.standard_normal((3000, 11, 11))
    A = B @ B.transpose(0, 2, 1) + 0.1 * np.eye(11)[None]
    X, st = run_fixed(bi, A, [5, 6], bi.BATCH_SPD)
    assert np.all(st == 0)
    assert np.array_equal(X, X.transpose(0, 2, 1))
    assert np.all(batched_rho(A, X) <= 1e-12)
    _vs_oracle(A, X, [5, 6], range(0, 3000, 97))
    # the general path (pivot search) on the same inputs agrees within rounding
    Xg, stg = run_fixed(bi, A, [5, 6])
    assert np.all(stg == 0) and np.all(batched_rho(A, Xg) <= 1e-12)


@pytest.mark.parametrize("n", [1, 2, 5, 9, 11, 16, 17, 24, 32])
def test_fixed_orders_paper_partition_vs_oracle(bi, n):
    g = inputs.rng(81 + n)
    A = g.uniform(-1, 1, size=(257, n, n)) + n * np.eye(n)[None]
    X, st = run_fixed(bi, A, None)
    assert np.all(st == 0)
    assert np.all(batched_rho(A, X) <= 1e-12)
    _vs_oracle(A, X, oracle.paper_partition(n) if n >= 2 else [1], range(0, 257, 16))


def test_fixed_pivoting_inside_blocks(bi):
    """Rows permuted inside each block: the diagonal pivots are zero-free only
    after the search inside the block."""
    g = inputs.rng(82)
    n, sizes = 13, [4, 4, 5]
    base = g.uniform(-1, 1, size=(200, n, n)) + n * np.eye(n)[None]
    A = base.copy()
    o = 0
    for b in sizes:
        A[:, o:o + b] = A[:, o:o + b][:, ::-1]   # reverse the block's rows
        o += b
    X, st = run_fixed(bi, A, sizes)
    assert np.all(st == 0) and np.all(batched_rho(A, X) <= 1e-12)
    _vs_oracle(A, X, sizes, range(0, 200, 11))


def test_fixed_status_and_untouched_failures(bi):
    g = inputs.rng(83)
    n = 11
    A = g.uniform(-1, 1, size=(100, n, n)) + n * np.eye(n)[None]
    A[3, :5, :5] = 0.0          # singular first block
    A[7, 2, 9] = np.inf
    keep = A.copy()
    X, st = run_fixed(bi, A, [5, 6])
    assert st[3] == bi.ERR_SINGULAR and st[7] == bi.ERR_NONFINITE
    ok = np.ones(100, bool)
    ok[[3, 7]] = False
    assert np.all(st[ok] == 0) and np.all(batched_rho(A[ok], X[ok]) <= 1e-12)
    assert np.array_equal(X[3], keep[3]) and np.array_equal(X[7], keep[7])
