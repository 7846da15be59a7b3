"""Resumable elimination: ranges of steps and checkpoints (the paper's
stop-and-resume by step) give the same bits as one blockinv_invert call."""
import numpy as np
import pytest

import oracle
from paper_2305_11103_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi(cuda_device):
    from paper_2305_11103_gb300 import build as libbuild
    libbuild.build()
    from paper_2305_11103_gb300 import blockinv
    blockinv.lib()
    return blockinv


def whole(bi, A, sizes):
    d = torch.from_numpy(A).cuda()
    assert bi.blockinv_invert(A.shape[0], sizes, d.data_ptr(), A.shape[0], bi.F64, None) == bi.OK
    return d.cpu().numpy()


@pytest.mark.parametrize("n,sizes,cuts", [
    (1000, [256, 256, 256, 232], [2]),
    (1000, [256, 256, 256, 232], [1, 2, 3]),
    (4096, [256] * 16, [5]),            # look-ahead inside each range
    (2300, [100] * 23, [0, 7, 7, 19]),  # empty ranges and misaligned blocks
])
def test_ranges_equal_whole_inversion(bi, n, sizes, cuts):
    A = inputs.gaussian_shifted(n, 70 + len(cuts), sigma=1.5)
    ref = whole(bi, A, sizes)
    d = torch.from_numpy(A).cuda()
    bounds = [0] + cuts + [len(sizes)]
    for k0, k1 in zip(bounds[:-1], bounds[1:]):
        assert bi.blockinv_invert_steps(n, sizes, d.data_ptr(), n, k0, k1) == bi.OK
    assert np.array_equal(d.cpu().numpy(), ref)


def test_checkpoint_resume_in_fresh_buffer(bi, tmp_path):
    n, sizes = 1500, [300, 300, 300, 300, 300]
    A = inputs.diag_dominant_uniform(n, 71, shift=n)
    ref = whole(bi, A, sizes)
    d = torch.from_numpy(A).cuda()
    assert bi.blockinv_invert_steps(n, sizes, d.data_ptr(), n, 0, 2) == bi.OK
    path = tmp_path / "state.ck"
    assert bi.blockinv_checkpoint_write(path, n, sizes, d.data_ptr(), n, 2) == bi.OK
    del d
    lda = 1536   # a different leading dimension on resume
    e = torch.full((n, lda), np.nan, dtype=torch.float64, device="cuda")
    st, k = bi.blockinv_checkpoint_read(path, n, sizes, e.data_ptr(), lda)
    assert st == bi.OK and k == 2
    assert bi.blockinv_invert_steps(n, sizes, e.data_ptr(), lda, k, len(sizes)) == bi.OK
    assert np.array_equal(e[:, :n].cpu().numpy(), ref)
    assert torch.isnan(e[:, n:]).all()
    Xo = oracle.block_inverse(A, sizes)
    assert np.linalg.norm(ref - Xo) / np.linalg.norm(Xo) <= 1e-12


def test_singular_block_reported_by_its_step(bi):
    n, sizes = 12, [4, 4, 4]
    A = np.eye(n)
    A[4:8, 4:8] = 0.0     # the second pivot block is zero
    d = torch.from_numpy(A).cuda()
    assert bi.blockinv_invert_steps(n, sizes, d.data_ptr(), n, 0, 1) == bi.OK
    assert bi.blockinv_invert_steps(n, sizes, d.data_ptr(), n, 1, 3) == bi.ERR_SINGULAR
    assert bi.blockinv_last_error_detail() == (bi.ERR_SINGULAR, 1)


# ---------------------------------------------- pivot order and fallbacks ---
def rho(A, X):
    return np.linalg.norm(A @ X - np.eye(A.shape[0])) / (np.linalg.norm(A) * np.linalg.norm(X))


def ex(bi, A, sizes, **kw):
    n = A.shape[0]
    d = torch.from_numpy(A).cuda()
    st, info = bi.blockinv_invert_ex(n, sizes, d.data_ptr(), n, bi.F64, None, **kw)
    return st, info, d.cpu().numpy()


def test_reverse_pivot_order_is_eq_d(bi):
    """Blocks last to first (Eq. (d) at every step) reach the same inverse."""
    A = inputs.gaussian_shifted(700, 72, sigma=1.5)
    sizes = [256, 256, 188]
    st, info, X = ex(bi, A, sizes, pivot_order=1)
    assert st == bi.OK and info.partition_fallback == 0 and info.blocks_used == 3
    Xo = oracle.block_inverse(A, sizes)
    kappa = np.linalg.norm(A) * np.linalg.norm(Xo)
    assert rho(A, X) <= 1e-12
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 4 * 700 * kappa * 2.0 ** -53


def test_singular_leading_block_falls_back_to_eq_d(bi):
    """A11 = 0 (Eq. (a) cannot start) but D and S_D = -B D^-1 C are invertible."""
    g = inputs.rng(73)
    b, m = 100, 200
    A = np.zeros((b + m, b + m))
    A[:b, b:] = g.standard_normal((b, m))
    A[b:, :b] = g.standard_normal((m, b))
    A[b:, b:] = g.uniform(-1, 1, (m, m)) + m * np.eye(m)
    sizes = [b, m]
    st, info, _ = ex(bi, A, sizes)
    assert st == bi.ERR_SINGULAR and info.failing_block == 0
    st, info, X = ex(bi, A, sizes, singular_fallback=1)
    assert st == bi.OK and info.partition_fallback == 1 and info.blocks_used == 2
    assert rho(A, X) <= 1e-12
    Xo = oracle.block_inverse(A, [b + m])   # one block: Gauss-Jordan with partial pivoting
    kappa = np.linalg.norm(A) * np.linalg.norm(Xo)
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 4 * (b + m) * kappa * 2.0 ** -53


@pytest.mark.parametrize("sizes", [[64, 64], [40, 40, 40, 40]])
def test_block_permutation_needs_merged_blocks(bi, sizes):
    """Every principal block of a block-reversal permutation is singular in both
    orders; merged blocks with partial pivoting inside invert it exactly."""
    n = sum(sizes)
    A = np.fliplr(np.eye(n)).copy()
    st, info, X = ex(bi, A, sizes, singular_fallback=1)
    assert st == bi.OK and info.partition_fallback == 2 and info.blocks_used < len(sizes)
    assert np.array_equal(X, A.T)


def test_singular_matrix_still_reported(bi):
    A = np.ones((300, 300))
    st, info, _ = ex(bi, A, [100, 100, 100], singular_fallback=1)
    assert st == bi.ERR_SINGULAR and info.partition_fallback == 2 and info.failing_block >= 0
