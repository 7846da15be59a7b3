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
