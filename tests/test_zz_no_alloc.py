"""blockinv_invert_noalloc: the FP64 inversion for callers that cannot
allocate device memory (inside an allocator callback, or a plugin whose host
owns all memory). Its scratch is a fixed device array inside the library.

Checked through the C ABI against blockinv_invert on two calls in a row (the
second call reuses the scratch the first one left behind), with the same
tolerances as the FP64 parity tests. Kept in a file of its own that pytest
collects last.
"""
import numpy as np
import pytest

from paper_2305_11103_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def bi(cuda_device):
    from paper_2305_11103_gb300 import build as libbuild
    libbuild.build()
    from paper_2305_11103_gb300 import blockinv
    blockinv.lib()
    return blockinv


def rho(A, X):
    return np.linalg.norm(A @ X - np.eye(A.shape[0])) / (np.linalg.norm(A) * np.linalg.norm(X))


def test_noalloc_matches_invert_twice(bi):
    cases = [
        (inputs.gaussian_shifted(1000, 71, sigma=1.5), [256, 256, 256, 232]),
        (inputs.diag_dominant_uniform(2048, 72, shift=2048), [256] * 8),
    ]
    for A, sizes in cases:
        n = A.shape[0]
        ref = torch.from_numpy(A).cuda()
        assert bi.blockinv_invert(n, sizes, ref.data_ptr(), n, bi.F64, None) == bi.OK
        got = torch.from_numpy(A).cuda()
        st, fb = bi.blockinv_invert_noalloc(n, sizes, got.data_ptr(), n, None)
        assert st == bi.OK and fb == -1
        X, Xr = got.cpu().numpy(), ref.cpu().numpy()
        assert rho(A, X) <= 1e-12
        kappa = np.linalg.norm(A) * np.linalg.norm(Xr)
        assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) <= 4 * n * kappa * U64


def test_noalloc_limits_and_errors(bi):
    A = inputs.diag_dominant_uniform(64, 73)
    d = torch.from_numpy(A).cuda()
    # a single block is fine; an order above the scratch limit (n > 2048) is not
    assert bi.blockinv_invert_noalloc(64, [64], d.data_ptr(), 64, None)[0] == bi.OK
    big = torch.zeros((2049, 2049), dtype=torch.float64, device="cuda")
    assert bi.blockinv_invert_noalloc(2049, [256] * 8 + [1], big.data_ptr(), 2049, None)[0] == bi.ERR_INVALID
    # a block order above the scratch limit (257 > 256) with n <= 2048 is
    # rejected and leaves A untouched
    B = inputs.diag_dominant_uniform(512, 74)
    g = torch.from_numpy(B).cuda()
    assert bi.blockinv_invert_noalloc(512, [257, 255], g.data_ptr(), 512, None)[0] == bi.ERR_INVALID
    assert torch.equal(g.cpu(), torch.from_numpy(B))
    # a partition that does not sum to n
    e = torch.from_numpy(A).cuda()
    assert bi.blockinv_invert_noalloc(64, [32, 31], e.data_ptr(), 64, None)[0] == bi.ERR_INVALID
    assert torch.equal(e.cpu(), torch.from_numpy(A))
    # a singular pivot block is reported with its index, and the next call is clean again
    J = torch.from_numpy(np.fliplr(np.eye(8)).copy()).cuda()
    assert bi.blockinv_invert_noalloc(8, [4, 4], J.data_ptr(), 8, None) == (bi.ERR_SINGULAR, 0)
    f = torch.from_numpy(A).cuda()
    assert bi.blockinv_invert_noalloc(64, [16] * 4, f.data_ptr(), 64, None) == (bi.OK, -1)
    assert rho(A, f.cpu().numpy()) <= 1e-12
