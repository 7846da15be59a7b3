"""GPU FP64 path vs the CPU oracle, through the C ABI.

Tolerances. The gate for every result is the normwise residual
rho = ||A X - I||_F / (||A||_F ||X||_F) <= 1e-12. The error against the oracle,
normwise eps = ||X - X_oracle||_F / ||X_oracle||_F and elementwise
max |X - X_oracle| / max |X_oracle|, is bounded by 16 sqrt(n) kappa_2(A) u
(u = 2^-53; see tests/tolerance.py): both sides are eliminations with partial
pivoting of the same matrix in different association orders.
Exact-arithmetic inputs (the unimodular pin) must match bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2305_11103_gb300 import inputs
from tolerance import eps_max, eps_norm, fwd_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
RHO_GATE = 1e-12


@pytest.fixture(scope="module")
def bi(cuda_device):
    from paper_2305_11103_gb300 import build as libbuild
    libbuild.build()
    from paper_2305_11103_gb300 import blockinv
    blockinv.lib()
    return blockinv


def gpu_invert(bi, A, sizes, mode="f64", lda=None):
    n = A.shape[0]
    if lda is None or lda == n:
        d = torch.from_numpy(A).cuda()
        bi.invert_(d, sizes, mode)
        return d.cpu().numpy()
    pad = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    pad[:, :n] = torch.from_numpy(A)
    st = bi.blockinv_invert(n, sizes, pad.data_ptr(), lda, mode, None)
    assert st == bi.OK, bi.blockinv_status_str(st)
    assert torch.all(pad[:, n:] == 0), "padding columns were written"
    return pad[:, :n].cpu().numpy()


def rho(A, X):
    return np.linalg.norm(A @ X - np.eye(A.shape[0])) / (np.linalg.norm(A) * np.linalg.norm(X))


def check(A, X, Xo):
    r, e, em = rho(A, X), eps_norm(X, Xo), eps_max(X, Xo)
    bound = fwd_bound(A, Xo)
    assert r <= RHO_GATE, f"rho {r:.3e}"
    assert e <= bound, f"eps {e:.3e} > {bound:.3e}"
    assert em <= bound, f"elementwise eps {em:.3e} > {bound:.3e}"
    return r, e


def test_small_config_256(bi):
    """256 x 256, 4 x 4 grid of 64 x 64 blocks, U[-1,1] + 256 I, seed 1."""
    A = inputs.diag_dominant_uniform(256, 1, shift=256)
    sizes = [64] * 4
    X = gpu_invert(bi, A, sizes)
    Xo = oracle.block_inverse(A, sizes)
    check(A, X, Xo)


@pytest.mark.parametrize("sizes", [[1], [2], [3], [17], [64], [65], [128], [200], [256], [300], [512]])
def test_single_block_is_the_pivot_kernel(bi, sizes):
    """p = 1: only the pivot-block Gauss-Jordan kernel runs (cluster sizes 1..16)."""
    n = sizes[0]
    A = inputs.gaussian_shifted(n, 10 + n, sigma=1.5)
    X = gpu_invert(bi, A, sizes)
    check(A, X, oracle.block_inverse(A, sizes))


@pytest.mark.parametrize("sizes", [
    [2, 3], [3, 4], [1, 1, 1, 1, 1], [5, 7, 1, 3, 8, 9],
    [64, 64, 1], [33, 65, 7], [100, 157], [65] * 5, [128, 3, 128, 60],
    [256, 256, 256, 57],
])
def test_ragged_partitions(bi, sizes):
    n = sum(sizes)
    A = inputs.diag_dominant_uniform(n, 7 * n, shift=n)
    X = gpu_invert(bi, A, sizes)
    check(A, X, oracle.block_inverse(A, sizes))


def test_gaussian_config_small(bi):
    """N(0,1)/sqrt(n) + 1.5 I at n = 1024, 4 blocks of 256 (the 8192 workload's block shape)."""
    A = inputs.gaussian_shifted(1024, 2, sigma=1.5)
    X = gpu_invert(bi, A, [256] * 4)
    check(A, X, oracle.block_inverse(A, [256] * 4))


@pytest.mark.parametrize("sizes", [[2, 3], [4, 4, 4, 4], [1, 2, 3, 4, 5, 6, 7], [8, 8, 8, 8]])
def test_unimodular_bitwise(bi, sizes):
    A, _, _ = inputs.unimodular_block_lu(sizes, 99)
    X = gpu_invert(bi, A, sizes)
    Xo = oracle.block_inverse(A, sizes)
    assert np.array_equal(X, Xo)


def test_padded_leading_dimension(bi):
    A = inputs.diag_dominant_uniform(150, 3, shift=150)
    sizes = [50, 60, 40]
    X = gpu_invert(bi, A, sizes, lda=203)
    check(A, X, oracle.block_inverse(A, sizes))


def test_default_partition(bi):
    for n in (5, 9, 16, 300, 700):
        A = inputs.diag_dominant_uniform(n, n, shift=n)
        X = gpu_invert(bi, A, None)
        assert rho(A, X) <= RHO_GATE


def test_deterministic(bi):
    A = inputs.gaussian_shifted(700, 5)
    X1 = gpu_invert(bi, A, [256, 256, 188])
    X2 = gpu_invert(bi, A, [256, 256, 188])
    assert np.array_equal(X1, X2)


def test_singular_block_reported(bi):
    J = np.fliplr(np.eye(6)).copy()
    d = torch.from_numpy(J).cuda()
    st = bi.blockinv_invert(6, [3, 3], d.data_ptr(), 6, 0, None)
    assert st == bi.ERR_SINGULAR
    assert bi.blockinv_last_error_detail() == (bi.ERR_SINGULAR, 0)
    A = np.eye(6)
    A[4, 5] = A[5, 4] = 1.0
    d = torch.from_numpy(A).cuda()
    assert bi.blockinv_invert(6, [2, 2, 2], d.data_ptr(), 6, 0, None) == bi.ERR_SINGULAR
    assert bi.blockinv_last_error_detail()[1] == 2


def test_nonfinite_reported(bi):
    A = inputs.diag_dominant_uniform(100, 4)
    A[70, 71] = np.nan
    d = torch.from_numpy(A).cuda()
    st = bi.blockinv_invert(100, [50, 50], d.data_ptr(), 100, 0, None)
    assert st in (bi.ERR_NONFINITE, bi.ERR_SINGULAR)


def test_argument_error_leaves_matrix_untouched(bi):
    A = inputs.diag_dominant_uniform(32, 8)
    d = torch.from_numpy(A).cuda()
    assert bi.blockinv_invert(32, [16, 15], d.data_ptr(), 32, 0, None) == bi.ERR_INVALID
    assert np.array_equal(d.cpu().numpy(), A)


def test_host_buffer_entry_point(bi):
    A = inputs.gaussian_shifted(600, 12)
    h = torch.from_numpy(A.copy()).pin_memory()
    bi.invert_host_(h, [200, 200, 200])
    check(A, h.numpy(), oracle.block_inverse(A, [200, 200, 200]))


def test_host_buffer_padded_rows(bi):
    """Host rows with a leading dimension above n (the pitched copies), and
    the padding columns left alone."""
    n, ld = 520, 531
    A = inputs.gaussian_shifted(n, 14)
    big = torch.full((n, ld), 7.25, dtype=torch.float64).pin_memory()
    big[:, :n] = torch.from_numpy(A)
    st = bi.blockinv_invert_host(n, [130] * 4, big.data_ptr(), ld, "f64")
    assert st == bi.OK
    X = big[:, :n].numpy()
    check(A, X, oracle.block_inverse(A, [130] * 4))
    assert torch.all(big[:, n:] == 7.25)


def test_async_entry_point_status(bi):
    A = inputs.diag_dominant_uniform(96, 9)
    d = torch.from_numpy(A).cuda()
    status = torch.full((2,), 77, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    st = bi.blockinv_invert_async(96, [32, 64], d.data_ptr(), 96, 0, s, status.data_ptr())
    assert st == bi.OK
    s.synchronize()
    assert status.tolist() == [0, 0]
    check(A, d.cpu().numpy(), oracle.block_inverse(A, [32, 64]))
    J = torch.from_numpy(np.fliplr(np.eye(4)).copy()).cuda()
    assert bi.blockinv_invert_async(4, [2, 2], J.data_ptr(), 4, 0, s, status.data_ptr()) == bi.OK
    s.synchronize()
    assert status.tolist() == [bi.ERR_SINGULAR, 0]


def test_gpu_residual_matches_numpy(bi):
    A = inputs.gaussian_shifted(333, 13)
    X = np.linalg.inv(A) * (1 + 1e-9)
    dA = torch.from_numpy(A).cuda()
    dX = torch.from_numpy(X).cuda()
    r = bi.residual(dA, dX)
    assert abs(r - rho(A, X)) <= 1e-3 * rho(A, X)


# Look-ahead (n >= 2048 with 3 or more blocks): the next pivot inverse and row
# panel run on a side stream while the rest of the current update runs. Each
# element still sees the same operations in the same order, so the result must
# equal, bit for bit, that of the plain step sequence, which the no-alloc entry
# point runs (n <= 2048, blocks <= 256).
@pytest.mark.parametrize("sizes", [[256] * 8, [200] * 10 + [48], [256] * 7 + [100, 92, 64], [1, 255] * 4 + [256] * 4])
def test_look_ahead_matches_plain_sequence_bitwise(bi, sizes):
    n = sum(sizes)
    assert n == 2048
    A = inputs.gaussian_shifted(n, 31, sigma=1.5)
    ref = torch.from_numpy(A).cuda()
    st, fb = bi.blockinv_invert_noalloc(n, sizes, ref.data_ptr(), n, None)
    assert st == bi.OK
    X = gpu_invert(bi, A, sizes)
    assert np.array_equal(X, ref.cpu().numpy())


@pytest.mark.parametrize("sizes", [[256] * 9, [300, 200, 500, 512, 512, 176]])
def test_look_ahead_option_off_same_bits(bi, sizes):
    """lookahead = -1 runs one step at a time on the caller's stream only."""
    n = sum(sizes)
    A = inputs.gaussian_shifted(n, 33, sigma=1.5)
    outs = []
    for la in (0, -1):
        d = torch.from_numpy(A).cuda()
        st, info = bi.blockinv_invert_ex(n, sizes, d.data_ptr(), n, "f64", None, lookahead=la)
        assert st == bi.OK
        outs.append(d.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert rho(A, outs[0]) <= 1e-12


@pytest.mark.parametrize("sizes", [[256] * 8 + [57], [300, 200, 500, 512, 512, 176], [100] * 21])
def test_look_ahead_ragged_vs_oracle(bi, sizes):
    n = sum(sizes)
    A = inputs.diag_dominant_uniform(n, 41, shift=n)
    X = gpu_invert(bi, A, sizes)
    check(A, X, oracle.block_inverse(A, sizes))
    assert np.array_equal(X, gpu_invert(bi, A, sizes))


@pytest.mark.slow
def test_full_size_8192(bi):
    """n = 8192, 32 x 32 grid of 256-blocks, N(0,1)/sqrt(n) + 1.5 I, seed 2 (the
    8192 benchmark workload, same launch sequence): rho on the GPU (FP64), and
    normwise and elementwise error against the oracle's inverse of the same
    matrix (about 20 s on 16 host cores)."""
    n = 8192
    A = inputs.gaussian_shifted(n, 2, sigma=1.5)
    dA = torch.from_numpy(A).cuda()
    dX = dA.clone()
    bi.invert_(dX, [256] * 32)
    assert bi.residual(dA, dX) <= RHO_GATE
    X = dX.cpu().numpy()
    Xo = oracle.block_inverse(A, [256] * 32)
    check(A, X, Xo)


def test_release_memory_then_invert_again(bi):
    A = inputs.diag_dominant_uniform(600, 77, shift=600)
    X1 = gpu_invert(bi, A, [256, 256, 88])
    assert bi.lib().blockinv_release_memory() == bi.OK
    X2 = gpu_invert(bi, A, [256, 256, 88])
    assert np.array_equal(X1, X2)
