"""Mixed-precision path with Newton-Schulz refinement, through the C ABI.

The FP64-accurate tensor-core residual is checked entry by entry against
exact rational arithmetic (Python fractions) on sampled entries: the error
must stay below 2^-40 of sum_k |a_ik| |x_kj| (44 bits are kept relative to
the row and column scales; 4 bits of margin). Refined inverses must meet the
same gate as the FP64 path, rho <= 1e-12, and the forward-error bound against
the oracle.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
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


def rho_np(A, X):
    return np.linalg.norm(A @ X - np.eye(A.shape[0])) / (np.linalg.norm(A) * np.linalg.norm(X))


def exact_residual_entries(A, X, idx):
    out = []
    for i, j in idx:
        exact = (1 if i == j else 0) - sum(Fraction(float(a)) * Fraction(float(x)) for a, x in zip(A[i], X[:, j]))
        out.append(float(exact))
    return np.array(out)


def tc_residual(bi, A, X, slices=0):
    n = A.shape[0]
    dA, dX = torch.from_numpy(A).cuda(), torch.from_numpy(X).cuda()
    E = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st, rho = bi.blockinv_residual_tc(n, dA.data_ptr(), n, dX.data_ptr(), n, E.data_ptr(), n, slices)
    assert st == bi.OK
    return E.cpu().numpy(), rho


@pytest.mark.parametrize("n,kind", [(300, "gauss"), (1000, "gauss"), (500, "dd"), (400, "general")])
def test_tc_residual_exact_on_samples(bi, n, kind):
    if kind == "gauss":
        A = inputs.gaussian_shifted(n, 40 + n, sigma=1.5)
    elif kind == "dd":
        A = inputs.diag_dominant_uniform(n, 40 + n, shift=n)
    else:  # no dominant diagonal: N(0, 1) entries
        A = inputs.rng(40 + n).standard_normal((n, n))
    g = inputs.rng(41 + n)
    X = np.linalg.inv(A) * (1 + 1e-7 * g.standard_normal((n, n)))
    idx = [(int(i), int(j)) for i, j in zip(g.integers(0, n, 40), g.integers(0, n, 40))] + [(k, k) for k in range(5)]
    exact = exact_residual_entries(A, X, idx)
    scale = np.array([np.abs(A[i]) @ np.abs(X[:, j]) for i, j in idx])
    errs = []
    for S in (7, 8, 9):
        E, rho = tc_residual(bi, A, X, S)
        got = np.array([E[i, j] for i, j in idx])
        errs.append(np.max(np.abs(got - exact) / scale))
    # the default (9 base-32 digits, 44 bits) keeps 2^-42 of |A| |X| on every
    # sampled entry
    assert errs[2] <= 2.0 ** -42, errs
    # each digit adds 5 bits until the FP64 floor: the error falls by >= 8x
    assert errs[1] <= errs[0] / 8 + 1e-17 and errs[2] <= errs[1] / 8 + 1e-17, errs
    E, rho = tc_residual(bi, A, X)
    dA, dX = torch.from_numpy(A).cuda(), torch.from_numpy(X).cuda()
    st, rho64 = bi.blockinv_residual(n, dA.data_ptr(), n, dX.data_ptr(), n)
    assert abs(rho - rho64) <= 1e-3 * rho64


def refine(bi, A, sizes, mode, **kw):
    n = A.shape[0]
    d = torch.from_numpy(A).cuda()
    st, info = bi.blockinv_invert_ex(n, sizes, d.data_ptr(), n, mode, None, **kw)
    return st, info, d.cpu().numpy()


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("n,sizes,kind", [
    (256, [64] * 4, "dd"),
    (1024, [256] * 4, "gauss"),
    (777, [256, 256, 265], "gauss"),
    (1500, [200] * 7 + [100], "dd"),
])
def test_refined_mixed_meets_gate(bi, mode, n, sizes, kind):
    A = inputs.diag_dominant_uniform(n, n, shift=n) if kind == "dd" else inputs.gaussian_shifted(n, 2 + n, sigma=1.5)
    st, info, X = refine(bi, A, sizes, mode)
    assert st == bi.OK, (bi.blockinv_status_str(st), info.as_dict())
    assert info.used_fallback == 0
    assert 0 <= info.rho <= 1e-12 and info.rho_initial > info.rho
    r = rho_np(A, X)
    assert r <= 1e-12
    Xo = oracle.block_inverse(A, sizes)
    kappa = np.linalg.norm(A) * np.linalg.norm(Xo)
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 4 * n * kappa * U64
    # the GPU's own rho agrees with the one measured here, down to the
    # rounding floor of evaluating A X - I in FP64 (about sqrt(n) u)
    assert abs(info.rho - r) <= 0.05 * r + 20 * np.sqrt(n) * U64


def test_poorly_conditioned_sigma_105(bi):
    """N(0,1)/sqrt(n) + 1.05 I: the smallest singular values approach 0.05."""
    n = 1024
    A = inputs.gaussian_shifted(n, 4, sigma=1.05)
    st, info, X = refine(bi, A, [256] * 4, "tf32")
    assert st == bi.OK
    assert rho_np(A, X) <= 1e-12


def test_ill_conditioned_spd_converges_without_fallback(bi):
    """B B^T + 0.1 I (kappa ~ 4e4 at n = 1024): the update maps E to E^2, so
    from ||E||_F < 1 it converges, over several updates, without the FP64 rerun."""
    n = 1024
    A = inputs.spd_covariance(n, 1924)
    st, info, X = refine(bi, A, [256] * 4, "tf32", fallback=0)
    assert st == bi.OK and info.used_fallback == 0 and info.refine_iters >= 2
    assert rho_np(A, X) <= 1e-12


def test_stall_at_the_rounding_floor_stops(bi):
    """A target below the rounding floor: the residual stops falling, and the
    refinement ends with NOT_CONVERGED before the iteration cap."""
    n = 512
    A = inputs.gaussian_shifted(n, 19, sigma=1.5)
    st, info, _ = refine(bi, A, [128] * 4, "tf32", tol=1e-30, max_refine=8, fallback=0)
    assert st == bi.ERR_NOT_CONVERGED and info.used_fallback == 0
    assert 1 <= info.refine_iters < 8


def test_not_converged_then_fallback(bi):
    n = 512
    A = inputs.gaussian_shifted(n, 9, sigma=1.5)
    # one update cannot reach 1e-30: NOT_CONVERGED without fallback ...
    st, info, _ = refine(bi, A, [128] * 4, "bf16", tol=1e-30, max_refine=1, fallback=0)
    assert st == bi.ERR_NOT_CONVERGED and info.used_fallback == 0
    # ... and the FP64 path's result with it
    st, info, X = refine(bi, A, [128] * 4, "bf16", tol=1e-30, max_refine=1, fallback=1)
    assert st == bi.OK and info.used_fallback == 1
    assert rho_np(A, X) <= 1e-12


def test_mixed_async_status(bi):
    n = 384
    A = inputs.diag_dominant_uniform(n, 3)
    d = torch.from_numpy(A).cuda()
    status = torch.full((2,), 5, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    assert bi.blockinv_invert_async(n, [128] * 3, d.data_ptr(), n, "tf32", s, status.data_ptr()) == bi.OK
    s.synchronize()
    assert status.tolist()[0] == 0
    assert rho_np(A, d.cpu().numpy()) <= 1e-12


def test_mixed_singular_reported(bi):
    J = np.fliplr(np.eye(8)).copy()
    st, info, _ = refine(bi, J, [4, 4], "tf32")
    assert st == bi.ERR_SINGULAR and info.failing_block == 0


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("sigma,seed", [(1.5, 3), (1.05, 4)])
def test_full_size_16384_mixed(bi, mode, sigma, seed):
    """n = 16384, 64 x 64 grid of 256-blocks, N(0,1)/sqrt(n) + sigma I: the
    mixed path with refinement to rho <= 1e-12. The oracle cannot invert it in
    test time: the GPU's own FP64-accurate residual, sampled rows of A X - I in
    FP64 on the CPU, and sampled columns against LAPACK solves."""
    n = 16384
    A = inputs.gaussian_shifted(n, seed, sigma=sigma)
    dA = torch.from_numpy(A).cuda()
    dX = dA.clone()
    st, info = bi.blockinv_invert_ex(n, [256] * 64, dX.data_ptr(), n, mode, None)
    assert st == bi.OK and info.used_fallback == 0, info.as_dict()
    assert info.rho <= 1e-12
    st, rho_tc = bi.blockinv_residual_tc(n, dA.data_ptr(), n, dX.data_ptr(), n)
    assert st == bi.OK and rho_tc <= 1e-12
    X = dX.cpu().numpy()
    g = inputs.rng(seed + 99)
    nA, nX = np.linalg.norm(A), np.linalg.norm(X)
    for i in g.choice(n, size=8, replace=False):
        e = A[i] @ X
        e[i] -= 1.0
        assert np.linalg.norm(e) * np.sqrt(n) / (nA * nX) <= 1e-12
    cols = g.choice(n, size=2, replace=False)
    E = np.zeros((n, 2))
    E[cols, range(2)] = 1.0
    S = np.linalg.solve(A, E)
    kappa = nA * nX
    for t, j in enumerate(cols):
        assert np.linalg.norm(X[:, j] - S[:, t]) / np.linalg.norm(S[:, t]) <= 4 * n * kappa * U64


# The mixed look-ahead splits step k's Schur update into the next pivot block's
# square (its covering tiles) and the rest, and runs the next FP32 pivot inverse
# beside the rest. Every element is the same tile sum either way, so with one
# step per sweep (the default, fuse = 0) the unrefined elimination must match the
# one-step-at-a-time sequence bit for bit, also where block edges cut through
# tiles (ragged sizes) and in reverse order.
@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("sizes,order,pf", [([256] * 12, 0, 0), ([200, 312, 256, 300, 212, 200, 300, 316, 300], 0, 0),
                                            ([256] * 12, 1, 0), ([500, 24, 512, 100, 412, 500], 0, 0),
                                            ([256] * 12, 0, -1), ([256] * 12, 0, 1)])
def test_mixed_look_ahead_same_bits(bi, mode, sizes, order, pf):
    # pf: pivot_f64 (0 condition-gated FP64 re-inversion, -1 none: the update
    # then depends on the pivot kernel directly, 1 every block)
    n = sum(sizes)
    assert n >= 2048
    A = inputs.gaussian_shifted(n, 7 + n, sigma=1.5)
    outs = []
    for la in (0, -1):
        d = torch.from_numpy(A).cuda()
        st, info = bi.blockinv_invert_ex(n, sizes, d.data_ptr(), n, mode, None, max_refine=0, pivot_order=order,
                                         lookahead=la, pivot_f64=pf)
        assert st == bi.OK
        outs.append(d.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert rho_np(A, outs[0]) < 1e-5


# Two elimination steps per sweep (option fuse = 1): step k updates block row and
# column k + 1 alone, then one rank-2b sweep applies both steps to the rest.
# The products are summed in one FP32 accumulator instead of being rounded to
# FP32 in between, so the unrefined result differs from one step per sweep by
# rounding only: its residual must be as small, and the refined result must
# meet the gate. Sizes cover an odd block count, two blocks only, ragged
# blocks cut through tiles, the reverse order, n below the look-ahead's 2048
# and the sizes of the 8192 workload.
@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("sizes,order", [([256] * 12, 0), ([256] * 11, 0), ([300, 212], 0),
                                         ([200, 312, 256, 300, 212, 200, 300, 316, 300], 0),
                                         ([500, 24, 512, 100, 412, 500], 1), ([100, 60, 140, 37], 0),
                                         ([256] * 9, 1)])
def test_fused_two_step_sweep_matches_one_step(bi, mode, sizes, order):
    n = sum(sizes)
    A = inputs.gaussian_shifted(n, 11 + n, sigma=1.5)
    outs = []
    for fuse in (1, 0):
        d = torch.from_numpy(A).cuda()
        st, info = bi.blockinv_invert_ex(n, sizes, d.data_ptr(), n, mode, None, max_refine=0, pivot_order=order,
                                         fuse=fuse)
        assert st == bi.OK
        outs.append(d.cpu().numpy())
    r_fused, r_one = rho_np(A, outs[0]), rho_np(A, outs[1])
    assert r_fused <= 4 * r_one + 1e-9, (r_fused, r_one)
    # the two unrefined inverses agree to FP32-level rounding of the elimination
    assert np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[1]) <= 1e-4
    d = torch.from_numpy(A).cuda()
    st, info = bi.blockinv_invert_ex(n, sizes, d.data_ptr(), n, mode, None, tol=1e-12, pivot_order=order, fuse=1)
    assert st == bi.OK and info.used_fallback == 0
    X = d.cpu().numpy()
    assert rho_np(A, X) <= 1e-12
    Xo = oracle.block_inverse(A, sizes)
    kappa = np.linalg.norm(A) * np.linalg.norm(Xo)
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-12 * kappa


def _ill_block(n, kappa, seed):
    """Q diag(logspace(0, -log10 kappa)) Q^T, rounded to FP32 values (so the
    mixed path's FP32 copy is exact)."""
    g = inputs.rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    d = np.logspace(0, -np.log10(kappa), n)
    return ((Q * d) @ Q.T).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_ill_conditioned_pivot_block_inverted_in_fp64(bi, mode):
    """A single 256-block with kappa ~ 1e6: the FP32 Gauss-Jordan leaves an error
    near kappa * 2^-24; FP64 arithmetic (chosen by the condition estimate, or
    forced) leaves only the FP32 rounding of the result."""
    n = 256
    A = _ill_block(n, 1e6, 91)
    Ainv = np.linalg.inv(A)
    got = {}
    for pf in (-1, 0, 1):
        d = torch.from_numpy(A).cuda()
        st, info = bi.blockinv_invert_ex(n, [n], d.data_ptr(), n, mode, None, max_refine=0, pivot_f64=pf)
        assert st == bi.OK
        got[pf] = (np.linalg.norm(d.cpu().numpy() - Ainv) / np.linalg.norm(Ainv), info.fp64_pivots)
    assert [got[pf][1] for pf in (-1, 0, 1)] == [0, 1, 1], got
    assert got[0][0] <= 1e-6 and got[1][0] <= 1e-6, got
    assert got[-1][0] >= 100 * got[0][0], got


def test_well_conditioned_pivots_stay_fp32(bi):
    n = 1024
    A = inputs.gaussian_shifted(n, 5, sigma=1.5)
    d = torch.from_numpy(A).cuda()
    st, info = bi.blockinv_invert_ex(n, [256] * 4, d.data_ptr(), n, "tf32", None)
    assert st == bi.OK and info.fp64_pivots == 0 and 0 <= info.rho <= 1e-12


def test_ill_conditioned_first_block_refines(bi):
    """An ill-conditioned leading 256-block inside a 768 matrix: the block is
    flagged and inverted in FP64; the solve still meets the gate."""
    n, b = 768, 256
    A = inputs.gaussian_shifted(n, 93, sigma=1.5)
    A[:b, :b] = _ill_block(b, 1e5 * 3, 94) * 4.0
    A[:b, b:] *= 1e-2
    A[b:, :b] *= 1e-2
    d = torch.from_numpy(A).cuda()
    st, info = bi.blockinv_invert_ex(n, [b] * 3, d.data_ptr(), n, "tf32", None)
    assert st == bi.OK and info.fp64_pivots >= 1
    X = d.cpu().numpy()
    r = np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X))
    assert r <= 1e-12, (r, info.as_dict())


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("sigma", [1.5, 1e3])
def test_incremental_residual_matches_fresh(bi, mode, sigma):
    """After the first update the residual is formed as E - A (X_new - X_old)
    from the leading digit groups of the change (fewer than 9 here: the change
    is far below X); it must agree with a fresh 9-digit residual of the same
    result and with FP64 numpy."""
    n = 2048
    A = inputs.gaussian_shifted(n, 95, sigma=sigma)
    st, info, X = refine(bi, A, [256] * 8, mode)
    assert st == bi.OK and info.incremental_residuals >= 1 and info.used_fallback == 0
    assert 1 <= info.incremental_groups < 9, info.as_dict()
    _, rho_fresh = tc_residual(bi, A, X)
    r = np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X))
    assert r <= 1e-12
    assert abs(info.rho - rho_fresh) <= 2e-14 + 0.05 * rho_fresh, (info.rho, rho_fresh, r)
    assert abs(info.rho - r) <= 2e-14 + 0.05 * r, (info.rho, r)
