"""The tcgen05 tensor-core GEMM (through blockinv_diag_gemm, on single-CTA
128 x 256 tiles and on CTA pairs with 256 x 256 tiles) and the unrefined
mixed-precision elimination, through the C ABI.

Tolerances: integer-valued operands whose products and sums stay below 2^24
must come out exact (FP32 accumulation of exact products), which is the
property the split-operand FP64-accurate residual relies on. Non-integer
operands are compared with an FP64 product of the same rounded operands at
K * 2^-23 relative to |A| |B|. The unrefined TF32 / BF16 elimination is
compared with the oracle at the precision of its operands.
"""
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


def run_gemm(bi, kind, A, B):
    M, K = A.shape
    N = B.shape[0]
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = bi.blockinv_diag_gemm(kind, M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                               C.data_ptr(), C.stride(0), None)
    assert st == bi.OK, bi.blockinv_status_str(st)
    return C


def padded(t, mult):
    M, K = t.shape
    Kp = (K + mult - 1) // mult * mult
    out = torch.zeros((M, Kp), dtype=t.dtype, device=t.device)
    out[:, :K] = t
    return out[:, :K]


PAIR = pytest.mark.parametrize("pair", [0, 3], ids=["cta", "pair"])  # kind offset of the CTA-pair GEMM


@PAIR
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 520, 200), (2125, 1100, 512), (77, 3000, 1024)])
def test_e4m3_integer_exact(bi, M, N, K, pair):
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    Ai = torch.randint(-15, 16, (M, K), generator=g)
    Bi = torch.randint(-8, 9, (N, K), generator=g)
    A = padded(Ai.to(torch.float32).to(torch.float8_e4m3fn).cuda(), 16)
    B = padded(Bi.to(torch.float32).to(torch.float8_e4m3fn).cuda(), 16)
    C = run_gemm(bi, 2 + pair, A, B).cpu().double()
    ref = Ai.double() @ Bi.double().T
    assert torch.equal(C, ref)


@PAIR
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 520, 200), (1500, 700, 320)])
def test_bf16_integer_exact(bi, M, N, K, pair):
    g = torch.Generator(device="cpu").manual_seed(7 + M)
    Ai = torch.randint(-100, 101, (M, K), generator=g)
    Bi = torch.randint(-100, 101, (N, K), generator=g)
    A = padded(Ai.to(torch.bfloat16).cuda(), 8)
    B = padded(Bi.to(torch.bfloat16).cuda(), 8)
    C = run_gemm(bi, 0 + pair, A, B).cpu().double()
    assert torch.equal(C, Ai.double() @ Bi.double().T)


@PAIR
@pytest.mark.parametrize("M,N,K", [(256, 256, 96), (1000, 1300, 260)])
def test_tf32_matches_fp64_of_rounded_operands(bi, M, N, K, pair):
    g = torch.Generator(device="cpu").manual_seed(11 + M)
    A = torch.randn(M, K, generator=g)
    B = torch.randn(N, K, generator=g)
    # round to TF32 (10 explicit mantissa bits) so that the hardware's operand
    # conversion is exact
    def tf32(x):
        u = x.view(torch.int32)
        u = (u + 0x1000) & ~0x1FFF
        return u.view(torch.float32)
    A, B = tf32(A), tf32(B)
    C = run_gemm(bi, 1 + pair, padded(A.cuda(), 4), padded(B.cuda(), 4)).cpu().double()
    ref = A.double() @ B.double().T
    scale = A.abs().double() @ B.abs().double().T
    assert torch.all((C - ref).abs() <= K * 2.0 ** -23 * scale + 1e-30)


@PAIR
def test_tf32_integer_exact(bi, pair):
    g = torch.Generator(device="cpu").manual_seed(5)
    Ai = torch.randint(-300, 301, (640, 128), generator=g).float()
    Bi = torch.randint(-300, 301, (384, 128), generator=g).float()
    C = run_gemm(bi, 1 + pair, Ai.cuda(), Bi.cuda()).cpu().double()
    assert torch.equal(C, Ai.double() @ Bi.double().T)


# ------------------------------------------------------ mixed elimination ---
def mixed_unrefined(bi, A, sizes, mode):
    d = torch.from_numpy(A).cuda()
    st, info = bi.blockinv_invert_ex(A.shape[0], sizes, d.data_ptr(), A.shape[0], mode, None, max_refine=0)
    assert st == bi.OK, bi.blockinv_status_str(st)
    return d.cpu().numpy()


@pytest.mark.parametrize("mode,tol", [("tf32", 2e-3), ("bf16", 3e-2)])
@pytest.mark.parametrize("sizes", [[256] * 4, [100, 157, 63], [64] * 5 + [37], [512, 300], [129], [256], [300, 33],
                                   [512], [65, 97]])
def test_mixed_elimination_vs_oracle(bi, mode, tol, sizes):
    n = sum(sizes)
    A = inputs.gaussian_shifted(n, 3 + n, sigma=1.5)
    X = mixed_unrefined(bi, A, sizes, mode)
    Xo = oracle.block_inverse(A, sizes)
    eps = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    assert eps <= tol, eps


def test_mixed_tf32_unimodular_exact(bi):
    """Small-integer inputs whose inverse stays below 2^11: every product and
    sum is exact in TF32 / FP32, so the mixed elimination is exact too."""
    sizes = [4, 4, 4, 4]
    A, _, _ = inputs.unimodular_block_lu(sizes, 5, lower_density=0.3)
    Xo = oracle.block_inverse(A, sizes)
    assert np.abs(Xo).max() < 2 ** 10
    X = mixed_unrefined(bi, A, sizes, "tf32")
    assert np.array_equal(X, Xo)


# ---------------------------------------------- accumulator exactness ------
# The split-operand residual adds many exact integer products per output in
# the FP32 accumulator and needs every partial sum below 2^24 to stay exact.
# Rows carry large equal products plus one small odd term at a row-dependent
# position, with alternating signs, so that any truncation of low bits during
# accumulation changes the result.
@pytest.mark.parametrize("kind,big_a,big_b,K", [
    (2, 16.0, 8.0, 4096),     # E4M3: products 2^7, sums near 2^19
    (2, 16.0, 8.0, 16384),    # sums near 2^21
    (2, 16.0, 16.0, 16384),   # sums near 2^22
    (0, 128.0, 64.0, 1024),   # BF16: products 2^13, sums near 2^23
    (1, 1024.0, 512.0, 32),   # TF32: products 2^19, sums near 2^24
])
@PAIR
def test_accumulator_exact_near_2_24(bi, kind, big_a, big_b, K, pair):
    M, N = 128, 256
    A = np.full((M, K), big_a)
    B = np.full((N, K), big_b)
    A[np.arange(M), (np.arange(M) * 37) % K] = 1.0
    B[np.arange(N), (np.arange(N) * 101 + 5) % K] = 1.0
    A[1::2] *= -1.0
    B[:, 1::3] *= -1.0
    expect = A.astype(np.int64) @ B.astype(np.int64).T
    assert np.abs(expect).max() < 2 ** 24
    dt = {2: torch.float8_e4m3fn, 0: torch.bfloat16, 1: torch.float32}[kind]
    tA = torch.from_numpy(A).float().to(dt).cuda()
    tB = torch.from_numpy(B).float().to(dt).cuda()
    C = run_gemm(bi, kind + pair, tA, tB).cpu().numpy().astype(np.int64)
    bad = np.count_nonzero(C != expect)
    assert bad == 0, f"{bad} inexact outputs; max error {np.abs(C - expect).max()}"


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_split_operands_tighten_unrefined_inverse(bi, mode):
    """hi + lo operand splitting (three products) must give a clearly smaller
    residual than one product before any refinement."""
    n = 1024
    A = inputs.gaussian_shifted(n, 81, sigma=1.5)
    rhos = []
    for split in (1, 2):
        d = torch.from_numpy(A).cuda()
        st, info = bi.blockinv_invert_ex(n, [256] * 4, d.data_ptr(), n, mode, None, max_refine=0, split=split)
        assert st == bi.OK
        X = d.cpu().numpy()
        rhos.append(np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X)))
    assert rhos[1] < 0.1 * rhos[0], rhos
