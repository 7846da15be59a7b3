"""Serving context (continuous batching) through the C ABI: every result is
the same alone and in the mix (bit for bit in FP64 mode), admission respects
the HBM budget, host-buffer requests, cancellation and per-request failures."""
import time

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


def rho(A, X):
    return np.linalg.norm(A @ X - np.eye(A.shape[0])) / (np.linalg.norm(A) * np.linalg.norm(X))


def request_mix(seed, count, lo=5, hi=700):
    sizes = inputs.log_uniform_sizes(count, lo, hi, seed)
    g = inputs.rng(seed + 1)
    mats = []
    for i, n in enumerate(sizes):
        n = int(n)
        if g.random() < 0.3:
            mats.append(inputs.spd_covariance(n, seed + 100 + i) / n + 0.0 * np.eye(n))
        else:
            mats.append(inputs.diag_dominant_uniform(n, seed + 200 + i, shift=n))
    return mats


def test_alone_equals_mix_fp64(bi):
    mats = request_mix(700, 40)
    # alone: one request at a time on a one-slot context
    ctx1 = bi.Context(0, 4 << 30, 1)
    alone = []
    for A in mats:
        d = torch.from_numpy(A).cuda()
        st, t = ctx1.submit(A.shape[0], None, d.data_ptr(), A.shape[0])
        assert st == bi.OK
        st, r = ctx1.wait(t)
        assert st == bi.OK, bi.blockinv_status_str(st)
        alone.append(d.cpu().numpy())
    ctx1.close()
    # in the mix: everything submitted at once on an 8-slot context
    ctx = bi.Context(0, 4 << 30, 8)
    ds = [torch.from_numpy(A).cuda() for A in mats]
    tickets = []
    for A, d in zip(mats, ds):
        st, t = ctx.submit(A.shape[0], None, d.data_ptr(), A.shape[0])
        assert st == bi.OK
        tickets.append(t)
    overlap = 0
    for t in tickets:
        st, r = ctx.wait(t)
        assert st == bi.OK
        assert r.t_total_ms >= r.t_device_ms * 0.5 and r.t_queue_ms >= 0
    for A, d, a in zip(mats, ds, alone):
        X = d.cpu().numpy()
        assert np.array_equal(X, a)
        assert rho(A, X) <= 1e-12
    ctx.close()


def test_mix_vs_oracle_sample(bi):
    mats = request_mix(710, 20, 5, 300)
    ctx = bi.Context(0, 2 << 30, 4)
    ds = [torch.from_numpy(A).cuda() for A in mats]
    tickets = [ctx.submit(A.shape[0], None, d.data_ptr(), A.shape[0])[1] for A, d in zip(mats, ds)]
    for A, d, t in zip(mats, ds, tickets):
        assert ctx.wait(t)[0] == bi.OK
        n = A.shape[0]
        sizes = [n] if n <= 3 else (oracle.paper_partition(n) if n <= 16 else [256] * (n // 256) + ([n % 256] if n % 256 else []))
        Xo = oracle.block_inverse(A, sizes)
        X = d.cpu().numpy()
        kappa = np.linalg.norm(A) * np.linalg.norm(Xo)
        assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 4 * n * kappa * 2.0 ** -53
    ctx.close()


def test_mixed_mode_requests(bi):
    mats = [inputs.gaussian_shifted(n, 720 + n, sigma=1.5) for n in (300, 700, 1100)]
    ctx = bi.Context(0, 8 << 30, 3)
    ds = [torch.from_numpy(A).cuda() for A in mats]
    tickets = [ctx.submit(A.shape[0], None, d.data_ptr(), A.shape[0], "tf32")[1] for A, d in zip(mats, ds)]
    for A, d, t in zip(mats, ds, tickets):
        st, r = ctx.wait(t)
        assert st == bi.OK and 0 <= r.rho <= 1e-12 and r.refine_iters >= 1
        assert rho(A, d.cpu().numpy()) <= 1e-12
    ctx.close()


def test_mixed_fallback_for_ill_conditioned(bi):
    """B B^T + 0.1 I at n = 1500 (kappa ~ 1e5): BF16 refinement does not
    contract, so the request is rerun in FP64 and still meets the gate."""
    n = 1500
    A = inputs.spd_covariance(n, 760)
    ctx = bi.Context(0, 8 << 30, 2)
    d = torch.from_numpy(A).cuda()
    st, t = ctx.submit(n, None, d.data_ptr(), n, "bf16")
    st, r = ctx.wait(t)
    assert st == bi.OK
    assert rho(A, d.cpu().numpy()) <= 1e-12
    ctx.close()


def test_budget_admission(bi):
    n = 1024
    A = inputs.diag_dominant_uniform(n, 730)
    # the whole request footprint (workspace) must fit; 1 MiB does not
    ctx = bi.Context(0, 1 << 20, 2)
    d = torch.from_numpy(A).cuda()
    assert ctx.submit(n, None, d.data_ptr(), n)[0] == bi.ERR_BUDGET
    ctx.close()
    # a budget that holds one request at a time: all complete, never two at once
    ctx = bi.Context(0, 3 << 20, 4)
    ds = [torch.from_numpy(A).cuda() for _ in range(6)]
    tickets = [ctx.submit(n, None, d.data_ptr(), n)[1] for d in ds]
    max_running = 0
    while True:
        q, r, b = ctx.stats()
        max_running = max(max_running, r)
        assert b <= 3 << 20
        if q == 0 and r == 0:
            break
        time.sleep(0.001)
    for t in tickets:
        assert ctx.wait(t)[0] == bi.OK
    assert max_running <= 1
    ctx.close()


def test_host_requests_and_failures(bi):
    ctx = bi.Context(0, 2 << 30, 4)
    A = inputs.diag_dominant_uniform(200, 740)
    h = torch.from_numpy(A.copy()).pin_memory()
    st, t_ok = ctx.submit(200, None, h.data_ptr(), 200, bi.F64, bi.SUBMIT_HOST)
    J = torch.from_numpy(np.fliplr(np.eye(64)).copy()).cuda()
    st, t_bad = ctx.submit(64, [32, 32], J.data_ptr(), 64)
    N = inputs.diag_dominant_uniform(50, 741)
    N[3, 4] = np.nan
    dn = torch.from_numpy(N).cuda()
    st, t_nan = ctx.submit(50, [25, 25], dn.data_ptr(), 50)
    assert ctx.wait(t_ok)[0] == bi.OK
    assert rho(A, h.numpy()) <= 1e-12
    assert ctx.wait(t_bad)[0] == bi.ERR_SINGULAR
    assert ctx.wait(t_nan)[0] in (bi.ERR_NONFINITE, bi.ERR_SINGULAR)
    assert ctx.poll(123456789)[0] == bi.ERR_INVALID
    ctx.close()


def test_cancel_queued(bi):
    ctx = bi.Context(0, 4 << 30, 1)
    big = inputs.diag_dominant_uniform(2048, 750)
    d0 = torch.from_numpy(big).cuda()
    _, t0 = ctx.submit(2048, None, d0.data_ptr(), 2048)
    small = [torch.from_numpy(inputs.diag_dominant_uniform(64, 751 + i)).cuda() for i in range(5)]
    ts = [ctx.submit(64, None, d.data_ptr(), 64)[1] for d in small]
    assert ctx.cancel(ts[-1]) in (bi.OK, bi.PENDING)
    st_last = ctx.wait(ts[-1])[0]
    assert st_last in (bi.ERR_CANCELLED, bi.OK)
    assert ctx.wait(t0)[0] == bi.OK
    for t in ts[:-1]:
        assert ctx.wait(t)[0] == bi.OK
    ctx.close()
