"""Serving context (continuous batching) through the C ABI: every result is
the same alone and in the mix (bit for bit, in FP64 and in the mixed modes),
small requests are coalesced into FP64 batch jobs, finished requests come out
of the completion queue once each, admission respects the HBM budget,
host-buffer requests, cancellation and per-request failures."""
import time

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
        assert eps_norm(X, Xo) <= fwd_bound(A, Xo) and eps_max(X, Xo) <= fwd_bound(A, Xo)
    ctx.close()


def test_alone_equals_mix_mixed(bi):
    """Mixed-mode requests (orders above the batching limit): the same bits
    alone on a one-slot context and all at once on a six-slot one."""
    mats = [inputs.gaussian_shifted(n, 770 + n, sigma=1.5) for n in (600, 800, 1000, 1400, 2100, 700)]
    modes = ["tf32", "bf16", "tf32", "bf16", "tf32", "tf32"]
    ctx1 = bi.Context(0, 8 << 30, 1)
    alone = []
    for A, m in zip(mats, modes):
        d = torch.from_numpy(A).cuda()
        st, t = ctx1.submit(A.shape[0], None, d.data_ptr(), A.shape[0], m)
        st, r = ctx1.wait(t)
        assert st == bi.OK and r.mode == bi.MODES[m] and 0 <= r.rho <= 1e-12
        alone.append(d.cpu().numpy())
    ctx1.close()
    ctx = bi.Context(0, 32 << 30, 6)
    ds = [torch.from_numpy(A).cuda() for A in mats]
    tickets = [ctx.submit(A.shape[0], None, d.data_ptr(), A.shape[0], m)[1] for A, d, m in zip(mats, ds, modes)]
    for t in tickets:
        assert ctx.wait(t)[0] == bi.OK
    for A, d, a in zip(mats, ds, alone):
        X = d.cpu().numpy()
        assert np.array_equal(X, a)
        assert rho(A, X) <= 1e-12
    ctx.close()


def test_small_requests_batched_and_completion_queue(bi):
    """Orders <= 512 in a mixed mode: coalesced into FP64 batch jobs (the
    record says FP64), each result within the FP64 tolerance of the oracle
    (with the batched engine's default partition, four near-equal blocks), and
    every ticket reported once by the completion queue."""
    mats = request_mix(780, 120, 5, 512)
    ctx = bi.Context(0, 8 << 30, 4)
    ds = [torch.from_numpy(A).cuda() for A in mats]
    tickets = [ctx.submit(A.shape[0], None, d.data_ptr(), A.shape[0], "tf32")[1] for A, d in zip(mats, ds)]
    seen = []
    t_end = time.time() + 60
    while len(seen) < len(tickets) and time.time() < t_end:
        seen += ctx.poll_done()
        time.sleep(0.001)
    assert sorted(seen) == sorted(tickets)
    assert ctx.poll_done() == []
    res = [ctx.poll(t) for t in tickets]
    bad = [(A.shape[0], st) for A, (st, r) in zip(mats, res) if st != bi.OK]
    assert not bad, (bad, bi.blockinv_last_cuda_error())
    for A, d, (st, r) in zip(mats, ds, res):
        assert r.mode == bi.F64 and r.rho == -1.0
        X = d.cpu().numpy()
        assert rho(A, X) <= 1e-12
        n = A.shape[0]
        sizes = [n] if n < 8 else oracle.quarter_partition(n)
        Xo = oracle.block_inverse(A, sizes)
        assert eps_norm(X, Xo) <= fwd_bound(A, Xo) and eps_max(X, Xo) <= fwd_bound(A, Xo)
    ctx.close()


def test_mixed_mode_requests(bi):
    # orders above 512 (smaller ones are coalesced into FP64 batch jobs)
    mats = [inputs.gaussian_shifted(n, 720 + n, sigma=1.5) for n in (600, 700, 1100)]
    ctx = bi.Context(0, 8 << 30, 3)
    ds = [torch.from_numpy(A).cuda() for A in mats]
    tickets = [ctx.submit(A.shape[0], None, d.data_ptr(), A.shape[0], "tf32")[1] for A, d in zip(mats, ds)]
    for A, d, t in zip(mats, ds, tickets):
        st, r = ctx.wait(t)
        assert st == bi.OK and 0 <= r.rho <= 1e-12 and r.refine_iters >= 1
        assert rho(A, d.cpu().numpy()) <= 1e-12
    ctx.close()


def test_mixed_fallback_for_ill_conditioned(bi):
    """B B^T + 0.1 I at n = 1500 (kappa ~ 1e5) in BF16: the refinement either
    brings it down or the request is rerun in FP64; either way it meets the gate."""
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


def test_block_size_autotuner_feeds_default_partition(bi):
    """blockinv_tune picks a block order per size class; calls with p = 0
    then use it (the result still meets the gate), and clearing restores 256."""
    assert bi.blockinv_tuning_clear() == bi.OK
    assert bi.blockinv_tune([900, 1000, 1100], "f64", 1) == bi.OK
    st, b = bi.blockinv_tuning("f64", 9)
    assert st == bi.OK and b in (64, 128, 192, 256, 320, 384, 512)
    A = inputs.gaussian_shifted(1000, 790, sigma=1.5)
    d = torch.from_numpy(A).cuda()
    bi.invert_(d, None)
    assert rho(A, d.cpu().numpy()) <= 1e-12
    assert bi.blockinv_tune([3000], "tf32", 1) == bi.OK
    assert bi.blockinv_tuning("tf32", 11)[1] > 0
    A = inputs.gaussian_shifted(3000, 791, sigma=1.5)
    d = torch.from_numpy(A).cuda()
    bi.invert_(d, None, "tf32")
    assert rho(A, d.cpu().numpy()) <= 1e-12
    assert bi.blockinv_tuning_clear() == bi.OK
