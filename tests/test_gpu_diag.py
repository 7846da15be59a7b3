"""Device helpers checked on their own through the C ABI's diagnostic entry
points: the FP64 reciprocal of the batched kernels against IEEE division, and
the bounded device wait that every tensor-core kernel uses, made to run out so
that it reports BLOCKINV_ERR_TIMEOUT."""
import numpy as np
import pytest

from paper_2305_11103_gb300 import blockinv

pytestmark = pytest.mark.gpu


def ulp_distance(a, b):
    """|a - b| in units in the last place (same-sign finite doubles)."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_recip64_within_one_ulp_of_ieee_division():
    import torch
    g = np.random.Generator(np.random.PCG64(2024))
    # log-uniform magnitudes over the normal range where 1/v is normal too,
    # both signs, plus powers of two and values next to them
    mag = np.exp2(g.uniform(-1020.0, 1020.0, size=4_000_000))
    v = mag * np.where(g.random(mag.size) < 0.5, -1.0, 1.0)
    p2 = np.exp2(np.arange(-1020, 1021, dtype=np.float64))
    v = np.concatenate([v, p2, -p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), [1.0, -1.0, 3.0, 0.1]])
    dv = torch.from_numpy(v).cuda()
    dout = torch.empty_like(dv)
    assert blockinv.blockinv_diag_recip64(dv.data_ptr(), dout.data_ptr(), v.size, None) == blockinv.OK
    torch.cuda.synchronize()
    got = dout.cpu().numpy()
    want = 1.0 / v
    d = ulp_distance(got, want)
    assert d.max() <= 1, (d.max(), v[d.argmax()])
    # powers of two have exact reciprocals
    k = v.size - 4 - 4 * p2.size
    assert np.array_equal(got[k:k + 2 * p2.size], want[k:k + 2 * p2.size])
    # outside the normal range the IEEE division itself
    edge = np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, 1e-310, 1.7e308, np.nan])
    de = torch.from_numpy(edge).cuda()
    do = torch.empty_like(de)
    assert blockinv.blockinv_diag_recip64(de.data_ptr(), do.data_ptr(), edge.size, None) == blockinv.OK
    torch.cuda.synchronize()
    with np.errstate(divide="ignore", over="ignore"):
        np.testing.assert_array_equal(do.cpu().numpy(), 1.0 / edge)


def test_bounded_wait_reports_timeout():
    # a wait on a barrier that nothing completes, limited to 1 ms
    assert blockinv.blockinv_diag_wait_timeout(1_000_000, None) == blockinv.ERR_TIMEOUT
    assert blockinv.blockinv_status_str(blockinv.ERR_TIMEOUT) == "device wait timed out"
    # the context stays usable: an inversion right after it succeeds
    import torch
    A = torch.eye(64, dtype=torch.float64, device="cuda") * 2.0
    blockinv.invert_(A, [32, 32])
    assert torch.equal(A, torch.eye(64, dtype=torch.float64, device="cuda") * 0.5)


def test_zero_limit_wait_times_out_at_once():
    assert blockinv.blockinv_diag_wait_timeout(0, None) == blockinv.ERR_TIMEOUT
