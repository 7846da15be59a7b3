"""The benchmark's reporting arithmetic, on the CPU: the rooflines it prints
(flop counts of the FP8 residual, fractions of the measured peaks, which bound
applies in which mode), the error against the oracle, percentiles, the
partition of the benchmark workloads and the staleness rule of the recorded
DRAM traffic."""
import math
import types

import numpy as np
import pytest

import bench


def _trace(n):
    return {
        "residual_group_gemm_e4m3": {"launches": 2, "ms": 160.0, "flops": 1.0, "bytes": 0.0},
        "schur_update_tf32_tc": {"launches": 64, "ms": 40.0, "flops": 8.0e13, "bytes": 4.0e11},
        "schur_update_bf16_tc": {"launches": 64, "ms": 50.0, "flops": 8.0e13, "bytes": 4.0e11},
        "finalize": {"launches": 2, "ms": 10.0, "flops": 0.0, "bytes": 0.0},
    }


def test_measured_peak_ratios():
    p = bench.measured_peaks()
    assert p["fp8"] == pytest.approx(2 * p["bf16"])
    assert p["fp8_sustained"] == pytest.approx(2 * p["bf16_sustained"])
    assert p["tf32"] == pytest.approx(p["bf16"] * 1.1 / 2.25)
    assert p["tf32_sustained"] == pytest.approx(p["bf16_sustained"] * 1.1 / 2.25)
    assert p["source"] in ("measured", "fallback")


@pytest.mark.parametrize("iters,inc,groups,pairs", [
    (1, 1, 6, 45 + 21),      # one fresh residual, one incremental of 6 digit groups
    (2, 1, 3, 2 * 45 + 6),   # two fresh, one incremental of 3 groups
    (0, 0, 9, 45),           # converged before any update: the first residual only
])
def test_residual_flops_count_the_digit_products_that_ran(iters, inc, groups, pairs):
    n, nsteps = 1024, 3
    info = types.SimpleNamespace(refine_iters=iters, incremental_residuals=inc, incremental_groups=groups)
    trace = _trace(n)
    tensor, _, kt = bench.mixed_rooflines(n, trace, info, nsteps, "tf32")
    flops = nsteps * pairs * 2.0 * n ** 3
    assert trace["residual_group_gemm_e4m3"]["flops"] == flops
    assert tensor["algorithmic_flops_per_launch"] == flops / 2
    achieved = flops / 0.160 / 1e12
    assert tensor["achieved"] == pytest.approx(achieved)
    peaks = bench.measured_peaks()
    assert tensor["frac"] == pytest.approx(achieved / peaks["fp8_sustained"])
    assert tensor["frac_of_burst_peak"] == pytest.approx(achieved / peaks["fp8"])
    assert kt == pytest.approx(160.0 + 40.0 + 50.0 + 10.0)
    assert tensor["share_of_kernel_time"] == pytest.approx(160.0 / kt)


def test_schur_bound_follows_the_mode():
    n = 1024
    info = types.SimpleNamespace(refine_iters=1, incremental_residuals=1, incremental_groups=6)
    peaks = bench.measured_peaks()
    _, tf, _ = bench.mixed_rooflines(n, _trace(n), info, 1, "tf32")
    assert tf["bound"] == "tensor" and tf["unit"] == "TFLOP/s"
    assert tf["achieved"] == pytest.approx(8.0e13 / 0.040 / 1e12)
    assert tf["frac"] == pytest.approx(tf["achieved"] / peaks["tf32_sustained"])
    assert tf["hbm_frac"] == pytest.approx(4.0e11 / 0.040 / 1e9 / peaks["hbm_gbs"])
    _, bf, _ = bench.mixed_rooflines(n, _trace(n), info, 1, "bf16")
    assert bf["bound"] == "hbm" and bf["unit"] == "GB/s"
    assert bf["achieved"] == pytest.approx(4.0e11 / 0.050 / 1e9)
    assert bf["frac"] == pytest.approx(bf["achieved"] / peaks["hbm_gbs"])
    assert bf["tensor_frac"] == pytest.approx(8.0e13 / 0.050 / 1e12 / peaks["bf16_sustained"])


def test_split_tf32_update_sits_between_the_ridges():
    # 3 split products of 2b flops per element of X, 8 bytes of X moved (read + write FP32)
    b = 256
    intensity = 3 * 2 * b / 8
    peaks = bench.measured_peaks()
    assert peaks["tf32_sustained"] * 1e12 / (peaks["hbm_gbs"] * 1e9) < intensity
    assert intensity < peaks["bf16_sustained"] * 1e12 / (peaks["hbm_gbs"] * 1e9)


def test_eps_vs_oracle_matches_direct_norms():
    g = np.random.default_rng(5)
    xo = g.standard_normal((1000, 300))
    x = xo + 1e-9 * g.standard_normal(xo.shape)
    e = bench.eps_vs_oracle(x, xo, rows=128)
    assert e["eps_vs_oracle"] == pytest.approx(np.linalg.norm(x - xo) / np.linalg.norm(xo), rel=1e-12)
    assert e["eps_max_vs_oracle"] == pytest.approx(np.abs(x - xo).max() / np.abs(xo).max(), rel=1e-12)
    assert bench.eps_vs_oracle(xo, xo)["eps_vs_oracle"] == 0.0


def test_percentiles():
    xs = list(range(100, 0, -1))
    p = bench.percentiles(xs)
    assert (p["min"], p["max"]) == (1, 100)
    assert p["p50"] in (50, 51) and p["p99"] in (99, 100)
    assert bench.percentiles([7.0]) == {"p50": 7.0, "p99": 7.0, "min": 7.0, "max": 7.0}


@pytest.mark.parametrize("n,b,sizes", [(256, 64, [64] * 4), (16384, 256, [256] * 64), (1000, 256, [256] * 3 + [232])])
def test_partition(n, b, sizes):
    assert bench.partition(n, b) == sizes
    assert sum(bench.partition(n, b)) == n


def test_l2_note():
    assert bench.l2_note(16384).startswith("inputs larger than L2")
    assert bench.l2_note(256) == "fits L2"


def test_traffic_record_is_dropped_once_its_source_changes(monkeypatch):
    name = "k_refine.cu"
    good = {"bytes_per_launch": 123.0, "src": (name, bench.src_hash(name))}
    stale = {"bytes_per_launch": 456.0, "src": (name, "0" * 16)}
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("fake_kernel", 1), good)
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("fake_kernel", 2), stale)
    assert bench.ncu_traffic("fake_kernel", 1) == 123.0
    assert bench.ncu_traffic("fake_kernel", 2) is None
    assert bench.ncu_traffic("fake_kernel", 3) is None


def test_traffic_records_name_existing_sources():
    for (kernel, n), rec in bench.NCU_TRAFFIC.items():
        names, h = rec["src"]
        assert len(h) == 16 and int(h, 16) >= 0
        assert rec["bytes_per_launch"] > 0 and math.isfinite(rec["bytes_per_launch"])
        bench.src_hash(names)  # raises if a named source file is missing
