#!/usr/bin/env python3
"""Benchmark of the blockwise (Schur-complement) inversion on GB300.

One step = one full inversion of the workload matrix through the library's
C ABI: every pivot-block inverse, row panel and Schur update of the p
elimination steps (Eq. (a) applied once per diagonal block, in place), plus
the device copy of the pristine input into the work buffer. Inputs are
seeded synthetic matrices resident in HBM before the timed region; each is
512 MiB, larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun (N > 1) every rank inverts its
own matrix (independent problems, no collective on the data path); the step
time is the max over ranks and `value` counts the work of all ranks.

--impl reference times the CPU FP64 oracle (plain C, all host cores) on a
bounded sample of the same workload (order 4096, same block order and
distribution) and prints the same line with "impl": "reference".
"""
import argparse
import numpy as np
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective TFLOP/s & inverses/s at resid≤1e-12 vs FP64 GPU path; p50/p99 latency"
RHO_GATE = 1e-12

# FP64 ALU peak from unit counts: 2 DFMA/clock/SM x 2 flop x 152 SMs x 2.07 GHz.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12


def measured_peaks():
    """HBM and dense BF16 peaks measured by the driver on the GB300s;
    FP8 and TF32 from BF16 by the nominal ratios (4.5 / 2.25 and 1.1 / 2.25)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        src = "measured"
    except OSError:
        m = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
        src = "fallback"
    bf = m["bf16_tflops"]
    return {"hbm_gbs": m["hbm_gbs"], "bf16": bf, "fp8": bf * 2.0, "tf32": bf * 1.1 / 2.25,
            "bf16_sustained": m.get("bf16_tflops_sustained", bf), "source": src}

WORKLOADS = {
    "f64_8192": dict(n=8192, block=256, sigma=1.5, seed=2, mode="f64",
                     desc="8192x8192 FP64, 32x32 grid of 256x256 blocks, N(0,1)/sqrt(n)+1.5I, seed 2, plain FP64 GPU path"),
    "f64_6144": dict(n=6144, block=256, sigma=1.5, seed=2, mode="f64",
                     desc="6144x6144 FP64, 24x24 grid of 256x256 blocks, N(0,1)/sqrt(n)+1.5I, seed 2 (profiling case)"),
    "f64_256": dict(n=256, block=64, sigma=None, seed=1, mode="f64",
                    desc="256x256 FP64, 4x4 grid of 64x64 blocks, U[-1,1]+256I, seed 1"),
}
CPU_SAMPLE_N = 4096

# DRAM traffic per launch of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the kernel source
# it was measured on; reported as null once that source changes.
NCU_TRAFFIC = {
    # 6144 capture of one elimination step with look-ahead: the next-block part
    # (48.28 + 0.15 MB) and the rest (278.09 + 206.40 MB), 5888 x 6144 updated
    # elements per step; per launch = the step's total over its two launches,
    # scaled by updated elements to 7936 x 8192 per step at 8192.
    ("schur_update_f64", "f64_8192"): {"bytes_per_launch": 532.9e6 / 2 * (7936 * 8192) / (5888 * 6144),
                                       "src": "1910ef6dd2b79f18"},
    ("schur_update_f64", "f64_6144"): {"bytes_per_launch": 532.9e6 / 2, "src": "1910ef6dd2b79f18"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="f64_8192")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision + refinement legs")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched legs")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--serve-seconds", type=float, default=0.5,
                    help="length of the Poisson arrival window of the serving leg")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="measure library GEMM rates (FP64, FP32, TF32, BF16, FP16, FP8, INT8) and exit")
    return ap.parse_args()


def probe_peaks():
    """Library (cuBLAS) GEMM throughput per dtype, best of N with CUDA events:
    the denominators that the measured peak file does not carry."""
    import torch
    out = {}

    def best(fn, flops, iters):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        b = 1e30
        for _ in range(iters):
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            b = min(b, s.elapsed_time(e) / 1e3)
        return flops / b / 1e12

    n = 8192
    torch.backends.cuda.matmul.allow_tf32 = False
    for name, dt, it in [("f64", torch.float64, 3), ("f32_simt", torch.float32, 5),
                         ("bf16", torch.bfloat16, 10), ("f16", torch.float16, 10)]:
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        out[name] = best(lambda: a @ b, 2 * n ** 3, it)
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = True
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    out["tf32"] = best(lambda: a @ b, 2 * n ** 3, 10)
    a8 = a.to(torch.float8_e4m3fn)
    b8 = b.to(torch.float8_e4m3fn).t()
    one = torch.tensor(1.0, device="cuda")
    out["fp8_e4m3"] = best(lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16),
                           2 * n ** 3, 10)
    ai = torch.randint(-8, 8, (n, n), device="cuda", dtype=torch.int8)
    bi8 = torch.randint(-8, 8, (n, n), device="cuda", dtype=torch.int8)
    out["int8"] = best(lambda: torch._int_mm(ai, bi8), 2 * n ** 3, 10)
    print(json.dumps({"probe": "library GEMM TFLOP/s, 8192^3", **out}))


def make_input(w):
    from paper_2305_11103_gb300 import inputs
    if w["sigma"] is None:
        return inputs.diag_dominant_uniform(w["n"], w["seed"], shift=w["n"])
    return inputs.gaussian_shifted(w["n"], w["seed"], sigma=w["sigma"])


def partition(n, b):
    sizes = [b] * (n // b)
    if n % b:
        sizes.append(n % b)
    return sizes


def config_of(w, extra=None):
    c = {"workload": w["desc"], "n": w["n"], "block": w["block"], "mode": w["mode"],
         "l2": "inputs larger than L2 (no flush)" if w["n"] * w["n"] * 8 > 129 * 2**20 else "fits L2"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------- clocks ------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                rows.append(parts)
        os.unlink(self.path)
        sm = sorted(float(r[0]) for r in rows if r[0].replace(".", "").isdigit())
        mx = max((float(r[1]) for r in rows if r[1].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(rows)}


# -------------------------------------------------------------- oracle -----
def time_oracle(n, block, sigma, seed, repeats=1):
    """Seconds per inversion of the CPU oracle (all host cores) at order n."""
    import oracle
    from paper_2305_11103_gb300 import inputs
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    A = inputs.gaussian_shifted(n, seed, sigma=sigma) if sigma else inputs.diag_dominant_uniform(n, seed, shift=n)
    sizes = partition(n, block)
    ts = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.block_inverse(A, sizes)
        ts.append(time.perf_counter() - t0)
    return sum(ts) / len(ts), oracle.max_threads()


def cpu_baseline(w):
    n = min(w["n"], CPU_SAMPLE_N)
    sec, cores = time_oracle(n, w["block"], w["sigma"], w["seed"])
    return {"value": 2.0 * n ** 3 / sec / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"one inversion at order {n} ({n // w['block']} blocks of {w['block']}, same distribution), "
                      f"{sec:.2f} s, scaled as 2n^3/t"}


# ---------------------------------------------------------- distributed ----
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(ms_local, flops_per_rank, world):
    """(ms, TFLOP/s) of the whole job: every rank did flops_per_rank of work;
    the job takes as long as its slowest rank."""
    ms = max_over_ranks(ms_local, world)
    return ms, world * flops_per_rank / (ms / 1e3) / 1e12


def src_hash(*names):
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_2305_11103_gb300", "csrc", nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def percentiles(xs):
    ys = sorted(xs)
    pick = lambda q: ys[min(len(ys) - 1, int(round(q * (len(ys) - 1))))]
    return {"p50": pick(0.5), "p99": pick(0.99), "min": ys[0], "max": ys[-1]}


def run_mixed_paths(args, bi, torch, dA, dX, n, sizes, stream, fp64_ms):
    """The same matrix through the mixed-precision elimination (TF32 or BF16
    Schur updates on tensor cores) and Newton-Schulz refinement to
    rho <= 1e-12 with the FP64-accurate FP8 residual."""
    peaks = measured_peaks()
    out = {}
    for mode in ("tf32", "bf16"):
        def step():
            dX.copy_(dA)
            st, info = bi.blockinv_invert_ex(n, sizes, dX.data_ptr(), n, mode, stream, tol=RHO_GATE)
            if st != bi.OK:
                raise bi.BlockinvError(st, info.failing_block, f"blockinv_invert_ex({mode})")
            return info
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        infos = []
        for k in range(args.steps):
            infos.append(step())
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        per = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
        ms = sum(per) / len(per)
        rho64 = bi.residual(dA, dX)
        # Per-kernel times from a second pass of the same steps with one event
        # pair around every launch: events between a pivot inverse and the
        # update launched as its programmatic dependent serialise the two, so
        # this pass is not the timed one.
        bi.blockinv_trace_enable(True)
        for k in range(args.steps):
            step()
        torch.cuda.synchronize()
        bi.blockinv_trace_enable(False)
        trace = bi.blockinv_trace_summary()
        info = infos[-1]
        g = trace.get("residual_group_gemm_e4m3", {"ms": 0, "flops": 0, "launches": 0})
        if g["ms"]:
            # The host enqueues all 9 digit groups of an incremental residual
            # and the device skips those past its group count, so the traced
            # flops are replaced by the products that ran: 45 digit pairs per
            # fresh residual, G (G + 1) / 2 per incremental one.
            G = infos[-1].incremental_groups
            inc = infos[-1].incremental_residuals
            fresh = infos[-1].refine_iters + 1 - inc
            pairs = fresh * 45 + inc * G * (G + 1) // 2
            g = dict(g, flops=args.steps * pairs * 2.0 * n ** 3, flops_note="digit products that ran")
            trace["residual_group_gemm_e4m3"] = g
        schur = trace.get(f"schur_update_{mode}_tc", {"ms": 0, "bytes": 0, "launches": 0})
        kt_total = sum(v["ms"] for v in trace.values())
        achieved_g = g["flops"] / (g["ms"] / 1e3) / 1e12 if g["ms"] else None
        achieved_s = schur["bytes"] / (schur["ms"] / 1e3) / 1e9 if schur["ms"] else None
        out[mode] = {
            "ms_per_step": ms, "value": 2.0 * n ** 3 / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
            "inverses_per_s": 1e3 / ms, "speedup_vs_fp64_path": fp64_ms / ms,
            "latency_ms": percentiles(per),
            "rho_refinement": info.rho, "rho_initial": info.rho_initial, "rho_fp64_check": rho64,
            "refine_iters": info.refine_iters, "used_fallback": info.used_fallback,
            "incremental_digit_groups": info.incremental_groups,
            "roofline": {
                "bound": "tensor", "kernel": "residual_group_gemm_e4m3", "achieved": achieved_g,
                "peak": peaks["fp8"], "unit": "TFLOP/s",
                "frac": achieved_g / peaks["fp8"] if achieved_g else None,
                "peak_source": f"BF16 dense {peaks['source']} x 2 (FP8 / BF16 nominal ratio)",
                "share_of_kernel_time": g["ms"] / kt_total if kt_total else None},
            "roofline_schur_update": {
                "bound": "hbm", "kernel": f"schur_update_{mode}_tc", "achieved": achieved_s,
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved_s / peaks["hbm_gbs"] if achieved_s else None},
            "gpu_launches_per_step": sum(v["launches"] for v in trace.values()) / args.steps,
            "kernels": trace,
            "kernels_pass": "a second pass of the same steps, one event pair per launch (no overlap)",
            "kernels_pass_ms_per_step": kt_total / args.steps,
        }
    return out


def time_calls(torch, stream, reps, reset, call):
    """Mean ms of call() with an event pair around each call on `stream`, so
    the input reset between calls (reset(), the harness restoring the batch)
    is outside the timed intervals; also the mean ms per call with the reset."""
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in pairs:
        reset()
        a.record(stream)
        call()
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in pairs) / reps, t0.elapsed_time(t1) / reps


def run_batched(args, bi, torch, stream):
    """200 000 SPD 5 x 5 (one thread per matrix) and 2000 uneven matrices
    n in [8, 512] (grouped launches replayed from a CUDA graph)."""
    from paper_2305_11103_gb300 import inputs
    out = {}
    # --- 200 000 x 5 x 5 SPD, B B^T + 0.1 I, seed 5
    count, n = 200_000, 5
    A = inputs.spd_covariance_batch(count, n, 5)
    dA = torch.from_numpy(A).cuda()
    dX = torch.empty_like(dA)
    st = torch.empty(count, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        dX.copy_(dA)
        bi.blockinv_invert_batched_small(count, n, dX.data_ptr(), st.data_ptr(), stream)
    torch.cuda.synchronize()
    bi.blockinv_trace_enable(True)
    reps = max(args.steps, 10)
    ms, ms_reset = time_calls(torch, stream, reps, lambda: dX.copy_(dA),
                              lambda: bi.blockinv_invert_batched_small(count, n, dX.data_ptr(), st.data_ptr(), stream))
    bi.blockinv_trace_enable(False)
    tr = bi.blockinv_trace_summary()["small_batched_f64"]
    X = dX.cpu().numpy()
    R = np.einsum("bij,bjk->bik", A, X) - np.eye(n)[None]
    rho = np.linalg.norm(R, axis=(1, 2)) / (np.linalg.norm(A, axis=(1, 2)) * np.linalg.norm(X, axis=(1, 2)))
    kms = tr["ms"] / tr["launches"]
    peaks = measured_peaks()
    gbs = tr["bytes"] / tr["launches"] / (kms / 1e3) / 1e9
    tfs = tr["flops"] / tr["launches"] / (kms / 1e3) / 1e12
    out["spd5x5_200k"] = {
        "workload": "200000 SPD 5x5 FP64 (B B^T + 0.1 I, seed 5), blocks [2, 3], one thread per matrix",
        "ms_per_batch": ms, "inverses_per_s": count / (ms / 1e3), "kernel_ms": kms,
        "ms_per_batch_with_input_reset": ms_reset,
        "max_rho": float(rho.max()), "failed": int((st != 0).sum().item()),
        "roofline": {"bound": "alu", "kernel": "small_batched_f64", "achieved": tfs, "unit": "TFLOP/s",
                     "peak": FP64_PEAK_TFLOPS, "frac": tfs / FP64_PEAK_TFLOPS,
                     "hbm_achieved_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"],
                     "algorithmic": "2 n^3 = 250 flop and 2 x 200 B per matrix"},
    }
    del dA, dX, st
    # --- 200 000 x 11 x 11 SPD with blocks [5, 6] (the paper's tau matrices), seed 8
    count, n = 200_000, 11
    A = inputs.spd_covariance_batch(count, n, 8)
    dA = torch.from_numpy(A).cuda()
    dX = torch.empty_like(dA)
    st = torch.empty(count, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        dX.copy_(dA)
        bi.blockinv_invert_batched_fixed(count, n, [5, 6], dX.data_ptr(), bi.BATCH_SPD, st.data_ptr(), stream)
    torch.cuda.synchronize()
    bi.blockinv_trace_enable(True)
    reps = max(args.steps, 10)
    ms, ms_reset = time_calls(
        torch, stream, reps, lambda: dX.copy_(dA),
        lambda: bi.blockinv_invert_batched_fixed(count, n, [5, 6], dX.data_ptr(), bi.BATCH_SPD, st.data_ptr(), stream))
    bi.blockinv_trace_enable(False)
    tr = bi.blockinv_trace_summary()["tiny_batched_f64"]
    X = dX.cpu().numpy()
    R = np.einsum("bij,bjk->bik", A, X) - np.eye(n)[None]
    rho = np.linalg.norm(R, axis=(1, 2)) / (np.linalg.norm(A, axis=(1, 2)) * np.linalg.norm(X, axis=(1, 2)))
    kms = tr["ms"] / tr["launches"]
    gbs = tr["bytes"] / tr["launches"] / (kms / 1e3) / 1e9
    tfs = tr["flops"] / tr["launches"] / (kms / 1e3) / 1e12
    out["spd11x11_200k"] = {
        "workload": "200000 SPD 11x11 FP64 (B B^T + 0.1 I, seed 8), blocks [5, 6], 4 lanes x 3 rows per matrix",
        "ms_per_batch": ms, "inverses_per_s": count / (ms / 1e3), "kernel_ms": kms,
        "ms_per_batch_with_input_reset": ms_reset,
        "max_rho": float(rho.max()), "failed": int((st != 0).sum().item()),
        "symmetric": bool(np.array_equal(X, X.transpose(0, 2, 1))),
        "roofline": {"bound": "alu", "kernel": "tiny_batched_f64", "achieved": tfs, "unit": "TFLOP/s",
                     "peak": FP64_PEAK_TFLOPS, "frac": tfs / FP64_PEAK_TFLOPS,
                     "hbm_achieved_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"],
                     "algorithmic": "2 n^3 = 2662 flop and 2 x 968 B per matrix"},
    }
    del dA, dX, st
    # --- 2000 uneven matrices, n = round(exp(U(ln 8, ln 512))), U[-1,1] + n I, seed 6
    mats = inputs.uneven_batch(2000, 8, 512, 6)
    src = [torch.from_numpy(M).cuda() for M in mats]
    dst = [torch.empty_like(t) for t in src]
    ns = [t.shape[0] for t in src]
    stt = torch.empty(len(mats), dtype=torch.int32, device="cuda")

    def refresh():
        torch._foreach_copy_(dst, src)

    def time_plan():
        plan = bi.BatchPlan(ns, None, [t.data_ptr() for t in dst], ns)
        for _ in range(args.warmup):
            refresh()
            plan.run(stream, stt.data_ptr())
        torch.cuda.synchronize()
        bi.blockinv_trace_enable(True)
        per = []
        for _ in range(args.steps):
            refresh()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.run(stream, stt.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
            per.append(a.elapsed_time(b))
        bi.blockinv_trace_enable(False)
        tr = bi.blockinv_trace_summary()["batched_grouped_f64"]
        plan.close()
        return per, tr

    # default partitions (four blocks of n/4), then the autotuner's choice per size class
    bi.blockinv_batch_tuning_clear()
    per_default, _ = time_plan()
    t0 = time.time()
    st_tune = bi.blockinv_batch_tune(ns, 3, stream)
    tune_s = time.time() - t0
    if st_tune != bi.OK:
        raise bi.BlockinvError(st_tune, -1, "blockinv_batch_tune")
    table = {}
    for c in range(3, 10):
        _, pc, tile = bi.blockinv_batch_tuning(c)
        if pc:
            table[f"{2 ** c}-{2 ** (c + 1) - 1}"] = {"blocks": pc, "tile": tile}
    per, tr = time_plan()
    bi.blockinv_batch_tuning_clear()
    ms = sum(per) / len(per)
    ms_default = sum(per_default) / len(per_default)
    flops = sum(2.0 * m ** 3 for m in ns)
    g = inputs.rng(66)
    rhos = []
    for i in g.choice(len(mats), size=20, replace=False):
        Xi = dst[i].cpu().numpy()
        Ai = mats[i]
        rhos.append(np.linalg.norm(Ai @ Xi - np.eye(Ai.shape[0])) / (np.linalg.norm(Ai) * np.linalg.norm(Xi)))
    tfs = flops / (ms / 1e3) / 1e12
    out["uneven_2000"] = {
        "workload": "2000 FP64 matrices, n log-uniform in [8, 512], U[-1,1] + n I (seed 6); partitions and "
                    "Schur tiles from the autotuner",
        "ms_per_batch": ms, "inverses_per_s": len(mats) / (ms / 1e3), "value": tfs, "unit": "TFLOP/s",
        "latency_ms": percentiles(per), "max_rho_sampled": float(max(rhos)),
        "failed": int((stt != 0).sum().item()),
        "launches_per_batch": tr["launches"] / args.steps,
        "default_partition_ms_per_batch": ms_default,
        "autotune": {"seconds": tune_s, "table": table},
        "roofline": {"bound": "alu", "kernel": "batched_grouped_f64 (graph)", "achieved": tfs,
                     "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS, "frac": tfs / FP64_PEAK_TFLOPS},
    }
    return out


def run_serving(args, bi, torch):
    """Poisson arrivals at 2000 req/s, sizes log-uniform in [5, 4096] (70%
    U[-1,1] + n I, 30% B B^T + 0.1 I), through a serving context with a
    120 GB budget; FP64 and mixed TF32 + refinement."""
    from paper_2305_11103_gb300 import inputs
    rate, window = 2000.0, args.serve_seconds
    arrivals = inputs.poisson_arrivals(rate, window, 7)
    nreq = len(arrivals)
    # sizes quantised to 32 log-spaced orders; one pooled matrix per (order, kind)
    grid = np.unique(np.rint(np.exp(np.linspace(np.log(5), np.log(4096), 32))).astype(int))
    want = inputs.log_uniform_sizes(nreq, 5, 4096, 7)
    idx = np.abs(np.log(want)[:, None] - np.log(grid)[None, :]).argmin(axis=1)
    kinds = (inputs.rng(8).random(nreq) < 0.3).astype(int)
    pool = {}
    for k in sorted(set(zip(idx.tolist(), kinds.tolist()))):
        n = int(grid[k[0]])
        if k[1] == 0:
            M = torch.from_numpy(inputs.diag_dominant_uniform(n, 7000 + n, shift=n)).cuda()
        else:
            B = torch.from_numpy(inputs.rng(8000 + n).standard_normal((n, n))).cuda()
            M = B @ B.T + 0.1 * torch.eye(n, dtype=torch.float64, device="cuda")
        pool[k] = M
    out = {"workload": f"Poisson {rate:.0f} req/s for {window:g} s ({nreq} requests), n log-uniform in [5, 4096] "
                       f"quantised to {len(grid)} orders, 70% U[-1,1]+nI / 30% B B^T+0.1I, seed 7; "
                       "budget 120 GB, 16 slots"}
    for mode in ("f64", "tf32"):
        ctx = bi.Context(0, 120 << 30, 16)
        bufs, tickets, lat = {}, {}, []
        done = 0
        t0 = time.perf_counter()
        i = 0
        statuses = []
        while done < nreq:
            now = time.perf_counter() - t0
            while i < nreq and arrivals[i] <= now:
                key = (int(idx[i]), int(kinds[i]))
                buf = pool[key].clone()
                n = buf.shape[0]
                st, t = ctx.submit(n, None, buf.data_ptr(), n, mode)
                if st != bi.OK:
                    raise bi.BlockinvError(st, -1, "blockinv_submit")
                bufs[t] = buf
                tickets[t] = arrivals[i]
                i += 1
            for t in list(tickets):
                st, r = ctx.poll(t)
                if st == bi.PENDING:
                    continue
                lat.append(1e3 * ((time.perf_counter() - t0) - tickets.pop(t)))
                statuses.append(st)
                bufs.pop(t)
                done += 1
            if i < nreq and not tickets:
                time.sleep(max(0.0, arrivals[i] - (time.perf_counter() - t0)))
        wall = time.perf_counter() - t0
        ctx.close()
        flops = sum(2.0 * float(grid[k]) ** 3 for k in idx)
        out[mode] = {"completed": done, "wall_s": wall, "throughput_req_s": done / wall,
                     "offered_req_s": rate, "effective_tflops": flops / wall / 1e12,
                     "latency_ms": percentiles(lat), "failed": sum(1 for s in statuses if s != bi.OK)}
    return out


# ----------------------------------------------------------- our arm -------
def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    from paper_2305_11103_gb300 import blockinv as bi
    from paper_2305_11103_gb300 import build as libbuild
    if rank == 0:
        libbuild.build()
    barrier(world)
    bi.lib()
    w = WORKLOADS[args.workload]
    n, sizes, mode = w["n"], partition(w["n"], w["block"]), w["mode"]
    A = make_input(w)
    dev = torch.device("cuda", local)
    dA = torch.from_numpy(A).to(dev)
    dX = torch.empty_like(dA)
    stream = torch.cuda.current_stream(dev)

    def step():
        dX.copy_(dA)
        st = bi.blockinv_invert(n, sizes, dX.data_ptr(), n, mode, stream)
        if st != bi.OK:
            raise bi.BlockinvError(st, bi.blockinv_last_error_detail()[1], "blockinv_invert")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    bi.blockinv_trace_enable(True)
    torch.cuda.synchronize()
    barrier(world)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    e0, e1 = evs[0], evs[-1]
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    lat = percentiles(per_step)
    barrier(world)
    bi.blockinv_trace_enable(False)
    clk = clocks.stop()
    trace = bi.blockinv_trace_summary()
    flops = 2.0 * n ** 3
    ms, value = whole_job(e0.elapsed_time(e1) / args.steps, flops, world)
    fp64_ms = ms
    rho = bi.residual(dA, dX)

    top = max(trace.items(), key=lambda kv: kv[1]["ms"])
    kname, kt = top
    achieved = kt["flops"] / (kt["ms"] / 1e3) / 1e12
    traffic = None
    rec = NCU_TRAFFIC.get((kname, args.workload))
    if rec and rec["src"] == src_hash("k_update_f64.cu"):
        traffic = rec["bytes_per_launch"]
    total_ms = sum(v["ms"] for v in trace.values())
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": kname,
                "peak_source": "FP64 unit counts: 2 DFMA/clk/SM x 2 x 152 SMs x 2.07 GHz (not in MEASURED_PEAKS.json)",
                "algorithmic_flops_per_launch": kt["flops"] / kt["launches"],
                "share_of_kernel_time": kt["ms"] / total_ms if total_ms else None}
    launches = sum(v["launches"] for v in trace.values())

    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(A).pin_memory()
        hX = torch.empty_like(hA).pin_memory()
        tot = 0.0
        for it in range(args.warmup + args.steps):
            hX.copy_(hA)
            t0 = time.perf_counter()
            st = bi.blockinv_invert_host(n, sizes, hX.data_ptr(), n, mode, stream)
            t1 = time.perf_counter()
            if st != bi.OK:
                raise bi.BlockinvError(st, -1, "blockinv_invert_host")
            if it >= args.warmup:
                tot += t1 - t0
        e2e_ms, e2e_value = whole_job(tot / args.steps * 1e3, flops, world)
        e2e = {"value": e2e_value, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 8,
               "api": "blockinv_invert_host (pinned host buffer, copies inside the timed region)"}
        del hA, hX

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    mixed = {} if args.no_mixed else run_mixed_paths(args, bi, torch, dA, dX, n, sizes, stream, fp64_ms)
    del dA, dX
    torch.cuda.empty_cache()
    batched = {} if args.no_batched else run_batched(args, bi, torch, stream)
    serving = {} if args.no_serve else run_serving(args, bi, torch)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": config_of(w, {"parallelism": f"replicas{world}" if world > 1 else "single"}),
            "inverses_per_s": world * 1e3 / ms, "rho": rho, "rho_gate": RHO_GATE,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches, "kernels": trace,
            "latency_ms": lat,
            "mixed": mixed,
            "batched": batched,
            "serving": serving,
        }
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------ reference arm ------
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    n = min(w["n"], CPU_SAMPLE_N)
    for _ in range(args.warmup):
        time_oracle(n, w["block"], w["sigma"], w["seed"])
    tot, cores = 0.0, 1
    for _ in range(args.steps):
        sec, cores = time_oracle(n, w["block"], w["sigma"], w["seed"])
        tot += sec
    sec = tot / args.steps
    value = 2.0 * n ** 3 / sec / 1e12
    sample = (f"one inversion per step at order {n} ({n // w['block']} blocks of {w['block']}, same distribution), "
              f"scaled as 2n^3/t")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    args = parse()
    if args.probe_peaks:
        probe_peaks()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
