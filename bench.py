#!/usr/bin/env python3
"""Benchmark of the blockwise (Schur-complement) inversion on GB300.

The headline workload is a 16384 x 16384 matrix, a 64 x 64 grid of 256 x 256
blocks, entries N(0,1)/sqrt(n) plus sigma I (sigma 1.5, seed 3). One step is
one full inversion through the library's C ABI in the mixed mode: Eq. (a)
applied once per diagonal block, in place, on an FP32 copy with the Schur
updates on TF32 tensor cores (FP32 accumulation), then Newton-Schulz
refinement X <- X + X (I - A X) with an FP64-accurate residual until
rho = ||AX - I||_F / (||A||_F ||X||_F) <= 1e-12, plus the device copy of the
pristine input into the work buffer. Inputs (2 GiB) are resident in HBM
before the timed region and larger than L2, so no flush is needed.

Beside it, in the same JSON line: the same matrix in BF16 mode and at
sigma 1.05 (seed 4); the plain FP64 GPU path on the same matrix (the "vs FP64
GPU path" comparison); the 8192 FP64 workload; the 256 FP64 workload
(microseconds per inverse from graph replays); the batched and serving legs;
and, for every result, the error against the CPU oracle,
eps = ||X - X_oracle||_F / ||X_oracle||_F, with the oracle (plain C, Eq. (a)
recursively) run at each workload's own order in a separate process while the
GPU legs run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun (N > 1) every rank inverts its
own matrices (independent problems, no collective on the data path); the
step time is the max over ranks and `value` counts the work of all ranks.

--impl reference times the CPU FP64 oracle (all host cores) on a bounded
sample of the headline workload (order 4096 with the same block order and
distribution per step, scaled as 2 n^3 / t) and prints the same line with
"impl": "reference".
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective TFLOP/s & inverses/s at resid≤1e-12 vs FP64 GPU path; p50/p99 latency"
RHO_GATE = 1e-12

# FP64 ALU peak from unit counts: 2 DFMA/clock/SM x 2 flop x 152 SMs x 2.07 GHz.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12


def measured_peaks():
    """HBM and dense BF16 peaks measured on the GB300s (burst and
    sustained); FP8 and TF32 from BF16 by the nominal ratios (4.5 / 2.25 and
    1.1 / 2.25)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        src = "measured"
    except OSError:
        m = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
        src = "fallback"
    bf = m["bf16_tflops"]
    bfs = m.get("bf16_tflops_sustained", bf)
    return {"hbm_gbs": m["hbm_gbs"], "bf16": bf, "bf16_sustained": bfs, "fp8": 2.0 * bf,
            "fp8_sustained": 2.0 * bfs, "tf32": bf * 1.1 / 2.25, "tf32_sustained": bfs * 1.1 / 2.25,
            "source": src}


WORKLOADS = {
    "mixed_16384": dict(
        n=16384, block=256, kind="mixed", legs=((3, 1.5), (4, 1.05)), modes=("tf32", "bf16"),
        desc="16384x16384, 64x64 grid of 256x256 blocks, N(0,1)/sqrt(n)+sigma I (sigma 1.5 seed 3, "
             "headline; sigma 1.05 seed 4), Schur GEMMs in TF32 (headline) and BF16 with FP32 "
             "accumulation + Newton-Schulz refinement to rho<=1e-12 with an FP64-accurate residual, "
             "vs the plain FP64 GPU path on the same matrix"),
    "mixed_8192": dict(
        n=8192, block=256, kind="mixed", legs=((2, 1.5),), modes=("tf32", "bf16"),
        desc="8192x8192, 32x32 grid of 256x256 blocks, N(0,1)/sqrt(n)+1.5I, seed 2, mixed TF32/BF16 + "
             "Newton-Schulz refinement to rho<=1e-12 (shorter run of the mixed path)"),
    "f64_8192": dict(n=8192, block=256, kind="f64", sigma=1.5, seed=2,
                     desc="8192x8192 FP64, 32x32 grid of 256x256 blocks, N(0,1)/sqrt(n)+1.5I, seed 2, "
                          "plain FP64 GPU path"),
    "f64_6144": dict(n=6144, block=256, kind="f64", sigma=1.5, seed=2,
                     desc="6144x6144 FP64, 24x24 grid of 256x256 blocks, N(0,1)/sqrt(n)+1.5I, seed 2 "
                          "(profiling case)"),
    "f64_256": dict(n=256, block=64, kind="f64", sigma=None, seed=1,
                    desc="256x256 FP64, 4x4 grid of 64x64 blocks, U[-1,1]+256I, seed 1"),
}
CPU_SAMPLE_N = 4096
SERVE_SLOTS = 32
SERVE_INFLIGHT = 512  # requests submitted and not finished, at most (device memory of their inputs)
SERVE_DRAIN_S = 240.0  # after a serving window, how long unfinished requests are waited for
stuck_contexts = []  # serving contexts with requests that never completed (not closed)

# DRAM traffic per launch of a kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the kernel source
# it was measured on; reported as null once that source changes.
NCU_TRAFFIC = {
    # 6144 capture of one FP64 elimination step with look-ahead: the
    # next-block part (48.28 + 0.15 MB) and the rest (278.09 + 206.40 MB),
    # 5888 x 6144 updated elements per step; per launch = the step's total
    # over its two launches, scaled by updated elements to 7936 x 8192 per
    # step at 8192.
    ("schur_update_f64", 8192): {"bytes_per_launch": 532.9e6 / 2 * (7936 * 8192) / (5888 * 6144),
                                 "src": ("k_update_f64.cu", "1910ef6dd2b79f18")},
    ("schur_update_f64", 6144): {"bytes_per_launch": 532.9e6 / 2, "src": ("k_update_f64.cu", "1910ef6dd2b79f18")},
    # 16384 mixed TF32 solve: the fresh residual (444.15 + 32.20 GB) and the
    # incremental one (187.43 + 17.16 GB), averaged over the two launches
    ("residual_group_gemm_e4m3", 16384): {"bytes_per_launch": (444.15e9 + 32.20e9 + 187.43e9 + 17.16e9) / 2,
                                          "src": (("k_refine.cu", "tc_gemm.cuh", "tc_common.cuh"),
                                                  "2bc8f9508a2b6ac1")},
    # the rest of one step's TF32 update (the launch after the next block's square)
    ("schur_update_tf32_tc", 16384): {"bytes_per_launch": 1.33e9 + 0.999e9,
                                      "src": (("k_mixed.cu", "tc_gemm.cuh", "tc_common.cuh"), "dd4ffd6395993da7")},
}


_T0 = time.time()


def progress(msg):
    """One line per leg on stderr (the JSON result goes to stdout)."""
    print(f"[bench {time.time() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="mixed_16384")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the CPU oracle (no eps against it, no cpu_baseline)")
    ap.add_argument("--no-fp64-path", action="store_true",
                    help="skip the plain FP64 GPU path on the headline matrix")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the 8192 and 256 FP64 legs")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched legs")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson arrival window of the mixed serving leg")
    ap.add_argument("--serve-seconds-f64", type=float, default=0.5,
                    help="length of the arrival window of the FP64 serving leg (it cannot keep up)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed inversions of the FP64 GPU path on the 16384 matrix (7 s each)")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="measure library GEMM rates (FP64, FP32, TF32, BF16, FP16, FP8, INT8) and exit")
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="for profilers: run this many plain blocking inversions of the workload's first "
                         "matrix in its first mode (no timing, no other leg) and exit")
    ap.add_argument("--profile-batch-runs", type=int, default=0,
                    help="for profilers: run the 2000-matrix uneven batch plan this many times and exit")
    return ap.parse_args()


def profile_run(args):
    """A bare workload for profilers (ncu): no timing, no oracle, no other leg."""
    import torch
    from paper_2305_11103_gb300 import blockinv as bi
    from paper_2305_11103_gb300 import build as libbuild
    from paper_2305_11103_gb300 import inputs
    libbuild.build()
    bi.lib()
    if args.profile_batch_runs:
        mats = inputs.uneven_batch(2000, 8, 512, 6)
        src = [torch.from_numpy(M).cuda() for M in mats]
        dst = [torch.empty_like(t) for t in src]
        ns = [t.shape[0] for t in src]
        st = torch.empty(len(mats), dtype=torch.int32, device="cuda")
        plan = bi.BatchPlan(ns, None, [t.data_ptr() for t in dst], ns)
        for _ in range(args.profile_batch_runs):
            torch._foreach_copy_(dst, src)
            plan.run(None, st.data_ptr())
        torch.cuda.synchronize()
        plan.close()
        print(json.dumps({"profile": "uneven batch plan", "runs": args.profile_batch_runs,
                          "failed": int((st != 0).sum().item())}))
        return
    w = WORKLOADS[args.workload]
    n, sizes = w["n"], partition(w["n"], w["block"])
    if w["kind"] == "mixed":
        (seed, sigma), mode = w["legs"][0], w["modes"][0]
    else:
        seed, sigma, mode = w["seed"], w["sigma"], "f64"
    dA = torch.from_numpy(make_matrix(n, sigma, seed)).cuda()
    dX = torch.empty_like(dA)
    for _ in range(args.profile_solves):
        dX.copy_(dA)
        st, info = bi.blockinv_invert_ex(n, sizes, dX.data_ptr(), n, mode, None, tol=RHO_GATE)
        if st != bi.OK:
            raise bi.BlockinvError(st, info.failing_block, "blockinv_invert_ex")
    torch.cuda.synchronize()
    print(json.dumps({"profile": w["desc"], "mode": mode, "solves": args.profile_solves}))


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


def make_matrix(n, sigma, seed):
    from paper_2305_11103_gb300 import inputs
    if sigma is None:
        return inputs.diag_dominant_uniform(n, seed, shift=n)
    return inputs.gaussian_shifted(n, seed, sigma=sigma)


def partition(n, b):
    sizes = [b] * (n // b)
    if n % b:
        sizes.append(n % b)
    return sizes


def l2_note(n):
    return "inputs larger than L2 (no flush)" if n * n * 8 > 129 * 2 ** 20 else "fits L2"


def src_hash(names):
    """Hash of the kernel sources a traffic record was measured on."""
    h = hashlib.sha256()
    for name in ((names,) if isinstance(names, str) else names):
        with open(os.path.join(ROOT, "paper_2305_11103_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n):
    rec = NCU_TRAFFIC.get((kernel, n))
    if rec and src_hash(rec["src"][0]) == rec["src"][1]:
        return rec["bytes_per_launch"]
    return None


def percentiles(xs):
    ys = sorted(xs)
    pick = lambda q: ys[min(len(ys) - 1, int(round(q * (len(ys) - 1))))]
    return {"p50": pick(0.5), "p99": pick(0.99), "min": ys[0], "max": ys[-1]}


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


class UtilSampler:
    """nvidia-smi utilization.gpu every 200 ms (mean and median over the window)."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=utilization.gpu", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait()
        vals = [float(v) for v in open(self.path).read().split() if v.replace(".", "").isdigit()]
        os.unlink(self.path)
        if not vals:
            return None
        vals.sort()
        return {"mean": sum(vals) / len(vals), "median": vals[len(vals) // 2], "samples": len(vals)}


# -------------------------------------------------------------- oracle -----
def oracle_threads():
    """Host threads for the oracle while GPU legs run: every core but one,
    which the process driving the GPU keeps."""
    return max(1, (os.cpu_count() or 1) - 1)


def _oracle_worker(jobs, threads, outdir, q):
    """Runs in a spawned process: the oracle's X for each (key, n, block,
    sigma, seed), saved as .npy under outdir; reports (key, seconds, threads,
    path) on q, then None."""
    try:
        import oracle
        oracle.set_threads(threads)
        for key, n, block, sigma, seed in jobs:
            A = make_matrix(n, sigma, seed)
            t0 = time.perf_counter()
            X = oracle.block_inverse(A, partition(n, block))
            sec = time.perf_counter() - t0
            del A
            path = os.path.join(outdir, key + ".npy")
            np.save(path, X)
            del X
            q.put((key, sec, oracle.max_threads(), path, None))
    except Exception as exc:  # reported to the parent, which states it in the JSON
        q.put(("error", 0.0, 0, None, repr(exc)))
    q.put(None)


class OracleRuns:
    """The oracle's inverses of the large workloads, computed in a spawned
    process (its own interpreter, no CUDA) while the GPU legs run."""

    def __init__(self, jobs):
        import multiprocessing as mp
        self.dir = tempfile.mkdtemp(prefix="blockinv_oracle_")
        self.threads = oracle_threads()
        self.results = {}
        self.error = None
        ctx = mp.get_context("spawn")
        self.q = ctx.Queue()
        self.proc = ctx.Process(target=_oracle_worker, args=(jobs, self.threads, self.dir, self.q), daemon=True)
        self.proc.start()
        self.done = False

    def get(self, key, limit_s=1800.0):
        """Block until the oracle's X for `key` is ready: (seconds, threads,
        X as a read-only memory map) or None if the worker failed or did not
        deliver within limit_s."""
        import queue
        t_end = time.time() + limit_s
        while key not in self.results and not self.done:
            if time.time() > t_end:
                self.error = self.error or f"no result for {key} within {limit_s:.0f} s"
                break
            try:
                item = self.q.get(timeout=5)
            except queue.Empty:
                if not self.proc.is_alive():
                    self.done = True
                    self.error = self.error or f"oracle worker exited with code {self.proc.exitcode}"
                continue
            if item is None:
                self.done = True
                break
            k, sec, thr, path, err = item
            if err:
                self.error = err
            else:
                self.results[k] = (sec, thr, path)
        if key not in self.results:
            return None
        sec, thr, path = self.results[key]
        return sec, thr, np.load(path, mmap_mode="r")

    def drop(self, key):
        if key in self.results:
            try:
                os.unlink(self.results[key][2])
            except OSError:
                pass

    def close(self):
        for k in list(self.results):
            self.drop(k)
        if self.proc.is_alive():
            self.proc.join(timeout=1)
        if self.proc.is_alive():
            self.proc.terminate()
        try:
            os.rmdir(self.dir)
        except OSError:
            pass


def eps_vs_oracle(X, Xo, rows=1024):
    """Normwise ||X - Xo||_F / ||Xo||_F and max-norm max|X - Xo| / max|Xo|,
    accumulated over row blocks (no full-size temporaries)."""
    n = Xo.shape[0]
    d2 = o2 = 0.0
    dmax = omax = 0.0
    for r in range(0, n, rows):
        xo = np.asarray(Xo[r:r + rows], dtype=np.float64)
        d = np.asarray(X[r:r + rows], dtype=np.float64) - xo
        d2 += float(np.einsum("ij,ij->", d, d))
        o2 += float(np.einsum("ij,ij->", xo, xo))
        dmax = max(dmax, float(np.abs(d).max()))
        omax = max(omax, float(np.abs(xo).max()))
    return {"eps_vs_oracle": math.sqrt(d2) / math.sqrt(o2), "eps_max_vs_oracle": dmax / omax}


def small_oracle(A, sizes):
    import oracle
    return oracle.block_inverse(A, sizes)


def time_oracle(n, block, sigma, seed, repeats=1):
    """Seconds per inversion of the CPU oracle (all host cores) at order n."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    A = make_matrix(n, sigma, seed)
    sizes = partition(n, block)
    ts = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.block_inverse(A, sizes)
        ts.append(time.perf_counter() - t0)
    return sum(ts) / len(ts), oracle.max_threads()


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


# ------------------------------------------------------------ GPU legs -----
def run_solves(bi, torch, stream, dA, dX, n, sizes, mode, steps, warmup):
    """warmup + steps blocking inversions of dA into dX (the copy of the
    pristine input is part of each step); per-step ms from CUDA events on the
    launching stream, and the report of each mixed solve."""
    def step():
        dX.copy_(dA)
        if mode == "f64":
            st = bi.blockinv_invert(n, sizes, dX.data_ptr(), n, mode, stream)
            if st != bi.OK:
                raise bi.BlockinvError(st, bi.blockinv_last_error_detail()[1], "blockinv_invert")
            return None
        st, info = bi.blockinv_invert_ex(n, sizes, dX.data_ptr(), n, mode, stream, tol=RHO_GATE)
        if st != bi.OK:
            raise bi.BlockinvError(st, info.failing_block, f"blockinv_invert_ex({mode})")
        return info

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    infos = []
    for k in range(steps):
        infos.append(step())
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return per, infos, step


def trace_pass(bi, torch, step, nsteps):
    """Per-kernel {launches, ms, flops, bytes} over nsteps more steps, with one
    event pair around every launch. Events between a kernel and its
    programmatic dependent serialise the two, so this pass is not the timed
    one."""
    bi.blockinv_trace_enable(True)
    for _ in range(nsteps):
        step()
    torch.cuda.synchronize()
    bi.blockinv_trace_enable(False)
    return bi.blockinv_trace_summary()


def mixed_report(n, per, info, fp64_rho):
    ms = sum(per) / len(per)
    return {"ms_per_step": ms, "value": 2.0 * n ** 3 / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
            "inverses_per_s": 1e3 / ms, "latency_ms": percentiles(per),
            "rho_refinement": info.rho, "rho_initial": info.rho_initial, "rho_fp64_check": fp64_rho,
            "refine_iters": info.refine_iters, "used_fallback": info.used_fallback,
            "incremental_residuals": info.incremental_residuals,
            "incremental_digit_groups": info.incremental_groups, "fp64_pivots": info.fp64_pivots}


def mixed_rooflines(n, trace, info, nsteps, mode):
    """Rooflines of the two mixed-path kernels that bound it, from the trace
    pass: the FP8 residual GEMM (tensor) and the TF32/BF16 Schur update. The
    update moves 8 bytes of X per element and does 3 x 2b flops on it (three
    split products): 192 flop/B at b = 256, above the TF32 ridge (the sustained
    TF32 peak / HBM, 125 flop/B) and below the BF16 one (250), so its bound is
    the TF32 tensor pipe in TF32 mode and HBM in BF16 mode; both fractions are
    given."""
    peaks = measured_peaks()
    g = dict(trace.get("residual_group_gemm_e4m3", {"ms": 0, "flops": 0, "launches": 0}))
    if g["ms"]:
        # The host enqueues all 9 digit groups of an incremental residual and
        # the device skips those past its group count, so the traced flops
        # are replaced by the digit products that ran: 45 pairs per fresh
        # residual, G (G + 1) / 2 per incremental one.
        G = info.incremental_groups
        inc = info.incremental_residuals
        fresh = info.refine_iters + 1 - inc
        pairs = fresh * 45 + inc * G * (G + 1) // 2
        g["flops"] = nsteps * pairs * 2.0 * n ** 3
        g["flops_note"] = "digit products that ran"
        trace["residual_group_gemm_e4m3"] = g
    schur = trace.get(f"schur_update_{mode}_tc", {"ms": 0, "bytes": 0, "launches": 0})
    kt_total = sum(v["ms"] for v in trace.values())
    ag = g["flops"] / (g["ms"] / 1e3) / 1e12 if g["ms"] else None
    ags = schur["bytes"] / (schur["ms"] / 1e3) / 1e9 if schur["ms"] else None
    tensor = {
        "bound": "tensor", "kernel": "residual_group_gemm_e4m3 (gemm_kernel<E4M3, EpiAccumI64>)",
        "achieved": ag, "peak": peaks["fp8_sustained"], "unit": "TFLOP/s",
        "frac": ag / peaks["fp8_sustained"] if ag else None,
        "frac_of_burst_peak": ag / peaks["fp8"] if ag else None,
        "peak_source": f"2 x the sustained dense BF16 figure ({peaks['source']}): FP8 / BF16 nominal ratio; "
                       "the kernel runs inside seconds-long loops of solves",
        "algorithmic_flops_per_launch": g["flops"] / g["launches"] if g["launches"] else None,
        "traffic": ncu_traffic("residual_group_gemm_e4m3", n),
        "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum per launch, mean of the fresh and the "
                        "incremental residual (profiles/mixed_solve_16384.md)",
        "share_of_kernel_time": g["ms"] / kt_total if kt_total else None}
    agf = schur["flops"] / (schur["ms"] / 1e3) / 1e12 if schur["ms"] else None
    tpeak = peaks["tf32_sustained"] if mode == "tf32" else peaks["bf16_sustained"]
    hbm_frac = ags / peaks["hbm_gbs"] if ags else None
    tensor_frac = agf / tpeak if agf else None
    common = {"kernel": f"schur_update_{mode}_tc (gemm_kernel<{mode.upper()}, EpiSchurF32>)",
              "algorithmic_bytes_per_launch": schur["bytes"] / schur["launches"] if schur["launches"] else None,
              "algorithmic_flops_per_launch": schur["flops"] / schur["launches"] if schur["launches"] else None,
              "hbm_achieved_gbs": ags, "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_frac": hbm_frac,
              "tensor_achieved_tflops": agf, "tensor_peak_tflops": tpeak, "tensor_frac": tensor_frac,
              "tensor_peak_source": f"sustained dense {mode.upper()}: " + (
                  "the sustained BF16 figure x 1.1 / 2.25 (nominal TF32 / BF16 ratio)" if mode == "tf32"
                  else "the sustained BF16 figure") + f" ({peaks['source']})",
              "traffic": ncu_traffic(f"schur_update_{mode}_tc", n),
              "traffic_note": "one launch of the rest of a step (after the next block's square)",
              "share_of_kernel_time": schur["ms"] / kt_total if kt_total else None}
    if mode == "tf32":
        schur_rl = dict({"bound": "tensor", "achieved": agf, "peak": tpeak, "unit": "TFLOP/s",
                         "frac": tensor_frac}, **common)
    else:
        schur_rl = dict({"bound": "hbm", "achieved": ags, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": hbm_frac}, **common)
    return tensor, schur_rl, kt_total


def run_cfg1(args, bi, torch):
    """256 x 256 FP64, [64] x 4, U[-1,1] + 256 I (seed 1): microseconds per
    inverse from back-to-back replays of a CUDA graph holding the input copy
    and blockinv_invert_async, and the pivot kernel's share from a traced
    pass of plain calls."""
    w = WORKLOADS["f64_256"]
    n, sizes = w["n"], partition(w["n"], w["block"])
    A = make_matrix(n, w["sigma"], w["seed"])
    dA = torch.from_numpy(A).cuda()
    dX = torch.empty_like(dA)
    st_dev = torch.zeros(2, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    out = {"workload": w["desc"]}

    def call(stream):
        with torch.cuda.stream(stream):  # the input copy on the stream the inversion runs on
            dX.copy_(dA)
        st = bi.blockinv_invert_async(n, sizes, dX.data_ptr(), n, "f64", stream, st_dev.data_ptr())
        if st != bi.OK:
            raise bi.BlockinvError(st, -1, "blockinv_invert_async")

    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup)):
            call(s)
    torch.cuda.synchronize()
    reps = 200
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            call(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(3):
                g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            a.record(s)
            for _ in range(reps):
                g.replay()
            b.record(s)
        torch.cuda.synchronize()
        out["method"] = f"{reps} back-to-back replays of one CUDA graph (input copy + blockinv_invert_async)"
        ms = a.elapsed_time(b) / reps
    except Exception as exc:  # capture not possible: plain back-to-back stream-ordered calls
        torch.cuda.synchronize()
        out["graph_error"] = repr(exc)[:200]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            a.record(s)
            for _ in range(reps):
                call(s)
            b.record(s)
        torch.cuda.synchronize()
        out["method"] = f"{reps} back-to-back stream-ordered blockinv_invert_async calls (no graph)"
        ms = a.elapsed_time(b) / reps
    status = int(st_dev[0].item())
    trace = trace_pass(bi, torch, lambda: call(s), 10)
    kt_total = sum(v["ms"] for v in trace.values())
    piv = trace.get("pivot_inverse_f64", {"ms": 0, "launches": 1})
    X = dX.cpu().numpy()
    Xo = small_oracle(A, sizes)
    out.update({"us_per_inverse": ms * 1e3, "inverses_per_s": 1e3 / ms, "status": status,
                "rho": bi.residual(dA, dX), **eps_vs_oracle(X, Xo),
                "pivot_share_of_kernel_time": piv["ms"] / kt_total if kt_total else None,
                "pivot_us_per_launch": 1e3 * piv["ms"] / max(1, piv["launches"]),
                "kernels": trace})
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


def batch_eps(A, X, sizes, count, seed):
    """eps against the oracle on `count` sampled matrices of a batch."""
    from paper_2305_11103_gb300 import inputs
    idx = inputs.rng(seed).choice(A.shape[0], size=count, replace=False)
    eps, epsm = [], []
    for i in idx:
        e = eps_vs_oracle(X[i], small_oracle(A[i], sizes))
        eps.append(e["eps_vs_oracle"])
        epsm.append(e["eps_max_vs_oracle"])
    return {"eps_vs_oracle_max_sampled": float(max(eps)), "eps_max_vs_oracle_max_sampled": float(max(epsm)),
            "eps_sample": f"{count} matrices (seed {seed})"}


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
    eps5 = batch_eps(A, X, [2, 3], 1000, 55)
    kms = tr["ms"] / tr["launches"]
    peaks = measured_peaks()
    gbs = tr["bytes"] / tr["launches"] / (kms / 1e3) / 1e9
    tfs = tr["flops"] / tr["launches"] / (kms / 1e3) / 1e12
    out["spd5x5_200k"] = {
        "workload": "200000 SPD 5x5 FP64 (B B^T + 0.1 I, seed 5), blocks [2, 3], one thread per matrix",
        "ms_per_batch": ms, "inverses_per_s": count / (ms / 1e3), "kernel_ms": kms,
        "ms_per_batch_with_input_reset": ms_reset,
        "max_rho": float(rho.max()), "failed": int((st != 0).sum().item()), **eps5,
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
    eps11 = batch_eps(A, X, [5, 6], 1000, 56)
    kms = tr["ms"] / tr["launches"]
    gbs = tr["bytes"] / tr["launches"] / (kms / 1e3) / 1e9
    tfs = tr["flops"] / tr["launches"] / (kms / 1e3) / 1e12
    out["spd11x11_200k"] = {
        "workload": "200000 SPD 11x11 FP64 (B B^T + 0.1 I, seed 8), blocks [5, 6], 4 lanes x 3 rows per matrix",
        "ms_per_batch": ms, "inverses_per_s": count / (ms / 1e3), "kernel_ms": kms,
        "ms_per_batch_with_input_reset": ms_reset,
        "max_rho": float(rho.max()), "failed": int((st != 0).sum().item()), **eps11,
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
    # gaps between the graph's nodes: the kernels of one stream-ordered run
    # (no graph), each with its own event pair, against the graph replay
    refresh()
    torch.cuda.synchronize()
    bi.blockinv_trace_enable(True)
    st_e = bi.blockinv_invert_batched(ns, None, [t.data_ptr() for t in dst], ns, bi.F64, stream, stt.data_ptr())
    torch.cuda.synchronize()
    bi.blockinv_trace_enable(False)
    tr_e = bi.blockinv_trace_summary()
    kernel_sum = sum(v["ms"] for k, v in tr_e.items() if k.startswith("batched_step_"))
    launches_e = sum(v["launches"] for k, v in tr_e.items() if k.startswith("batched_step_"))
    bi.blockinv_batch_tuning_clear()
    ms = sum(per) / len(per)
    ms_default = sum(per_default) / len(per_default)
    flops = sum(2.0 * m ** 3 for m in ns)
    g = inputs.rng(66)
    rhos, eps, epsm = [], [], []
    import oracle
    for i in g.choice(len(mats), size=50, replace=False):
        Xi = dst[i].cpu().numpy()
        Ai = mats[i]
        rhos.append(np.linalg.norm(Ai @ Xi - np.eye(Ai.shape[0])) / (np.linalg.norm(Ai) * np.linalg.norm(Xi)))
        e = eps_vs_oracle(Xi, small_oracle(Ai, oracle.quarter_partition(Ai.shape[0])))
        eps.append(e["eps_vs_oracle"])
        epsm.append(e["eps_max_vs_oracle"])
    tfs = flops / (ms / 1e3) / 1e12
    out["uneven_2000"] = {
        "workload": "2000 FP64 matrices, n log-uniform in [8, 512], U[-1,1] + n I (seed 6); partitions and "
                    "Schur tiles from the autotuner",
        "ms_per_batch": ms, "inverses_per_s": len(mats) / (ms / 1e3), "value": tfs, "unit": "TFLOP/s",
        "latency_ms": percentiles(per), "max_rho_sampled": float(max(rhos)),
        "eps_vs_oracle_max_sampled": float(max(eps)), "eps_max_vs_oracle_max_sampled": float(max(epsm)),
        "eps_sample": "50 matrices (seed 66), oracle with four blocks of n/4 (the last n mod 4 one larger)",
        "failed": int((stt != 0).sum().item()),
        "launches_per_batch": tr["launches"] / args.steps,
        "graph_gap_analysis": {
            "eager_status": int(st_e), "eager_kernel_groups": launches_e,
            "sum_of_kernel_ms_eager": kernel_sum,
            "graph_ms": sum(per) / len(per),
            "note": "kernels of one stream-ordered run, each timed alone; their sum against one graph replay "
                    "bounds what removing the graph's inter-node gaps (one persistent launch) could save"},
        "default_partition_ms_per_batch": ms_default,
        "autotune": {"seconds": tune_s, "table": table},
        "roofline": {"bound": "alu", "kernel": "batched_grouped_f64 (graph)", "achieved": tfs,
                     "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS, "frac": tfs / FP64_PEAK_TFLOPS},
    }
    return out



def run_serving(args, bi, torch):
    """Poisson arrivals at 2000 req/s, sizes log-uniform in [5, 4096] (70%
    U[-1,1] + n I, 30% B B^T + 0.1 I), through a serving context with a
    120 GB budget and SERVE_SLOTS slots: mixed TF32 + refinement over the full window
    (60 s by default), and plain FP64 over a shorter one (it cannot keep up).
    Orders <= 512 are coalesced by the context into batch jobs on the FP64
    batched engine; larger ones run the single-matrix path of their mode with
    block sizes from the default partition. Latency counts from each request's
    scheduled arrival to the host seeing its completion."""
    from paper_2305_11103_gb300 import inputs
    rate = 2000.0
    # sizes quantised to 32 log-spaced orders; one pooled matrix per (order, kind)
    grid = np.unique(np.rint(np.exp(np.linspace(np.log(5), np.log(4096), 32))).astype(int))
    pool = {}

    def matrix(key):
        if key not in pool:
            n = int(grid[key[0]])
            if key[1] == 0:
                M = torch.from_numpy(inputs.diag_dominant_uniform(n, 7000 + n, shift=n)).cuda()
            else:
                B = torch.from_numpy(inputs.rng(8000 + n).standard_normal((n, n))).cuda()
                M = B @ B.T + 0.1 * torch.eye(n, dtype=torch.float64, device="cuda")
            pool[key] = M
        return pool[key]

    # block sizes from the autotuners on this stream's orders: the batch tuner
    # for the orders coalesced into FP64 batch jobs, the single-matrix tuner
    # per mode for the rest (one matrix per size class, its median order)
    tune = {}
    t0 = time.time()
    small = [int(v) for v in grid if 8 <= v <= 512]
    mix = np.repeat(small, 8).tolist()
    st = bi.blockinv_batch_tune(mix, 3, None)
    tune["batch_tune_status"] = int(st)
    large = [int(v) for v in grid if v > 512]
    for mode in ("f64", "tf32"):
        st = bi.blockinv_tune(large, mode, 2)
        tune[f"tune_status_{mode}"] = int(st)
        tune[f"blocks_{mode}"] = {f"{2 ** c}-{2 ** (c + 1) - 1}": bi.blockinv_tuning(mode, c)[1]
                                  for c in range(9, 13)}
    tune["batch_table"] = {}
    for c in range(3, 10):
        _, pc, tile = bi.blockinv_batch_tuning(c)
        if pc:
            tune["batch_table"][f"{2 ** c}-{2 ** (c + 1) - 1}"] = {"blocks": pc, "tile": tile}
    tune["seconds"] = time.time() - t0
    oracle_x = {}
    out = {"autotune": tune,
           "workload": f"Poisson {rate:.0f} req/s, n log-uniform in [5, 4096] quantised to {len(grid)} orders, "
                       f"70% U[-1,1]+nI / 30% B B^T+0.1I, seed 7; budget 120 GB, {SERVE_SLOTS} slots; orders <= 512 "
                       f"coalesced into FP64 batch jobs; at most {SERVE_INFLIGHT} requests in flight, later "
                       "arrivals wait at the client (latency from arrival)"}
    for mode, window in (("f64", args.serve_seconds_f64), ("tf32", args.serve_seconds)):
        arrivals = inputs.poisson_arrivals(rate, window, 7)
        nreq = len(arrivals)
        want = inputs.log_uniform_sizes(nreq, 5, 4096, 7)
        idx = np.abs(np.log(want)[:, None] - np.log(grid)[None, :]).argmin(axis=1)
        kinds = (inputs.rng(8).random(nreq) < 0.3).astype(int)
        keys = [(int(a), int(b)) for a, b in zip(idx, kinds)]
        for k in sorted(set(keys)):
            matrix(k)
        torch.cuda.synchronize()
        sample = set(inputs.rng(77).choice(nreq, size=min(nreq, 60), replace=False).tolist())
        ctx = bi.Context(0, 120 << 30, SERVE_SLOTS)
        cs = torch.cuda.Stream()
        util = UtilSampler()
        util.start()
        pending = {}
        lat, fin, statuses, used_modes = [], [], [], []
        kept = {}
        done = i = 0
        progress(f"serving {mode}: {nreq} requests over {window} s")
        t0 = time.perf_counter()
        # a request that never completes must not stall the benchmark: after
        # the window and a generous drain, the rest is reported as incomplete
        deadline = window + SERVE_DRAIN_S
        incomplete = 0
        while done < nreq:
            if time.perf_counter() - t0 > deadline:
                incomplete = nreq - done
                break
            now = time.perf_counter() - t0
            new = []
            with torch.cuda.stream(cs):
                # arrived requests are materialised (their matrix copied into a
                # buffer of their own) and submitted while fewer than
                # SERVE_INFLIGHT are in flight; the rest wait at the client as
                # descriptors, their latency still counted from arrival
                while i < nreq and arrivals[i] <= now and len(pending) + len(new) < SERVE_INFLIGHT:
                    new.append((i, pool[keys[i]].clone()))
                    i += 1
            if new:
                cs.synchronize()  # the copies are in place before the context's streams read them
                for ri, buf in new:
                    n = buf.shape[0]
                    st, t = ctx.submit(n, None, buf.data_ptr(), n, mode)
                    if st != bi.OK:
                        raise bi.BlockinvError(st, -1, "blockinv_submit")
                    pending[t] = (ri, buf)
            finished = ctx.poll_done()
            for t in finished:
                st, r = ctx.poll(t)
                ri, buf = pending.pop(t)
                tf = time.perf_counter() - t0
                lat.append(1e3 * (tf - arrivals[ri]))
                fin.append(arrivals[ri])
                statuses.append(st)
                used_modes.append(r.mode)
                if ri in sample:
                    kept[ri] = buf
                done += 1
            if not new and not finished:
                if i < nreq and not pending and arrivals[i] > time.perf_counter() - t0:
                    time.sleep(max(0.0, arrivals[i] - (time.perf_counter() - t0)))
                else:
                    time.sleep(0.0002)
        wall = time.perf_counter() - t0
        gpu_util = util.stop()
        if incomplete:
            progress(f"serving {mode}: {incomplete} requests incomplete at the deadline; context left open")
            stuck_contexts.append(ctx)  # closing it would wait for them
        else:
            ctx.close()
        flops = sum(2.0 * float(grid[k]) ** 3 for k in idx)
        # latency over the window: the requests arriving in its first and last thirds
        order = np.argsort(fin)
        third = max(1, len(order) // 3)
        lat_a = np.asarray(lat)
        early, late = lat_a[order[:third]], lat_a[order[-third:]]
        # the sampled requests against the oracle (cached per pooled matrix) and by rho on the GPU
        rhos, eps, epsm = [], [], []
        for r, b in sorted(kept.items()):
            M = pool[keys[r]]
            if keys[r] not in oracle_x:
                oracle_x[keys[r]] = small_oracle(M.cpu().numpy(), partition(M.shape[0], 256))
            rhos.append(bi.residual(M, b))
            e = eps_vs_oracle(b.cpu().numpy(), oracle_x[keys[r]])
            eps.append(e["eps_vs_oracle"])
            epsm.append(e["eps_max_vs_oracle"])
        out[mode] = {"window_s": window, "requests": nreq, "completed": done, "incomplete": incomplete, "wall_s": wall,
                     "throughput_req_s": done / wall, "offered_req_s": rate, "effective_tflops": flops / wall / 1e12,
                     "latency_ms": percentiles(lat),
                     "latency_p99_first_third_ms": float(np.percentile(early, 99)),
                     "latency_p99_last_third_ms": float(np.percentile(late, 99)),
                     "failed": sum(1 for s in statuses if s != bi.OK),
                     "served_fp64_batched_or_fp64": sum(1 for m in used_modes if m == bi.F64),
                     "gpu_utilization_pct": gpu_util,
                     "sampled_requests": len(kept),
                     "max_rho_sampled": float(max(rhos)) if rhos else None,
                     "eps_vs_oracle_max_sampled": float(max(eps)) if eps else None,
                     "eps_max_vs_oracle_max_sampled": float(max(epsm)) if epsm else None}
    out["eps_sample"] = ("60 requests (seed 77) per mode, each against the oracle on its pooled input "
                         "(blocks of 256, the last one the remainder)")
    return out


def f64_leg(args, bi, torch, stream, w, world, steps, warmup, orc, key):
    """A workload through the plain FP64 GPU path: ms per inversion, rho, the
    roofline of the dominant kernel (the FP64 Schur update, FP64 pipe) from a
    traced pass, and eps against the oracle's X (computed under `key`)."""
    n, sizes = w["n"], partition(w["n"], w["block"])
    A = make_matrix(n, w["sigma"], w["seed"])
    dA = torch.from_numpy(A).cuda()
    dX = torch.empty_like(dA)
    per, _, step = run_solves(bi, torch, stream, dA, dX, n, sizes, "f64", steps, warmup)
    ms, value = whole_job(sum(per) / len(per), 2.0 * n ** 3, world)
    rho = bi.residual(dA, dX)
    trace = trace_pass(bi, torch, step, min(3, steps))
    kname, kt = max(trace.items(), key=lambda kv: kv[1]["ms"])
    achieved = kt["flops"] / (kt["ms"] / 1e3) / 1e12
    traffic = ncu_traffic(kname, n)
    total = sum(v["ms"] for v in trace.values())
    out = {"workload": w["desc"], "n": n, "block": w["block"], "ms_per_step": ms, "value": value,
           "unit": "TFLOP/s", "inverses_per_s": world * 1e3 / ms, "latency_ms": percentiles(per), "rho": rho,
           "steps": steps, "warmup": warmup, "l2": l2_note(n),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": kname,
                        "peak_source": "FP64 unit counts: 2 DFMA/clk/SM x 2 x 152 SMs x 2.07 GHz "
                                       "(MEASURED_PEAKS.json has no FP64 figure)",
                        "algorithmic_flops_per_launch": kt["flops"] / kt["launches"],
                        "share_of_kernel_time": kt["ms"] / total if total else None},
           "kernels": trace, "gpu_launches_per_step": sum(v["launches"] for v in trace.values()) / min(3, steps)}
    X = dX.cpu().numpy() if orc else None
    del dA, dX
    torch.cuda.empty_cache()
    return out, A, X


def attach_eps(res, X, orc, key):
    """Add eps against the oracle's X for `key` to res (waits for it)."""
    if orc is None or X is None:
        return None
    got = orc.get(key)
    if got is None:
        res["eps_vs_oracle"] = None
        res["eps_note"] = f"oracle worker failed: {orc.error}"
        return None
    sec, thr, Xo = got
    res.update(eps_vs_oracle(X, Xo))
    return sec, thr, Xo


# ----------------------------------------------------------- our arm -------
def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    from paper_2305_11103_gb300 import blockinv as bi
    from paper_2305_11103_gb300 import build as libbuild
    if rank == 0:
        libbuild.build()
        import oracle
        oracle.build_oracle()
    barrier(world)
    bi.lib()
    w = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    use_oracle = rank == 0 and world == 1 and not args.no_oracle

    if w["kind"] == "f64":
        return run_ours_f64(args, bi, torch, stream, w, world, rank, local, use_oracle)

    n, sizes = w["n"], partition(w["n"], w["block"])
    flops = 2.0 * n ** 3
    # serving first: its host loop must not share the cores with the oracle
    serving = {} if args.no_serve else run_serving(args, bi, torch)
    progress("mixed legs")
    jobs = [(f"x{n}_s{seed}", n, w["block"], sig, seed) for seed, sig in w["legs"]]
    side = not args.no_side and n != 8192
    if side:
        jobs.append(("x8192_s2", 8192, 256, 1.5, 2))
    orc = OracleRuns(jobs) if use_oracle else None

    legs, host_X = {}, {}
    head = fp64 = e2e = clk = None
    head_A = None
    for li, (seed, sig) in enumerate(w["legs"]):
        A = make_matrix(n, sig, seed)
        dA = torch.from_numpy(A).to(dev)
        dX = torch.empty_like(dA)
        if li == 0:
            head_A = A
        del A
        for mode in w["modes"]:
            is_head = li == 0 and mode == w["modes"][0]
            if is_head:
                barrier(world)
                sampler = ClockSampler(local)
                sampler.start()
            per, infos, step = run_solves(bi, torch, stream, dA, dX, n, sizes, mode, args.steps, args.warmup)
            if is_head:
                clk = sampler.stop()
            ms, value = whole_job(sum(per) / len(per), flops, world)
            rep = mixed_report(n, per, infos[-1], bi.residual(dA, dX))
            rep.update({"ms_per_step": ms, "value": value, "sigma": sig, "seed": seed, "mode": mode})
            if is_head:
                nt = 3
                trace = trace_pass(bi, torch, step, nt)
                tensor, schur_rl, kt_total = mixed_rooflines(n, trace, infos[-1], nt, mode)
                launches = sum(v["launches"] for v in trace.values()) / nt
                head = dict(rep, trace=trace, tensor=tensor, schur_rl=schur_rl, kt_total=kt_total, launches=launches,
                            nt=nt)
            if orc:
                host_X[(seed, mode)] = dX.cpu().numpy()
            legs[f"{mode}_sigma{sig}"] = rep
        if li == 0 and not args.no_fp64_path:
            per, _, _ = run_solves(bi, torch, stream, dA, dX, n, sizes, "f64", args.fp64_steps, 1)
            ms, value = whole_job(sum(per) / len(per), flops, world)
            fp64 = {"ms_per_step": ms, "value": value, "unit": "TFLOP/s", "latency_ms": percentiles(per),
                    "steps": args.fp64_steps, "warmup": 1, "rho": bi.residual(dA, dX), "sigma": sig, "seed": seed}
            if orc:
                host_X[(seed, "f64")] = dX.cpu().numpy()
        del dA, dX
        torch.cuda.empty_cache()
    if fp64:
        for rep in legs.values():
            rep["speedup_vs_fp64_path"] = fp64["ms_per_step"] / rep["ms_per_step"]

    if not args.no_e2e:
        mode = w["modes"][0]
        hA = torch.from_numpy(head_A).pin_memory()
        hX = torch.empty_like(hA).pin_memory()
        tot = 0.0
        for it in range(args.warmup + args.steps):
            hX.copy_(hA)
            torch.cuda.synchronize()
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
               "api": f"blockinv_invert_host mode {mode} (pinned host buffer in and out, copies inside the "
                      "timed region; stream-ordered refinement)"}
        del hA, hX
    del head_A

    side_legs = {}
    if side:
        progress("side legs: FP64 8192 and 256")
        f64_steps, f64_warm = min(args.steps, 5), min(args.warmup, 2)
        res, _, X8 = f64_leg(args, bi, torch, stream, WORKLOADS["f64_8192"], world, f64_steps, f64_warm, orc,
                             "x8192_s2")
        side_legs["f64_8192"] = (res, X8)
        side_legs["f64_256"] = (run_cfg1(args, bi, torch), None)
    progress("batched legs")
    batched = {} if args.no_batched else run_batched(args, bi, torch, stream)
    progress("waiting for the oracle")

    # eps against the oracle for every large result, as its inverses arrive
    cpu = None
    if orc:
        for seed, sig in w["legs"]:
            key = f"x{n}_s{seed}"
            got = orc.get(key)
            for (s_, mode), X in list(host_X.items()):
                if s_ != seed:
                    continue
                target = fp64 if mode == "f64" else legs[f"{mode}_sigma{sig}"]
                if got is None:
                    target["eps_vs_oracle"] = None
                    target["eps_note"] = f"oracle worker failed: {orc.error}"
                else:
                    target.update(eps_vs_oracle(X, got[2]))
                del host_X[(s_, mode)]
            if got is not None:
                dXo = torch.from_numpy(np.array(got[2])).to(dev)
                dAo = torch.from_numpy(make_matrix(n, sig, seed)).to(dev)
                legs[f"{w['modes'][0]}_sigma{sig}"]["rho_of_oracle_X"] = bi.residual(dAo, dXo)
                del dXo, dAo
                torch.cuda.empty_cache()
                if seed == w["legs"][0][0]:
                    sec, thr = got[0], got[1]
                    cpu = {"value": flops / sec / 1e12, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
                           "sample": f"one inversion of the headline matrix itself (order {n}, seed {seed}, "
                                     f"{n // w['block']} blocks of {w['block']}), {sec:.1f} s, run with {thr} "
                                     "threads in a spawned process beside the GPU legs"}
            orc.drop(key)
        if side:
            res, X8 = side_legs["f64_8192"]
            attach_eps(res, X8, orc, "x8192_s2")
            orc.drop("x8192_s2")
        orc.close()
    for k, (res, _) in side_legs.items():
        side_legs[k] = res

    if rank == 0:
        head_key = f"{w['modes'][0]}_sigma{w['legs'][0][1]}"
        h = legs[head_key]
        out = {
            "metric": METRIC, "value": h["value"], "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"{w['modes'][0]}+f64", "data": "synthetic",
            "config": {"workload": w["desc"], "n": n, "block": w["block"], "mode": w["modes"][0],
                       "sigma": w["legs"][0][1], "seed": w["legs"][0][0], "l2": l2_note(n),
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "inverses_per_s": world * 1e3 / h["ms_per_step"], "latency_ms": h["latency_ms"],
            "rho": h["rho_refinement"], "rho_fp64_check": h["rho_fp64_check"], "rho_gate": RHO_GATE,
            "refine_iters": h["refine_iters"],
            "eps_vs_oracle": h.get("eps_vs_oracle"), "eps_max_vs_oracle": h.get("eps_max_vs_oracle"),
            "speedup_vs_fp64_path": h.get("speedup_vs_fp64_path"),
            "roofline": head["tensor"], "roofline_schur_update": head["schur_rl"],
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": int(round(head["launches"] * args.steps)),
            "kernels": head["trace"],
            "kernels_pass": f"{head['nt']} more steps, one event pair per launch (no overlap)",
            "kernels_pass_ms_per_step": head["kt_total"] / head["nt"],
            "mixed": legs, "fp64_path": fp64,
            "side": side_legs, "batched": batched, "serving": serving,
        }
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ours_f64(args, bi, torch, stream, w, world, rank, local, use_oracle):
    """An FP64 workload as the headline (profiling runs): the plain FP64 GPU
    path, its roofline, eps against the oracle and the end-to-end leg."""
    n = w["n"]
    key = f"x{n}_s{w['seed']}"
    orc = OracleRuns([(key, n, w["block"], w["sigma"], w["seed"])]) if use_oracle else None
    barrier(world)
    sampler = ClockSampler(local)
    sampler.start()
    res, A, X = f64_leg(args, bi, torch, stream, w, world, args.steps, args.warmup, orc, key)
    clk = sampler.stop()
    e2e = None
    if not args.no_e2e:
        sizes = partition(n, w["block"])
        hA = torch.from_numpy(A).pin_memory()
        hX = torch.empty_like(hA).pin_memory()
        tot = 0.0
        for it in range(args.warmup + args.steps):
            hX.copy_(hA)
            t0 = time.perf_counter()
            st = bi.blockinv_invert_host(n, sizes, hX.data_ptr(), n, "f64", stream)
            t1 = time.perf_counter()
            if st != bi.OK:
                raise bi.BlockinvError(st, -1, "blockinv_invert_host")
            if it >= args.warmup:
                tot += t1 - t0
        e2e_ms, e2e_value = whole_job(tot / args.steps * 1e3, 2.0 * n ** 3, world)
        e2e = {"value": e2e_value, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 8,
               "api": "blockinv_invert_host (pinned host buffer, copies inside the timed region)"}
    cpu = None
    if orc:
        got = attach_eps(res, X, orc, key)
        if got:
            sec, thr = got[0], got[1]
            cpu = {"value": 2.0 * n ** 3 / sec / 1e12, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
                   "sample": f"one inversion of the workload matrix itself (order {n}), {sec:.2f} s, {thr} threads"}
        orc.close()
    if rank == 0:
        out = {"metric": METRIC, "value": res["value"], "unit": "TFLOP/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic",
               "config": {"workload": w["desc"], "n": n, "block": w["block"], "mode": "f64", "l2": l2_note(n),
                          "parallelism": f"replicas{world}" if world > 1 else "single"},
               "inverses_per_s": res["inverses_per_s"], "latency_ms": res["latency_ms"], "rho": res["rho"],
               "rho_gate": RHO_GATE, "eps_vs_oracle": res.get("eps_vs_oracle"),
               "eps_max_vs_oracle": res.get("eps_max_vs_oracle"),
               "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": int(round(res["gpu_launches_per_step"] * args.steps)), "kernels": res["kernels"]}
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
    import oracle
    oracle.build_oracle()
    if w["kind"] == "mixed":
        seed, sigma = w["legs"][0]
        cfg = {"workload": w["desc"], "n": w["n"], "block": w["block"], "mode": w["modes"][0], "sigma": sigma,
               "seed": seed, "l2": l2_note(w["n"])}
    else:
        seed, sigma = w["seed"], w["sigma"]
        cfg = {"workload": w["desc"], "n": w["n"], "block": w["block"], "mode": "f64", "l2": l2_note(w["n"])}
    n = min(w["n"], CPU_SAMPLE_N)
    for _ in range(args.warmup):
        time_oracle(n, w["block"], sigma, seed)
    tot, cores = 0.0, 1
    for _ in range(args.steps):
        sec, cores = time_oracle(n, w["block"], sigma, seed)
        tot += sec
    sec = tot / args.steps
    value = 2.0 * n ** 3 / sec / 1e12
    sample = (f"one FP64 inversion per step at order {n} ({n // w['block']} blocks of {w['block']}, the same "
              f"distribution and seed), scaled as 2n^3/t")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    args = parse()
    if args.probe_peaks:
        probe_peaks()
    elif args.profile_solves or args.profile_batch_runs:
        profile_run(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if stuck_contexts:  # their worker threads may never finish: leave without waiting for them
        sys.stdout.flush()
        sys.stderr.flush()
        os._exit(0)


if __name__ == "__main__":
    main()
