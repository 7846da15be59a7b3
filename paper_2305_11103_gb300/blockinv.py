"""Thin ctypes binding of libblockinv.so (include/blockinv.h), same entry-point names.

Argument marshalling only: every step of the inversion runs in the library's
CUDA kernels. PyTorch tensors are accepted for convenience (device memory and
streams); the C ABI itself sees plain pointers and sizes. The library must be
built first (``__graft_entry__.build()``); loading fails loudly otherwise, and
there is no CPU fallback.
"""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libblockinv.so")

F64, MIXED_TF32, MIXED_BF16 = 0, 1, 2
MODES = {"f64": F64, "tf32": MIXED_TF32, "bf16": MIXED_BF16}

OK, PENDING = 0, 1
ERR_INVALID, ERR_SINGULAR, ERR_NONFINITE, ERR_NOMEM = -1, -2, -3, -4
ERR_BUDGET, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA = -5, -6, -7, -8
ERR_CANCELLED = -9
SUBMIT_HOST = 1

_lock = threading.Lock()
_lib = None

_i64, _i32, _int, _vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); the declarations of include/blockinv.h
SIGNATURES = {
    "blockinv_invert": (_int, [_i64, _i32, _i32p, _vp, _i64, _int, _vp]),
    "blockinv_invert_async": (_int, [_i64, _i32, _i32p, _vp, _i64, _int, _vp, _vp]),
    "blockinv_invert_host": (_int, [_i64, _i32, _i32p, _vp, _i64, _int, _vp]),
    "blockinv_invert_batched_small": (_int, [_i64, _i32, _vp, _vp, _vp]),
    "blockinv_invert_batched_fixed": (_int, [_i64, _i32, _i32, _i32p, _i32, _vp, _vp, _vp]),
    "blockinv_invert_batched": (_int, [_i32, _i32p, _i32p, _i32p, _vp, ctypes.POINTER(ctypes.c_int64), _int, _vp,
                                        _vp]),
    "blockinv_batch_plan_create": (_int, [_i32, _i32p, _i32p, _i32p, _vp, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "blockinv_batch_plan_run": (_int, [_vp, _vp, _vp]),
    "blockinv_batch_plan_destroy": (_int, [_vp]),
    "blockinv_invert_steps": (_int, [_i64, _i32, _i32p, _vp, _i64, _i32, _i32, _vp]),
    "blockinv_checkpoint_write": (_int, [ctypes.c_char_p, _i64, _i32, _i32p, _vp, _i64, _i32, _vp]),
    "blockinv_checkpoint_read": (_int, [ctypes.c_char_p, _i64, _i32, _i32p, _vp, _i64, _i32p, _vp]),
    "blockinv_batch_tune": (_int, [_i32, _i32p, _i32, _vp]),
    "blockinv_tune": (_int, [_i32, _i32p, _i32, _i32, _vp]),
    "blockinv_tuning": (_int, [_i32, _i32, _i32p]),
    "blockinv_tuning_set": (_int, [_i32, _i32, _i32]),
    "blockinv_tuning_clear": (_int, []),
    "blockinv_batch_tuning": (_int, [_i32, _i32p, _i32p]),
    "blockinv_batch_tuning_set": (_int, [_i32, _i32, _i32]),
    "blockinv_batch_tuning_clear": (_int, []),
    "blockinv_batch_tuning_save": (_int, [ctypes.c_char_p]),
    "blockinv_batch_tuning_load": (_int, [ctypes.c_char_p]),
    "blockinv_ctx_create": (_int, [_int, ctypes.c_size_t, _int, ctypes.POINTER(ctypes.c_void_p)]),
    "blockinv_submit": (_int, [_vp, _i64, _i32, _i32p, _vp, _i64, _int, _int, ctypes.POINTER(ctypes.c_uint64)]),
    "blockinv_poll": (_int, [_vp, ctypes.c_uint64, _vp]),
    "blockinv_wait": (_int, [_vp, ctypes.c_uint64, _vp]),
    "blockinv_cancel": (_int, [_vp, ctypes.c_uint64]),
    "blockinv_ctx_stats": (_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_size_t)]),
    "blockinv_ctx_destroy": (_int, [_vp]),
    "blockinv_poll_done": (_int, [_vp, ctypes.POINTER(ctypes.c_uint64), _i32, ctypes.POINTER(ctypes.c_int32)]),
    "blockinv_invert_noalloc": (_int, [_i64, _i32, _i32p, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_int64)]),
    "blockinv_residual": (_int, [_i64, _vp, _i64, _vp, _i64, ctypes.POINTER(ctypes.c_double), _vp]),
    "blockinv_residual_tc": (_int, [_i64, _vp, _i64, _vp, _i64, _vp, _i64, _int, ctypes.POINTER(ctypes.c_double),
                                     _vp]),
    "blockinv_status_str": (ctypes.c_char_p, [_int]),
    "blockinv_last_error_detail": (_int, [ctypes.POINTER(ctypes.c_int64)]),
    "blockinv_last_cuda_error": (_int, [ctypes.POINTER(ctypes.c_char_p)]),
    "blockinv_version": (_int, []),
    "blockinv_struct_sizes": (_int, [_i32p, _i32p, _i32p]),
    "blockinv_release_memory": (_int, []),
    "blockinv_invert_ex": (_int, [_i64, _i32, _i32p, _vp, _i64, _int, _vp, _vp, _vp]),
    "blockinv_diag_gemm": (_int, [_int, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "blockinv_diag_recip64": (_int, [_vp, _vp, _i64, _vp]),
    "blockinv_diag_wait_timeout": (_int, [_i64, _vp]),
    "blockinv_trace_enable": (_int, [_int]),
    "blockinv_trace_summary": (ctypes.c_int64, [ctypes.c_char_p, ctypes.c_int64]),
}


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_refine", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("split", ctypes.c_int32), ("pivot_f64", ctypes.c_int32), ("pivot_order", ctypes.c_int32),
                ("singular_fallback", ctypes.c_int32), ("lookahead", ctypes.c_int32), ("fuse", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("refine_iters", ctypes.c_int32), ("failing_block", ctypes.c_int64),
                ("rho", ctypes.c_double), ("rho_initial", ctypes.c_double), ("used_fallback", ctypes.c_int32),
                ("fp64_pivots", ctypes.c_int32), ("partition_fallback", ctypes.c_int32),
                ("blocks_used", ctypes.c_int32), ("incremental_residuals", ctypes.c_int32),
                ("incremental_groups", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BlockinvError(RuntimeError):
    def __init__(self, status, failing_block=-1, what=""):
        name = lib().blockinv_status_str(status).decode() if _lib else str(status)
        super().__init__(f"{what}: {name} (status {status}, block {failing_block})")
        self.status = status
        self.failing_block = failing_block


def lib():
    """Load libblockinv.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
        return _lib


def _sizes(block_sizes):
    if block_sizes is None:
        return 0, None, None
    arr = (ctypes.c_int32 * len(block_sizes))(*[int(v) for v in block_sizes])
    return len(block_sizes), arr, arr


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _mode(mode):
    return MODES[mode] if isinstance(mode, str) else int(mode)


# ------------------------------------------------------------- raw C ABI ---
def blockinv_invert(n, block_sizes, A_ptr, lda, mode=F64, stream=None):
    p, arr, _ = _sizes(block_sizes)
    return lib().blockinv_invert(n, p, arr, A_ptr, lda, _mode(mode), _stream_ptr(stream))


def blockinv_invert_async(n, block_sizes, A_ptr, lda, mode, stream, status_dev_ptr):
    p, arr, _ = _sizes(block_sizes)
    return lib().blockinv_invert_async(n, p, arr, A_ptr, lda, _mode(mode), _stream_ptr(stream),
                                       status_dev_ptr)


def blockinv_invert_ex(n, block_sizes, A_ptr, lda, mode=F64, stream=None, tol=0.0, max_refine=-1, fallback=1,
                       split=0, pivot_f64=0, pivot_order=0, singular_fallback=0, lookahead=0, fuse=0):
    """Returns (status, Info)."""
    p, arr, _ = _sizes(block_sizes)
    opt = Options(tol=tol, max_refine=max_refine, fallback=fallback, split=split, pivot_f64=pivot_f64,
                  pivot_order=pivot_order, singular_fallback=singular_fallback, lookahead=lookahead, fuse=fuse)
    info = Info()
    st = lib().blockinv_invert_ex(n, p, arr, A_ptr, lda, _mode(mode), _stream_ptr(stream), ctypes.byref(opt),
                                  ctypes.byref(info))
    return st, info


def blockinv_last_cuda_error():
    """(code, name) of the last CUDA runtime failure the library reported as
    ERR_CUDA / ERR_NOMEM (0, "cudaSuccess" if none); clears it."""
    name = ctypes.c_char_p()
    code = lib().blockinv_last_cuda_error(ctypes.byref(name))
    return code, (name.value.decode() if name.value else "")


def blockinv_diag_gemm(kind, M, N, K, A_ptr, lda, B_ptr, ldb, C_ptr, ldc, stream=None):
    return lib().blockinv_diag_gemm(kind, M, N, K, A_ptr, lda, B_ptr, ldb, C_ptr, ldc, _stream_ptr(stream))


def blockinv_diag_recip64(v_ptr, out_ptr, count, stream=None):
    return lib().blockinv_diag_recip64(v_ptr, out_ptr, count, _stream_ptr(stream))


def blockinv_diag_wait_timeout(limit_ns, stream=None):
    return lib().blockinv_diag_wait_timeout(limit_ns, _stream_ptr(stream))


def blockinv_invert_batched_small(count, n, A_ptr, status_ptr=None, stream=None):
    return lib().blockinv_invert_batched_small(count, n, A_ptr, status_ptr, _stream_ptr(stream))


BATCH_SPD = 1


def blockinv_invert_batched_fixed(count, n, block_sizes, A_ptr, flags=0, status_ptr=None, stream=None):
    p, arr, _ = _sizes(block_sizes)
    return lib().blockinv_invert_batched_fixed(count, n, p, arr, flags, A_ptr, status_ptr, _stream_ptr(stream))


def _batch_args(ns, partitions, A_ptrs, ldas):
    count = len(ns)
    n_arr = (ctypes.c_int32 * count)(*ns)
    if partitions is None:
        p_arr, s_arr = None, None
    else:
        p_arr = (ctypes.c_int32 * count)(*[len(q) for q in partitions])
        flat = [int(v) for q in partitions for v in q]
        s_arr = (ctypes.c_int32 * len(flat))(*flat)
    a_arr = (ctypes.c_void_p * count)(*A_ptrs)
    l_arr = (ctypes.c_int64 * count)(*ldas)
    return count, n_arr, p_arr, s_arr, a_arr, l_arr


def blockinv_invert_batched(ns, partitions, A_ptrs, ldas, mode=F64, stream=None, status_ptr=None):
    count, n_arr, p_arr, s_arr, a_arr, l_arr = _batch_args(ns, partitions, A_ptrs, ldas)
    return lib().blockinv_invert_batched(count, n_arr, p_arr, s_arr, a_arr, l_arr, _mode(mode),
                                         _stream_ptr(stream), status_ptr)


def blockinv_invert_steps(n, block_sizes, A_ptr, lda, k0, k1, stream=None):
    p, arr, _ = _sizes(block_sizes)
    return lib().blockinv_invert_steps(n, p, arr, A_ptr, lda, k0, k1, _stream_ptr(stream))


def blockinv_checkpoint_write(path, n, block_sizes, A_ptr, lda, k_done, stream=None):
    p, arr, _ = _sizes(block_sizes)
    return lib().blockinv_checkpoint_write(str(path).encode(), n, p, arr, A_ptr, lda, k_done, _stream_ptr(stream))


def blockinv_checkpoint_read(path, n, block_sizes, A_ptr, lda, stream=None):
    """(status, k_done)."""
    p, arr, _ = _sizes(block_sizes)
    k = ctypes.c_int32(-1)
    st = lib().blockinv_checkpoint_read(str(path).encode(), n, p, arr, A_ptr, lda, ctypes.byref(k),
                                        _stream_ptr(stream))
    return st, k.value


def blockinv_batch_tune(ns, reps=3, stream=None):
    n_arr = (ctypes.c_int32 * len(ns))(*ns)
    return lib().blockinv_batch_tune(len(ns), n_arr, reps, _stream_ptr(stream))


def blockinv_tune(ns, mode=F64, reps=3, stream=None):
    arr = (ctypes.c_int32 * len(ns))(*[int(v) for v in ns])
    return lib().blockinv_tune(len(ns), arr, _mode(mode), reps, _stream_ptr(stream))


def blockinv_tuning(mode, size_class):
    """(status, block) of one (mode, size class) entry (block 0: not tuned)."""
    b = ctypes.c_int32(0)
    st = lib().blockinv_tuning(_mode(mode), size_class, ctypes.byref(b))
    return st, b.value


def blockinv_tuning_set(mode, size_class, block):
    return lib().blockinv_tuning_set(_mode(mode), size_class, block)


def blockinv_tuning_clear():
    return lib().blockinv_tuning_clear()


def blockinv_batch_tuning(size_class):
    """(status, nblocks, tile) of one size class (nblocks 0: not tuned)."""
    p, t = ctypes.c_int32(0), ctypes.c_int32(0)
    st = lib().blockinv_batch_tuning(size_class, ctypes.byref(p), ctypes.byref(t))
    return st, p.value, t.value


def blockinv_batch_tuning_set(size_class, nblocks, tile):
    return lib().blockinv_batch_tuning_set(size_class, nblocks, tile)


def blockinv_batch_tuning_clear():
    return lib().blockinv_batch_tuning_clear()


def blockinv_batch_tuning_save(path):
    return lib().blockinv_batch_tuning_save(str(path).encode())


def blockinv_batch_tuning_load(path):
    return lib().blockinv_batch_tuning_load(str(path).encode())


class BatchPlan:
    """A reusable batch plan (graph-replayed grouped launches)."""

    def __init__(self, ns, partitions, A_ptrs, ldas):
        count, n_arr, p_arr, s_arr, a_arr, l_arr = _batch_args(ns, partitions, A_ptrs, ldas)
        self.handle = ctypes.c_void_p()
        st = lib().blockinv_batch_plan_create(count, n_arr, p_arr, s_arr, a_arr, l_arr, ctypes.byref(self.handle))
        if st != OK:
            raise BlockinvError(st, -1, "blockinv_batch_plan_create")

    def run(self, stream=None, status_ptr=None):
        return lib().blockinv_batch_plan_run(self.handle, _stream_ptr(stream), status_ptr)

    def close(self):
        if self.handle:
            lib().blockinv_batch_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("mode", ctypes.c_int32), ("n", ctypes.c_int64),
                ("refine_iters", ctypes.c_int32), ("used_fallback", ctypes.c_int32), ("rho", ctypes.c_double),
                ("t_queue_ms", ctypes.c_double), ("t_device_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Context:
    """Serving context: submit / poll / wait / cancel (see include/blockinv.h)."""

    def __init__(self, device=0, hbm_budget_bytes=8 << 30, max_slots=8):
        self.handle = ctypes.c_void_p()
        st = lib().blockinv_ctx_create(device, hbm_budget_bytes, max_slots, ctypes.byref(self.handle))
        if st != OK:
            raise BlockinvError(st, -1, "blockinv_ctx_create")

    def submit(self, n, block_sizes, A_ptr, lda, mode=F64, flags=0):
        p, arr, _ = _sizes(block_sizes)
        t = ctypes.c_uint64(0)
        st = lib().blockinv_submit(self.handle, n, p, arr, A_ptr, lda, _mode(mode), flags, ctypes.byref(t))
        return st, t.value

    def poll(self, ticket):
        r = Result()
        st = lib().blockinv_poll(self.handle, ticket, ctypes.byref(r))
        return st, r

    def poll_done(self, max_tickets=4096):
        """Tickets of requests finished since the last call (results still taken with poll)."""
        buf = (ctypes.c_uint64 * max_tickets)()
        k = ctypes.c_int32(0)
        st = lib().blockinv_poll_done(self.handle, buf, max_tickets, ctypes.byref(k))
        if st != OK:
            raise BlockinvError(st, -1, "blockinv_poll_done")
        return list(buf[:k.value])

    def wait(self, ticket):
        r = Result()
        st = lib().blockinv_wait(self.handle, ticket, ctypes.byref(r))
        return st, r

    def cancel(self, ticket):
        return lib().blockinv_cancel(self.handle, ticket)

    def stats(self):
        q, r, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        lib().blockinv_ctx_stats(self.handle, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b))
        return q.value, r.value, b.value

    def close(self):
        if self.handle:
            lib().blockinv_ctx_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def blockinv_invert_noalloc(n, block_sizes, A_ptr, lda, stream=None):
    """FP64 inversion without device allocation (n <= 2048, blocks <= 256).
    Returns (status, failing_block)."""
    p, arr, _ = _sizes(block_sizes)
    fb = ctypes.c_int64(-1)
    st = lib().blockinv_invert_noalloc(n, p, arr, A_ptr, lda, _stream_ptr(stream), ctypes.byref(fb))
    return st, fb.value


def blockinv_invert_host(n, block_sizes, A_host_ptr, lda, mode=F64, stream=None):
    p, arr, _ = _sizes(block_sizes)
    return lib().blockinv_invert_host(n, p, arr, A_host_ptr, lda, _mode(mode), _stream_ptr(stream))


def blockinv_residual(n, A_ptr, lda, X_ptr, ldx, stream=None):
    rho = ctypes.c_double(0.0)
    st = lib().blockinv_residual(n, A_ptr, lda, X_ptr, ldx, ctypes.byref(rho), _stream_ptr(stream))
    return st, rho.value


def blockinv_residual_tc(n, A_ptr, lda, X_ptr, ldx, E_ptr=None, lde=0, slices=0, stream=None):
    rho = ctypes.c_double(0.0)
    st = lib().blockinv_residual_tc(n, A_ptr, lda, X_ptr, ldx, E_ptr, lde, slices, ctypes.byref(rho),
                                    _stream_ptr(stream))
    return st, rho.value


def blockinv_status_str(status):
    return lib().blockinv_status_str(status).decode()


def blockinv_last_error_detail():
    blk = ctypes.c_int64(-1)
    st = lib().blockinv_last_error_detail(ctypes.byref(blk))
    return st, blk.value


def blockinv_version():
    return lib().blockinv_version()


def blockinv_struct_sizes():
    """(sizeof blockinv_options, blockinv_info, blockinv_result) in the library."""
    o, i, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    lib().blockinv_struct_sizes(ctypes.byref(o), ctypes.byref(i), ctypes.byref(r))
    return o.value, i.value, r.value


def blockinv_trace_enable(on):
    return lib().blockinv_trace_enable(1 if on else 0)


def blockinv_trace_summary():
    """Per-kernel {launches, ms, flops, bytes} recorded since tracing was enabled."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    need = lib().blockinv_trace_summary(buf, len(buf))
    if need > len(buf):
        raise RuntimeError("trace summary truncated")
    return json.loads(buf.value.decode())


# ---------------------------------------------------- tensor conveniences ---
def _check_matrix(t):
    import torch
    if t.dtype != torch.float64 or t.dim() != 2 or t.shape[0] != t.shape[1] or t.stride(1) != 1:
        raise ValueError("expected a square float64 matrix with unit column stride")


def invert_(A, block_sizes=None, mode="f64", stream=None):
    """Invert the square float64 CUDA tensor A in place; raises BlockinvError."""
    _check_matrix(A)
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor (use invert_host_ for host memory)")
    n = A.shape[0]
    st = blockinv_invert(n, block_sizes, A.data_ptr(), A.stride(0), mode, stream)
    if st != OK:
        raise BlockinvError(st, blockinv_last_error_detail()[1], "blockinv_invert")
    return A


def invert_host_(A, block_sizes=None, mode="f64", stream=None):
    """Invert a host float64 matrix (torch CPU tensor, pinned or not) in place via the GPU."""
    _check_matrix(A)
    n = A.shape[0]
    st = blockinv_invert_host(n, block_sizes, A.data_ptr(), A.stride(0), mode, stream)
    if st != OK:
        raise BlockinvError(st, blockinv_last_error_detail()[1], "blockinv_invert_host")
    return A


def residual(A, X, stream=None):
    """rho = ||A X - I||_F / (||A||_F ||X||_F) on the GPU (float64 CUDA tensors)."""
    _check_matrix(A)
    _check_matrix(X)
    st, rho = blockinv_residual(A.shape[0], A.data_ptr(), A.stride(0), X.data_ptr(), X.stride(0), stream)
    if st != OK:
        raise BlockinvError(st, -1, "blockinv_residual")
    return rho
