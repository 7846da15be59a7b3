"""ctypes marshalling for the C oracle (``blockinv_oracle.c``).

Test infrastructure: no arithmetic of the method happens here, only argument
checks, array layout and the gcc build. Status codes follow the C file:
0 success, -1 bad argument, -2 singular pivot block, -4 out of memory.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "blockinv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs = {}

_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


class OracleError(RuntimeError):
    def __init__(self, status, failing_block=-1):
        super().__init__(f"oracle status {status} (failing block {failing_block})")
        self.status = status
        self.failing_block = failing_block


def _so_path(mutant):
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build_oracle(mutant=0, openmp=True, force=False):
    """Compile the oracle with gcc (-O2 -ffp-contract=off). Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _so_path(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared",
           "-fPIC", f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", out + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def load(mutant=0):
    with _lock:
        if mutant in _libs:
            return _libs[mutant]
        lib = ctypes.CDLL(build_oracle(mutant))
        lib.oracle_gj_inverse.argtypes = [ctypes.c_int, _DP, ctypes.c_long, _DP, ctypes.c_long]
        lib.oracle_small_inverse.argtypes = [ctypes.c_int, _DP, ctypes.c_long, _DP, ctypes.c_long]
        lib.oracle_block_inverse.argtypes = [ctypes.c_int, ctypes.c_int, _IP, _DP, ctypes.c_long,
                                             _DP, ctypes.c_long, _IP]
        lib.oracle_paper_partition.argtypes = [ctypes.c_int, _IP, ctypes.c_int]
        lib.oracle_quarter_partition.argtypes = [ctypes.c_int, _IP]
        lib.oracle_residual.argtypes = [ctypes.c_int, _DP, ctypes.c_long, _DP, ctypes.c_long]
        lib.oracle_residual.restype = ctypes.c_double
        lib.oracle_ns_step.argtypes = [ctypes.c_int, _DP, ctypes.c_long, _DP, ctypes.c_long,
                                       _DP, ctypes.c_long]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_mutant.restype = ctypes.c_int
        assert lib.oracle_mutant() == mutant
        _libs[mutant] = lib
        return lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.ndim == 2 and a.shape[0] == a.shape[1]
    return a


def _ptr(a):
    return a.ctypes.data_as(_DP)


def set_threads(t):
    load().oracle_set_threads(int(t))


def max_threads():
    return int(load().oracle_max_threads())


def gj_inverse(M, mutant=0):
    M = _f64(M)
    m = M.shape[0]
    out = np.empty_like(M)
    st = load(mutant).oracle_gj_inverse(m, _ptr(M), m, _ptr(out), m)
    if st != 0:
        raise OracleError(st)
    return out


def small_inverse(M, mutant=0):
    M = _f64(M)
    m = M.shape[0]
    out = np.empty_like(M)
    st = load(mutant).oracle_small_inverse(m, _ptr(M), m, _ptr(out), m)
    if st != 0:
        raise OracleError(st)
    return out


def block_inverse(A, sizes, mutant=0):
    """A^-1 by Eq. (a) applied recursively over the diagonal blocks `sizes`."""
    A = _f64(A)
    n = A.shape[0]
    s = np.ascontiguousarray(sizes, dtype=np.int32)
    X = np.empty_like(A)
    fb = ctypes.c_int(-1)
    st = load(mutant).oracle_block_inverse(n, len(s), s.ctypes.data_as(_IP), _ptr(A), n,
                                           _ptr(X), n, ctypes.byref(fb))
    if st != 0:
        raise OracleError(st, fb.value)
    return X


def paper_partition(m, mutant=0):
    buf = np.zeros(max(1, m), dtype=np.int32)
    k = load(mutant).oracle_paper_partition(int(m), buf.ctypes.data_as(_IP), len(buf))
    if k < 0:
        raise OracleError(k)
    return [int(v) for v in buf[:k]]


def quarter_partition(m, mutant=0):
    buf = np.zeros(4, dtype=np.int32)
    k = load(mutant).oracle_quarter_partition(int(m), buf.ctypes.data_as(_IP))
    if k < 0:
        raise OracleError(k)
    return [int(v) for v in buf[:k]]


def residual(A, X, mutant=0):
    A = _f64(A)
    X = _f64(X)
    return float(load(mutant).oracle_residual(A.shape[0], _ptr(A), A.shape[0], _ptr(X), X.shape[0]))


def ns_step(A, X, mutant=0):
    A = _f64(A)
    X = _f64(X)
    n = A.shape[0]
    Xn = np.empty_like(X)
    st = load(mutant).oracle_ns_step(n, _ptr(A), n, _ptr(X), n, _ptr(Xn), n)
    if st != 0:
        raise OracleError(st)
    return Xn
