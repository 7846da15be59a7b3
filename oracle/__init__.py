"""CPU FP64 oracle for blockwise (Schur-complement) matrix inversion.

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the CPU-baseline leg of the benchmark, never by the GPU library. The
arithmetic lives in ``blockinv_oracle.c`` (plain C, FP64); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from .oracle import (  # noqa: F401
    build_oracle,
    load,
    gj_inverse,
    small_inverse,
    block_inverse,
    paper_partition,
    quarter_partition,
    residual,
    ns_step,
    set_threads,
    max_threads,
)
