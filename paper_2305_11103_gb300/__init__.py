"""GB300-native blockwise (Schur-complement) matrix inversion.

The compute path lives in ``libblockinv.so`` (hand-written sm_103a CUDA behind
a C ABI, declared in ``include/blockinv.h``). ``paper_2305_11103_gb300.blockinv``
is the thin ctypes binding with the same entry-point names. Importing this
package does not load the library; the binding does, and raises if it is
missing.
"""
__all__ = ["blockinv", "inputs", "build"]
