"""The C ABI: libblockinv.so builds, loads, and exports every symbol that
include/blockinv.h declares. No GPU work is done here: the calls below fail
argument validation on the host before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2305_11103_gb300 import blockinv
from paper_2305_11103_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(blockinv_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return blockinv.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "blockinv_invert" in names and "blockinv_residual" in names
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (blockinv_\w+)", out))
    missing = names - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for n in names:
        getattr(lib, n)


def test_binding_matches_header():
    assert set(blockinv.SIGNATURES) <= declared_symbols()


def test_binding_structs_match_the_library(lib):
    """The ctypes copies of blockinv_options / blockinv_info / blockinv_result
    have the sizes the library was compiled with (a field added on one side
    only would shift every field after it)."""
    o, i, r = blockinv.blockinv_struct_sizes()
    assert (o, i, r) == (ctypes.sizeof(blockinv.Options), ctypes.sizeof(blockinv.Info),
                         ctypes.sizeof(blockinv.Result))


def test_status_strings_and_version(lib):
    assert blockinv.blockinv_version() >= 100
    assert blockinv.blockinv_status_str(0) == "ok"
    assert "singular" in blockinv.blockinv_status_str(-2)


@pytest.mark.parametrize("n,sizes,lda", [
    (0, None, 0),            # empty order
    (4, [2, 1], 4),          # sizes do not sum to n
    (4, [4, 0], 4),          # zero block
    (4, [4], 3),             # lda < n
    (600, [600], 600),       # block above the pivot-kernel limit
    (-3, None, 4),
])
def test_argument_errors_are_synchronous(lib, n, sizes, lda):
    st = blockinv.blockinv_invert(n, sizes, 0x1000, lda, 0, None)
    assert st == blockinv.ERR_INVALID
    assert blockinv.blockinv_last_error_detail() == (blockinv.ERR_INVALID, -1)


def test_argument_errors_leave_no_cuda_error(lib):
    # argument errors return before any CUDA call, so no runtime failure is
    # recorded; reading the record clears it
    blockinv.blockinv_last_cuda_error()
    assert blockinv.blockinv_invert(4, [2, 1], 0x1000, 4, 0, None) == blockinv.ERR_INVALID
    assert blockinv.blockinv_invert(8, [8], 0x1000, 8, 7, None) == blockinv.ERR_INVALID
    assert blockinv.blockinv_last_cuda_error() == (0, "cudaSuccess")
    assert blockinv.blockinv_last_cuda_error() == (0, "cudaSuccess")


def test_null_pointer_rejected(lib):
    assert blockinv.blockinv_invert(8, None, None, 8, 0, None) == blockinv.ERR_INVALID


def test_unknown_mode_rejected_before_gpu_work(lib):
    assert blockinv.blockinv_invert(8, [8], 0x1000, 8, 7, None) == blockinv.ERR_INVALID


def test_mixed_modes_reject_orders_above_16384(lib):
    # the refinement residual's digit products are exact only up to n = 16384
    for mode in (1, 2):
        assert blockinv.blockinv_invert(16385, None, 0x1000, 16385, mode, None) == blockinv.ERR_INVALID
    st, _ = blockinv.blockinv_residual_tc(16385, 0x1000, 16385, 0x2000, 16385)
    assert st == blockinv.ERR_INVALID
    st, _ = blockinv.blockinv_residual_tc(64, 0x1000, 64, 0x2000, 64, slices=10)
    assert st == blockinv.ERR_INVALID


def test_batch_tuning_table_roundtrip(lib, tmp_path):
    """The tuning table is host state: set, read, save, clear, load."""
    assert blockinv.blockinv_batch_tuning_clear() == blockinv.OK
    assert blockinv.blockinv_batch_tuning(5) == (blockinv.OK, 0, 64)
    assert blockinv.blockinv_batch_tuning_set(5, 4, 32) == blockinv.OK
    assert blockinv.blockinv_batch_tuning_set(9, 8, 64) == blockinv.OK
    assert blockinv.blockinv_batch_tuning(5) == (blockinv.OK, 4, 32)
    path = tmp_path / "tuning.txt"
    assert blockinv.blockinv_batch_tuning_save(path) == blockinv.OK
    assert path.read_text().splitlines() == ["blockinv-batch-tuning 1", "5 4 32", "9 8 64"]
    assert blockinv.blockinv_batch_tuning_clear() == blockinv.OK
    assert blockinv.blockinv_batch_tuning(9) == (blockinv.OK, 0, 64)
    assert blockinv.blockinv_batch_tuning_load(path) == blockinv.OK
    assert blockinv.blockinv_batch_tuning(9) == (blockinv.OK, 8, 64)
    # malformed files and arguments are rejected and leave the table as it was
    bad = tmp_path / "bad.txt"
    bad.write_text("blockinv-batch-tuning 1\n5 4 48\n")
    assert blockinv.blockinv_batch_tuning_load(bad) == blockinv.ERR_INVALID
    assert blockinv.blockinv_batch_tuning(5) == (blockinv.OK, 4, 32)
    assert blockinv.blockinv_batch_tuning_set(2, 4, 64) == blockinv.ERR_INVALID
    assert blockinv.blockinv_batch_tuning_set(5, 4, 16) == blockinv.ERR_INVALID
    assert blockinv.blockinv_batch_tuning(17)[0] == blockinv.ERR_INVALID
    assert blockinv.blockinv_batch_tuning_load(tmp_path / "missing.txt") == blockinv.ERR_INVALID
    assert blockinv.blockinv_batch_tuning_clear() == blockinv.OK


def _checkpoint_bytes(n, sizes, k, data, magic=b"BLKINVC1", hash_delta=0):
    import struct
    payload = np.ascontiguousarray(data, dtype="<f8").tobytes()
    h = 1469598103934665603
    for byte in payload:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return (magic + struct.pack("<qii", n, len(sizes), k) + struct.pack(f"<{len(sizes)}i", *sizes)
            + struct.pack("<Q", (h + hash_delta) & 0xFFFFFFFFFFFFFFFF) + payload)


def test_checkpoint_read_rejects_bad_files_before_gpu_work(lib, tmp_path):
    """Every check of a checkpoint file happens on the host: a file that does
    not match is refused before any device copy (the target pointer is fake)."""
    n, sizes = 6, [2, 4]
    data = np.arange(36.0).reshape(6, 6)
    cases = {
        "magic": _checkpoint_bytes(n, sizes, 1, data, magic=b"BLKINVC0"),
        "order": _checkpoint_bytes(7, sizes, 1, np.zeros((7, 7))),
        "partition": _checkpoint_bytes(n, [3, 3], 1, data),
        "hash": _checkpoint_bytes(n, sizes, 1, data, hash_delta=1),
        "truncated": _checkpoint_bytes(n, sizes, 1, data)[:-8],
        "trailing": _checkpoint_bytes(n, sizes, 1, data) + b"x",
        "steps": _checkpoint_bytes(n, sizes, 3, data),
    }
    for name, blob in cases.items():
        path = tmp_path / f"{name}.ck"
        path.write_bytes(blob)
        st, k = blockinv.blockinv_checkpoint_read(path, n, sizes, 0x1000, n)
        assert st == blockinv.ERR_INVALID and k == -1, name
    assert blockinv.blockinv_checkpoint_read(tmp_path / "none.ck", n, sizes, 0x1000, n)[0] == blockinv.ERR_INVALID


def test_step_range_argument_errors(lib):
    for k0, k1 in [(-1, 1), (2, 1), (0, 3)]:
        assert blockinv.blockinv_invert_steps(6, [2, 4], 0x1000, 6, k0, k1) == blockinv.ERR_INVALID


def test_fixed_batched_argument_errors(lib):
    f = blockinv.blockinv_invert_batched_fixed
    assert f(10, 33, None, 0x1000) == blockinv.ERR_INVALID          # order above 32
    assert f(10, 11, [5, 5], 0x1000) == blockinv.ERR_INVALID        # partition does not sum to n
    assert f(10, 11, [5, 6, 0], 0x1000) == blockinv.ERR_INVALID
    assert f(10, 11, [5, 6], 0x1000, flags=2) == blockinv.ERR_INVALID
    assert f(10, 11, [5, 6], None) == blockinv.ERR_INVALID
    assert f(0, 11, [5, 6], None) == blockinv.OK


def test_diagnostic_argument_errors(lib):
    """The diagnostic entry points reject bad arguments before any CUDA call."""
    assert blockinv.blockinv_diag_wait_timeout(-1, None) == blockinv.ERR_INVALID
    assert blockinv.blockinv_diag_wait_timeout(2_000_000_001, None) == blockinv.ERR_INVALID
    assert blockinv.blockinv_diag_recip64(None, None, -1, None) == blockinv.ERR_INVALID
    assert blockinv.blockinv_diag_recip64(None, None, 4, None) == blockinv.ERR_INVALID
    assert blockinv.blockinv_diag_recip64(None, None, 0, None) == blockinv.OK


def test_block_tuning_table(lib):
    """The single-matrix block-size table: set / read / clear and argument
    checks, all on the host."""
    assert blockinv.blockinv_tuning_clear() == blockinv.OK
    assert blockinv.blockinv_tuning("tf32", 12) == (blockinv.OK, 0)
    assert blockinv.blockinv_tuning_set("tf32", 12, 384) == blockinv.OK
    assert blockinv.blockinv_tuning("tf32", 12) == (blockinv.OK, 384)
    assert blockinv.blockinv_tuning("f64", 12) == (blockinv.OK, 0)
    assert blockinv.blockinv_tuning_set("f64", 12, 513) == blockinv.ERR_INVALID
    assert blockinv.blockinv_tuning_set(3, 12, 256) == blockinv.ERR_INVALID
    assert blockinv.blockinv_tuning("f64", 21)[0] == blockinv.ERR_INVALID
    assert blockinv.blockinv_tuning_clear() == blockinv.OK
    assert blockinv.blockinv_tuning("tf32", 12) == (blockinv.OK, 0)
    assert blockinv.blockinv_tune([100], "f64", 0) == blockinv.ERR_INVALID
    assert blockinv.blockinv_tune([16385], "tf32", 1) == blockinv.ERR_INVALID
