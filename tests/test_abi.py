"""The C ABI library builds, loads without a GPU, and exports every function
declared in include/raduls.h; host-side argument checks work without a GPU."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(raduls_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_1612_02557_gb300 as p
    p.build_library()
    return p.load()


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ["raduls_sort", "raduls_sort_ex", "raduls_sort_batched", "raduls_stream_status",
                 "raduls_status_string", "raduls_histogram", "raduls_distribution_pass"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1612_02557_gb300 as p
    out = subprocess.run(["nm", "-D", "--defined-only", p.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (raduls_[a-z_0-9]+)", out))
    for name in _declared_functions():
        assert name in exported, f"{name} declared but not exported"
        assert hasattr(lib, name)


def test_status_strings(lib):
    import paper_1612_02557_gb300 as p
    for code in range(8):
        assert p.raduls_status_string(code) != "unknown status"
    assert p.raduls_status_string(99) == "unknown status"


def test_host_argument_checks_without_gpu(lib):
    # all of these are rejected on the host before any CUDA call
    assert lib.raduls_sort(16, 4096, 10, 12, 8, None) == 1        # rec_bytes not a multiple of 8
    assert lib.raduls_sort(16, 4096, 10, 16, 24, None) == 1       # key longer than record
    assert lib.raduls_sort(16, 4096, 10, 264, 8, None) == 3       # record too wide
    assert lib.raduls_sort(8, 4096, 10, 16, 8, None) == 2         # misaligned
    assert lib.raduls_sort(16, 32, 10, 16, 8, None) == 2          # overlapping buffers
    assert lib.raduls_sort(0, 0, 1, 16, 8, None) == 0             # n <= 1 is a no-op
    assert lib.raduls_sort(0, 0, 0, 16, 8, None) == 0
    assert lib.raduls_distribution_pass(16, 4096, 10, 16, 8, 9, None) == 1  # digit out of range
    assert lib.raduls_debug_inject(5, 0) == 1
    # the allocation-free histogram: one record past its fixed tile map
    # (260,928 tiles of 16,384 records) is rejected before any CUDA call
    assert lib.raduls_histogram_static(16, 260928 * 16384 + 1, 16, 8, 7, 4096, None) == 3
    assert lib.raduls_histogram_static(16, 10, 16, 8, 8, 4096, None) == 1   # digit out of range
    assert lib.raduls_histogram_static(8, 10, 16, 8, 7, 4096, None) == 2    # misaligned records
    assert lib.raduls_set_wait_limit_ns(0) == 1
    # the key-index sort and the run counter: the same record rules, plus their own
    assert lib.raduls_sort_indexed(16, 4096, 10, 12, 8, None) == 1     # rec_bytes not a multiple of 8
    assert lib.raduls_sort_indexed(8, 4096, 10, 16, 8, None) == 2      # misaligned
    assert lib.raduls_sort_indexed(0, 0, 1, 64, 8, None) == 0          # n <= 1 is a no-op
    assert lib.raduls_unique_counts(8, 10, 16, 8, 8, 8, None, None) == 1   # no place for the run count
    assert lib.raduls_unique_counts(4, 10, 16, 8, 8, 8, 8, None) == 2      # misaligned records
    assert lib.raduls_unique_counts(8, 10, 16, 24, 8, 8, 8, None) == 1     # key longer than record
    # the host entry point: the same record rules, plus its own buffer rules
    assert lib.raduls_sort_host(16, 4096, 10, 12, 8, None, None) == 1   # rec_bytes not a multiple of 8
    assert lib.raduls_sort_host(None, 4096, 10, 16, 8, None, None) == 1  # no input
    assert lib.raduls_sort_host(16, None, 10, 16, 8, None, None) == 1   # no output
    assert lib.raduls_sort_host(16, 32, 10, 16, 8, None, None) == 1     # partly overlapping host ranges
    assert lib.raduls_sort_host(None, None, 0, 16, 8, None, None) == 0  # nothing to sort
    from paper_1612_02557_gb300._lib import Opts
    bad = Opts(7, 0, 0.0, 0, None)
    assert lib.raduls_sort_host(16, 4096, 10, 16, 8, ctypes.byref(bad), None) == 1  # unknown mode
    bad = Opts(2, 20, 0.0, 0, None)
    assert lib.raduls_sort_host(16, 4096, 10, 16, 8, ctypes.byref(bad), None) == 1  # learned buckets > 2^16


def test_python_binding_rejects_bad_modes(lib):
    import paper_1612_02557_gb300 as p
    with pytest.raises(KeyError):
        p.raduls_sort_ex(0, 0, 0, 16, 8, mode="bogus")
