"""GPU parity of the host entry point (raduls_sort_host: copy in, sort, copy
out) against the CPU oracle, bit for bit: pinned and pageable buffers, in
place and out of place, several record shapes, the degenerate sizes, and the
statistics it reports."""
from __future__ import annotations

import numpy as np
import pytest

import datagen
from gpu_util import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


def _sync():
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("name,n", [("uniform16", 300_001), ("uniform16", 5_000_000), ("widekey32", 70_001),
                                    ("uniform8", 1 << 20), ("skewed16", 400_000)])
def test_pinned_out_of_place_matches_oracle(oracle_mod, name, n):
    import torch
    p = lib()
    recs = datagen.WORKLOADS[name](n)
    kb = datagen.KEY_BYTES[name]
    rw = recs.shape[1]
    h_in = torch.from_numpy(recs.view(np.int64)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    p.raduls_sort_host(h_in, h_out, n, rw * 8, kb)
    assert p.raduls_stream_status() == 0
    want = oracle_mod.sort(recs, kb, threads=8)
    np.testing.assert_array_equal(h_out.numpy().view(np.uint64), want)
    np.testing.assert_array_equal(h_in.numpy().view(np.uint64), recs)  # the input is left alone


def test_pageable_in_place_matches_oracle(oracle_mod):
    p = lib()
    n = 123_457
    recs = datagen.random_records(n, 24, 16, 5)
    buf = recs.copy()
    p.raduls_sort_host(buf, buf, n, 24, 16, mode="plain")
    _sync()
    assert p.raduls_stream_status() == 0
    np.testing.assert_array_equal(buf, oracle_mod.sort(recs, 16, threads=8))


def test_stats_and_modes(oracle_mod):
    p = lib()
    n = 1 << 21
    recs = datagen.WORKLOADS["skewed16"](n)
    want = oracle_mod.sort(recs, 8, threads=8)
    for mode in ("plain", "learned", "auto"):
        out = np.empty_like(recs)
        st = p.raduls_sort_host(recs, out, n, 16, 8, mode=mode, stats=True)
        _sync()
        assert p.raduls_stream_status() == 0
        np.testing.assert_array_equal(out, want, err_msg=mode)
        assert st["gpu_launches"] > 0
        if mode == "learned":
            assert st["learned_used"] == 1


@pytest.mark.parametrize("n", [0, 1, 2])
def test_degenerate_sizes(oracle_mod, n):
    p = lib()
    recs = datagen.random_records(max(n, 1), 16, 8, 9)[:n].copy()
    out = np.full_like(recs, 7)
    p.raduls_sort_host(recs, out, n, 16, 8)
    _sync()
    assert p.raduls_stream_status() == 0
    np.testing.assert_array_equal(out, oracle_mod.sort(recs, 8, threads=1) if n else recs)


def test_bad_arguments_are_refused():
    p = lib()
    buf = datagen.random_records(65, 16, 8, 1)
    with pytest.raises(ValueError):
        p.raduls_sort_host(buf, buf[1:], 65, 16, 8)          # output too small: caught before the call
    with pytest.raises(p.RaduLSError):
        p.raduls_sort_host(buf[:64], buf[1:], 64, 16, 8)     # partly overlapping ranges: refused by the library
    with pytest.raises(p.RaduLSError):
        p.raduls_sort_host(buf, buf, 65, 12, 8)              # record size not a multiple of 8


@pytest.mark.parametrize("windows", ["1", "0"])
@pytest.mark.parametrize("mid_size", ["0", "40960"])
def test_window_copy_back_on_and_off(oracle_mod, windows, mid_size, monkeypatch):
    """The last step copied back window by window (default) and the whole
    array copied after the sort (RADULS_HOST_WINDOWS=0) give the same bytes:
    2^23 + 12,345 uniform records end in runs of small sub-bins for the
    streamed on-chip sort (the default) or, with the mid-size class on, in
    256 mid-size bins; windows do not fall on item boundaries."""
    import torch
    p = lib()
    monkeypatch.setenv("RADULS_HOST_WINDOWS", windows)
    monkeypatch.setenv("RADULS_BUCKET_MAX", mid_size)
    n = (1 << 23) + 12_345
    recs = datagen.WORKLOADS["uniform16"](n)
    h_in = torch.from_numpy(recs.view(np.int64)).pin_memory()
    h_out = torch.zeros_like(h_in).pin_memory()
    p.raduls_sort_host(h_in, h_out, n, 16, 8, mode="plain")
    assert p.raduls_stream_status() == 0
    np.testing.assert_array_equal(h_out.numpy().view(np.uint64), oracle_mod.sort(recs, 8, threads=8))
