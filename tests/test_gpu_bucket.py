"""GPU parity of the mid-size bin path (one CTA sorts a bin through L2)
against the CPU oracle, bit for bit.

Inputs are built so that every branch of that kernel runs: bins at the first
and at later levels, runs of small sub-bins, single sub-bins sorted by the
whole CTA, sub-bins too big for shared memory that go on to the next level,
bins whose last digit is split (no digit left after it) from either buffer,
and heavy duplicates (with 8-bit digits in every distribution pass, as the
inputs are built around them, and the class switched on: plain sorts leave it
off by default).  The same inputs sorted with the path switched off
(RADULS_BUCKET_MAX=0) must give the same bytes.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import datagen
from gpu_util import from_dev, gpu_sort, lib, scratch, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


@pytest.fixture(scope="module", autouse=True)
def _byte_digits():
    """8-bit digits in every distribution pass, so that the bins these inputs
    are built around occur as described, and the mid-size class switched on
    (plain sorts leave it off by default) for bins of up to 640 KB."""
    want = {"RADULS_WMAX": "8", "RADULS_BUCKET_MAX": "40960"}
    old = {k: os.environ.get(k) for k in want}
    os.environ.update(want)
    yield
    for k, v in old.items():
        if v is None:
            del os.environ[k]
        else:
            os.environ[k] = v


def _set_byte(keys: np.ndarray, byte: int, values: np.ndarray) -> None:
    sh = np.uint64(8 * byte)
    keys &= ~(np.uint64(0xFF) << sh)
    keys |= values.astype(np.uint64) << sh


def _structured(kind: str, n: int, rec_bytes: int, key_bytes: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    recs = datagen.random_records(n, rec_bytes, key_bytes, seed)
    k0 = recs[:, 0].copy()
    if kind == "spill":
        # top byte over 64 values (bins of n/64); next byte 0 for 60% of records:
        # one sub-bin per bin is bigger than the on-chip capacity
        _set_byte(k0, 7, rng.integers(0, 64, n))
        _set_byte(k0, 6, np.where(rng.random(n) < 0.6, 0, rng.integers(1, 256, n)))
    elif kind == "mid_children":
        # next byte over 16 values: sub-bins of a few thousand records
        _set_byte(k0, 7, rng.integers(0, 64, n))
        _set_byte(k0, 6, rng.integers(0, 16, n))
    elif kind == "last_digit":
        # only the lowest byte varies: the split reaches digit 0 in one bin
        k0[:] = np.uint64(0x0123456789ABCD00)
        _set_byte(k0, 0, rng.integers(0, 256, n))
    elif kind == "last_digit_two_bins":
        # two top-byte values, then constant bytes, then a random low byte
        k0[:] = np.uint64(0x0023456789ABCD00)
        _set_byte(k0, 7, rng.integers(0, 2, n) * 0x80)
        _set_byte(k0, 0, rng.integers(0, 256, n))
    elif kind == "duplicates":
        # few distinct keys per bin: long tie groups
        _set_byte(k0, 7, rng.integers(0, 64, n))
        k0 &= np.uint64(0xFF00000000000003)
    else:
        raise ValueError(kind)
    recs[:, 0] = k0
    return recs


def _with_env(name: str, value: str, fn):
    old = os.environ.get(name)
    os.environ[name] = value
    try:
        return fn()
    finally:
        if old is None:
            del os.environ[name]
        else:
            os.environ[name] = old


def _sort_both_ways(recs: np.ndarray, key_bytes: int):
    """The mid-size path on (the module's setting) and switched off (RADULS_BUCKET_MAX=0)."""
    got = gpu_sort(recs, key_bytes)
    off = _with_env("RADULS_BUCKET_MAX", "0", lambda: gpu_sort(recs, key_bytes))
    return {"on": got, "off": off}


@pytest.mark.parametrize("rec_bytes,key_bytes", [(8, 8), (16, 8), (32, 16), (24, 8), (16, 16)])
@pytest.mark.parametrize("n", [4097, 9000, 20000, 40960, 40961, 81920, 3_000_001])
def test_mid_size_bins_match_oracle(oracle_mod, rec_bytes, key_bytes, n):
    if n > 100_000 and rec_bytes > 16:
        pytest.skip("large case on the main shapes only")
    recs = datagen.random_records(n, rec_bytes, key_bytes, n + rec_bytes)
    ways = _sort_both_ways(recs, key_bytes)
    want = oracle_mod.sort(recs, key_bytes, threads=8)
    for name, got in ways.items():
        np.testing.assert_array_equal(got, want, err_msg=f"{name} n={n} shape={rec_bytes},{key_bytes}")


@pytest.mark.parametrize("kind", ["spill", "mid_children", "last_digit", "last_digit_two_bins", "duplicates"])
@pytest.mark.parametrize("rec_bytes,key_bytes,n", [(16, 8, 1 << 20), (8, 8, 1 << 20), (32, 16, 300_001),
                                                   (16, 8, 20_000)])
def test_structured_keys_match_oracle(oracle_mod, kind, rec_bytes, key_bytes, n):
    recs = _structured(kind, n, rec_bytes, key_bytes, 11 + n % 97)
    ways = _sort_both_ways(recs, key_bytes)
    want = oracle_mod.sort(recs, key_bytes, threads=8)
    for name, got in ways.items():
        np.testing.assert_array_equal(got, want, err_msg=f"{name} {kind} n={n} shape={rec_bytes},{key_bytes}")


def test_stats_count_mid_size_bins(oracle_mod):
    """2^23 uniform 16-byte records: one device-wide pass, then 256 bins of
    about 32K records, each sorted by one CTA that counts for itself: the
    bytes moved are one histogram read plus two read+write passes."""
    p = lib()
    n = 1 << 23
    recs = datagen.uniform16(n)
    d = to_dev(recs)
    t = scratch(n, 2)
    st = p.raduls_sort_ex(d, t, n, 16, 8, mode="plain", stats=True)
    assert p.raduls_stream_status() == 0
    assert st["grid_passes"] == 1
    assert st["bucket_items"] == 256
    assert st["bucket_bytes"] == 2 * n * 16
    assert st["scatter_bytes"] == 2 * n * 16
    assert st["hist_bytes_read"] == n * 16             # level 0 only: mid-size bins need no histogram pass
    assert st["kernel_launches"]["bucket"] >= 1
    np.testing.assert_array_equal(from_dev(d, n, 2), oracle_mod.sort(recs, 8, threads=8))

