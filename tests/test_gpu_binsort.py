"""The streamed on-chip finisher (binsort.cu) against the oracle, bit for bit.

Small bins (and runs of small sub-bins) are sorted in shared memory by a
13-bit code count, a placement of (code, next 38 key bits, index) words and a
rank inside each code group; items with large groups of near-equal keys are
handed to the general on-chip kernel.  Every case runs with the finisher on
and off (RADULS_BIN_SORT), so both paths, and the hand-over between them, are
checked on the same inputs."""
from __future__ import annotations

import contextlib
import os

import numpy as np
import pytest

import datagen
from gpu_util import gpu_sort, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


@contextlib.contextmanager
def _env(**kv):
    old = {k: os.environ.get(k) for k in kv}
    os.environ.update({k: str(v) for k, v in kv.items()})
    try:
        yield
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _keys_from(words: np.ndarray, n: int, rw: int) -> np.ndarray:
    recs = np.empty((n, rw), dtype=np.uint64)
    recs[:, : words.shape[1]] = words
    recs[:, words.shape[1]:] = np.arange(n, dtype=np.uint64)[:, None]  # payload = input index
    return recs


@pytest.mark.parametrize("on", [0, 1])
@pytest.mark.parametrize("n", [2, 2047, 4097, 5119, 5121, 200_003, 3_000_017])
@pytest.mark.parametrize("rec_bytes,key_bytes", [(16, 8), (8, 8), (32, 8), (32, 16)])
def test_uniform_sizes(oracle_mod, on, n, rec_bytes, key_bytes):
    recs = datagen.random_records(n, rec_bytes, key_bytes, 1000 + n)
    with _env(RADULS_BIN_SORT=on):
        got = gpu_sort(recs, key_bytes)
    np.testing.assert_array_equal(got, oracle_mod.sort(recs, key_bytes, threads=8))


@pytest.mark.parametrize("on", [0, 1])
@pytest.mark.parametrize("distinct", [1, 3, 70, 5000])
def test_near_equal_keys_hand_over(oracle_mod, on, distinct):
    # few distinct keys: code groups far above the ranking bound, so items
    # leave the finisher for the general kernel
    rng = np.random.default_rng(distinct)
    n = 1_000_003
    vals = rng.integers(0, 2**64, size=distinct, dtype=np.uint64)
    keys = vals[rng.integers(0, distinct, size=n)]
    recs = _keys_from(keys[:, None], n, 2)
    with _env(RADULS_BIN_SORT=on):
        got = gpu_sort(recs, 8)
    np.testing.assert_array_equal(got, oracle_mod.sort(recs, 8, threads=8))


@pytest.mark.parametrize("on", [0, 1])
@pytest.mark.parametrize("low_bits", [4, 20, 40])
def test_constant_top_bits_and_close_keys(oracle_mod, on, low_bits):
    # keys that differ only in their low bits: the first code window is
    # constant, the finisher moves it down to the highest varying bit
    rng = np.random.default_rng(low_bits)
    n = 700_001
    top = np.uint64(0xA5A5A5A5A5A5A5A5) & ~np.uint64((1 << low_bits) - 1)
    keys = top | rng.integers(0, 1 << low_bits, size=n, dtype=np.uint64)
    recs = _keys_from(keys[:, None], n, 2)
    with _env(RADULS_BIN_SORT=on):
        got = gpu_sort(recs, 8)
    np.testing.assert_array_equal(got, oracle_mod.sort(recs, 8, threads=8))


@pytest.mark.parametrize("on", [0, 1])
def test_two_word_keys_tied_on_the_compared_bits(oracle_mod, on):
    # 16-byte keys (in 16-byte records) whose words tie often: the 32 bits
    # after the code tie, the rest of the key decides
    rng = np.random.default_rng(5)
    n = 600_011
    w0 = rng.integers(0, 64, size=n, dtype=np.uint64) << np.uint64(58)
    w1 = rng.integers(0, 4, size=n, dtype=np.uint64)
    recs = np.stack([w0, w1], axis=1)
    with _env(RADULS_BIN_SORT=on):
        got = gpu_sort(recs, 16)
    np.testing.assert_array_equal(got, oracle_mod.sort(recs, 16, threads=8))


@pytest.mark.parametrize("on", [0, 1])
@pytest.mark.parametrize("wmax,leaf", [(8, 0), (10, 4096), (10, 1024), (9, 2048)])
def test_digit_widths_feed_the_finisher(oracle_mod, on, wmax, leaf):
    recs = datagen.random_records(2_500_007, 16, 8, wmax * 100 + leaf)
    kw = {"RADULS_BIN_SORT": on, "RADULS_WMAX": wmax}
    if leaf:
        kw["RADULS_LEAF"] = leaf
    with _env(**kw):
        got = gpu_sort(recs, 8)
    np.testing.assert_array_equal(got, oracle_mod.sort(recs, 8, threads=8))


@pytest.mark.parametrize("rec_bytes", [8, 32])
@pytest.mark.parametrize("distinct", [3, 5000])
def test_near_equal_keys_other_widths(oracle_mod, rec_bytes, distinct):
    rng = np.random.default_rng(distinct + rec_bytes)
    n = 600_007
    vals = rng.integers(0, 2**64, size=distinct, dtype=np.uint64)
    keys = vals[rng.integers(0, distinct, size=n)]
    recs = _keys_from(keys[:, None], n, rec_bytes // 8)
    for on in (0, 1):
        with _env(RADULS_BIN_SORT=on):
            np.testing.assert_array_equal(gpu_sort(recs, 8), oracle_mod.sort(recs, 8, threads=8))


def test_skewed_prefix_both_ways(oracle_mod):
    recs = datagen.skewed16(1 << 21)
    want = oracle_mod.sort(recs, 8, threads=8)
    for on in (0, 1):
        with _env(RADULS_BIN_SORT=on):
            np.testing.assert_array_equal(gpu_sort(recs, 8), want)
