"""GPU tests of the wide-digit distribution pass: digit windows of 8 to 10
bits, windows that reach
across a key-word boundary, sub-bins aimed at different sizes, and bins that
span many chunks, each sort equal to the oracle bit for bit."""
from __future__ import annotations

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


class _env:
    """Set environment overrides of the launch shape for one block."""

    def __init__(self, **kv):
        self.kv = {k: str(v) for k, v in kv.items()}
        self.old = {}

    def __enter__(self):
        for k, v in self.kv.items():
            self.old[k] = os.environ.get(k)
            os.environ[k] = v

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


@pytest.mark.parametrize("wmax", [8, 9, 10])
@pytest.mark.parametrize("leaf", [64, 2048])
def test_digit_widths_match_oracle(oracle_mod, wmax, leaf):
    recs = datagen.random_records(300_001, 16, 8, wmax * 100 + leaf)
    with _env(RADULS_WMAX=wmax, RADULS_LEAF=leaf):
        got = gpu_sort(recs, 8)
    np.testing.assert_array_equal(got, oracle_mod.sort(recs, 8, threads=8))


@pytest.mark.parametrize("rec_bytes,key_bytes", [(8, 8), (24, 16), (32, 16), (40, 32)])
def test_wide_digits_every_shape_with_duplicates(oracle_mod, rec_bytes, key_bytes):
    for alphabet in (None, 3):
        recs = datagen.random_records(200_003, rec_bytes, key_bytes, rec_bytes + key_bytes, alphabet=alphabet)
        with _env(RADULS_WMAX=10, RADULS_LEAF=100):
            got = gpu_sort(recs, key_bytes)
        np.testing.assert_array_equal(got, oracle_mod.sort(recs, key_bytes, threads=8))


def test_windows_across_a_key_word_boundary(oracle_mod):
    """Only the low 4 bits of key word 0 and the top bits of word 1 vary, so
    after the constant bits are skipped the next window straddles the two
    words; equal word-1 tops make some windows constant too."""
    rng = np.random.default_rng(7)
    n = 400_000
    recs = np.empty((n, 4), dtype=np.uint64)
    recs[:, 0] = np.uint64(0xABCDEF0123456780) | rng.integers(0, 16, size=n, dtype=np.uint64)
    recs[:, 1] = (rng.integers(0, 1 << 12, size=n, dtype=np.uint64) << np.uint64(52)) | \
        rng.integers(0, 4, size=n, dtype=np.uint64)
    recs[:, 2] = np.arange(n, dtype=np.uint64)
    recs[:, 3] = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    for wmax, leaf in ((10, 64), (9, 300), (8, 2048)):
        with _env(RADULS_WMAX=wmax, RADULS_LEAF=leaf):
            got = gpu_sort(recs, 16)
        np.testing.assert_array_equal(got, oracle_mod.sort(recs, 16, threads=8), err_msg=f"wmax {wmax}")


def test_many_chunks_and_skewed_bins(oracle_mod):
    """3,000,001 records (46 chunks) of the skewed mixture: bins of very
    different sizes, heavy duplicates, constant windows."""
    recs = datagen.skewed16(3_000_001)
    for wmax in (10, 9):
        with _env(RADULS_WMAX=wmax):
            got = gpu_sort(recs, 8)
        np.testing.assert_array_equal(got, oracle_mod.sort(recs, 8, threads=8), err_msg=f"wmax {wmax}")


@pytest.mark.parametrize("rec_bytes,v9,v10", [(16, 9, 11), (16, 17, 16), (16, 19, 18), (16, 21, 20), (32, 14, 15), (8, 12, 13)])
@pytest.mark.parametrize("case", ["uniform", "few_values", "two_word_keys", "ragged"])
def test_scatter_shapes_of_9_and_10_bit_digits(oracle_mod, rec_bytes, v9, v10, case):
    # every two-CTA shape of 9- and 10-bit digits gives the same bytes, with
    # tag ranks (the default), match ranks (16-byte shapes 17 and 16) or vote
    # ranks (19 and 18), evict-last stores (the default) or plain ones (21 and
    # 20): partial last tiles, values shared by many records (the tags' vote
    # fallback), windows in the second key word
    n, key_bytes, alphabet = 1_000_003, 8, None
    if case == "few_values":
        alphabet = 7
    elif case == "two_word_keys":
        if rec_bytes == 8:
            pytest.skip("8-byte records hold one key word")
        key_bytes = 16
    elif case == "ragged":
        n = 4096 * 37 + 1
    recs = datagen.random_records(n, rec_bytes, key_bytes, v10 * 1000 + len(case), alphabet=alphabet)
    if case == "two_word_keys":
        recs[:, 0] &= np.uint64(0xFFFF)  # the top key bits tie: later windows reach into word 1
    want = oracle_mod.sort(recs, key_bytes, threads=8)
    # 8-byte records take one shape for every level (no per-width shapes)
    shapes = ([{"RADULS_SCATTER_VARIANT": v9}, {"RADULS_SCATTER_VARIANT": v10}] if rec_bytes == 8 else
              [{"RADULS_SCATTER9": v9, "RADULS_SCATTER10": v10}])
    for leaf in (300, 4096):
        for sh in shapes:
            with _env(RADULS_LEAF=leaf, **sh):
                np.testing.assert_array_equal(gpu_sort(recs, key_bytes), want)
