"""Pins of the CPU oracle against the definition of the stable sort.

Every check here is independent of the oracle's own arithmetic: Python's
stable ``sorted`` on key tuples, numpy ``lexsort`` with an index tie-break,
``bincount`` of raw record bytes, and order-free invariants.  The mutant test
at the end plants plausible mistakes in a copy of ``oracle.c`` and shows that
these pins catch each one.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

import datagen
from checks import (brute_force_sort, check_sorted_output, is_sorted, lexsort_sort,
                    multiset_hash, stable_by_payload)

# Three key values that sort differently under each plausible byte-order mistake:
# as little-endian u64 words: B < A < C; read as big-endian bytes: A < C < B.
KEY_ALPHABET_1W = [0x0000000000000100, 0x00000000000000FF, 0x0100000000000000]
# Two-word keys, word 0 most significant: (0, 9) < (0, 0x100) < (1, 0); the order
# changes if word 1 were taken as the more significant one.
KEY_ALPHABET_2W = [(1, 0), (0, 0x100), (0, 9)]


def _recs_from_keys(keys, rec_words, key_words):
    n = len(keys)
    out = np.zeros((n, rec_words), dtype=np.uint64)
    for i, k in enumerate(keys):
        kk = k if isinstance(k, tuple) else (k,)
        for j in range(key_words):
            out[i, j] = kk[j]
        if rec_words > key_words:
            out[i, key_words] = i
    return out


def test_exhaustive_tiny_one_word(oracle_mod):
    """All key sequences of length <= 6 over a 3-value alphabet (729 at n=6)."""
    for n in range(0, 7):
        for combo in itertools.product(KEY_ALPHABET_1W, repeat=n):
            recs = _recs_from_keys(list(combo), 2, 1)
            got = oracle_mod.sort(recs, 8)
            np.testing.assert_array_equal(got, brute_force_sort(recs, 8))


def test_exhaustive_tiny_two_words(oracle_mod):
    for n in range(0, 6):
        for combo in itertools.product(KEY_ALPHABET_2W, repeat=n):
            recs = _recs_from_keys(list(combo), 3, 2)
            got = oracle_mod.sort(recs, 16)
            np.testing.assert_array_equal(got, brute_force_sort(recs, 16))


SHAPES = [(8, 8), (16, 8), (24, 8), (16, 16), (24, 16), (32, 16), (32, 24), (64, 8), (40, 32)]


@pytest.mark.parametrize("rec_bytes,key_bytes", SHAPES)
@pytest.mark.parametrize("alphabet", [2, 3, None])
def test_random_vs_brute_force(oracle_mod, rec_bytes, key_bytes, alphabet):
    for n, seed in [(1, 1), (2, 2), (33, 3), (517, 4)]:
        recs = datagen.random_records(n, rec_bytes, key_bytes, seed * 131 + rec_bytes, alphabet)
        got = oracle_mod.sort(recs, key_bytes)
        np.testing.assert_array_equal(got, brute_force_sort(recs, key_bytes))


@pytest.mark.parametrize("rec_bytes,key_bytes", SHAPES)
def test_random_vs_lexsort_4096(oracle_mod, rec_bytes, key_bytes):
    recs = datagen.random_records(4096, rec_bytes, key_bytes, 77 + key_bytes, alphabet=3)
    got = oracle_mod.sort(recs, key_bytes)
    np.testing.assert_array_equal(got, lexsort_sort(recs, key_bytes))
    check_sorted_output(recs, got, key_bytes, payload_index=rec_bytes > key_bytes)


@pytest.mark.parametrize("threads", [2, 3, 7, 16])
def test_threaded_equals_single(oracle_mod, threads):
    for n in [0, 1, 5, 1000, 65537]:
        recs = datagen.random_records(n, 16, 8, n + threads, alphabet=4)
        a = oracle_mod.sort(recs, 8, threads=1)
        b = oracle_mod.sort(recs, 8, threads=threads)
        np.testing.assert_array_equal(a, b)


def test_invariants_workloads(oracle_mod):
    """The five workload generators, small prefixes: ordered, permutation, stable."""
    cases = [
        (datagen.uniform8(20000), 8, False),
        (datagen.uniform16(50000), 8, True),
        (datagen.skewed16(50000), 8, True),
        (datagen.widekey32(30000), 16, True),
    ]
    r, _ = datagen.batched16(n_arrays=8, sizes=np.array([16, 100, 1, 0, 3000, 17, 5000, 2]))
    cases.append((r, 8, True))
    for recs, kb, payload in cases:
        out = oracle_mod.sort(recs, kb, threads=4)
        check_sorted_output(recs, out, kb, payload)
        np.testing.assert_array_equal(out, lexsort_sort(recs, kb))


def test_degenerate_cases(oracle_mod):
    # all keys equal: output equals input (stability), for a wide key too
    recs = np.zeros((1000, 4), dtype=np.uint64)
    recs[:, 2] = np.arange(1000)
    recs[:, 3] = np.arange(1000)[::-1]
    np.testing.assert_array_equal(oracle_mod.sort(recs, 16), recs)
    # already sorted stays, reverse-sorted reverses
    k = np.arange(500, dtype=np.uint64) * np.uint64(0x0101010101010101 // 255 * 3)
    recs = np.stack([k, np.arange(500, dtype=np.uint64)], axis=1)
    np.testing.assert_array_equal(oracle_mod.sort(recs, 8), recs)
    np.testing.assert_array_equal(oracle_mod.sort(recs[::-1].copy(), 8), recs[::-1][np.argsort(k[::-1], kind="stable")])
    # extreme values: 0 and 2^64-1
    recs = np.array([[2**64 - 1, 0], [0, 1], [2**63, 2], [2**63 - 1, 3], [2**64 - 1, 4]], dtype=np.uint64)
    out = oracle_mod.sort(recs, 8)
    np.testing.assert_array_equal(out[:, 1], np.array([1, 3, 2, 0, 4], dtype=np.uint64))
    # rec_bytes == key_bytes (no payload), 3 words
    recs = datagen.random_records(300, 24, 24, 5, alphabet=2, payload_index=False)
    np.testing.assert_array_equal(oracle_mod.sort(recs, 24), brute_force_sort(recs, 24))


def test_bad_args(oracle_mod):
    recs = np.zeros((4, 2), dtype=np.uint64)
    with pytest.raises(ValueError):
        oracle_mod.sort(recs, 24)       # key longer than the record
    with pytest.raises(ValueError):
        oracle_mod.sort(recs, 12)       # key not a multiple of 8 bytes


def _digit_bytes(recs: np.ndarray, key_bytes: int, digit: int) -> np.ndarray:
    """Digit ``digit`` straight from raw bytes: byte digit%8 of word W-1-digit//8."""
    kw = key_bytes // 8
    word = kw - 1 - digit // 8
    raw = recs.view(np.uint8).reshape(recs.shape[0], -1)
    return raw[:, 8 * word + digit % 8]


@pytest.mark.parametrize("rec_bytes,key_bytes", [(8, 8), (16, 8), (32, 16)])
def test_counting_pass_and_histogram(oracle_mod, rec_bytes, key_bytes):
    recs = datagen.random_records(3001, rec_bytes, key_bytes, 9, alphabet=5)
    for digit in range(8 * key_bytes // 8):
        d = _digit_bytes(recs, key_bytes, digit)
        h = oracle_mod.histogram(recs, key_bytes, digit)
        np.testing.assert_array_equal(h, np.bincount(d, minlength=256).astype(np.uint64))
        out = oracle_mod.counting_pass(recs, key_bytes, digit)
        np.testing.assert_array_equal(out, recs[np.argsort(d, kind="stable")])


def test_segmented_pass_and_segment_sort(oracle_mod):
    recs = datagen.random_records(5000, 16, 8, 11, alphabet=3)
    offs = np.array([0, 0, 1, 700, 701, 3000, 5000], dtype=np.uint64)
    d = _digit_bytes(recs, 8, 7)
    out = oracle_mod.segmented_counting_pass(recs, 8, 7, offs)
    ref = recs.copy()
    for s in range(len(offs) - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        ref[a:b] = recs[a:b][np.argsort(d[a:b], kind="stable")]
    np.testing.assert_array_equal(out, ref)
    out = oracle_mod.sort_segments(recs, 8, offs)
    for s in range(len(offs) - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        np.testing.assert_array_equal(out[a:b], brute_force_sort(recs[a:b], 8))


def test_check_helpers_reject_wrong_outputs():
    """The invariant helpers themselves must fail on broken outputs."""
    recs = datagen.random_records(200, 16, 8, 3, alphabet=2)
    good = lexsort_sort(recs, 8)
    assert is_sorted(good, 8) and stable_by_payload(good, 8)
    bad = good.copy()
    bad[[0, -1]] = bad[[-1, 0]]
    assert not is_sorted(bad, 8)
    unstable = good.copy()
    eq = np.flatnonzero(np.all(unstable[:-1, :1] == unstable[1:, :1], axis=1))[0]
    unstable[[eq, eq + 1]] = unstable[[eq + 1, eq]]
    assert is_sorted(unstable, 8) and not stable_by_payload(unstable, 8)
    dup = good.copy()
    dup[5] = dup[4]
    assert multiset_hash(dup) != multiset_hash(good)


# ------------------------------------------------------------- planted mistakes

MUTANTS = {
    "word_order": ("uint32_t word = key_words - 1u - p / 8u;", "uint32_t word = p / 8u;"),
    "byte_order": ("rec[8u * word + (p % 8u)]", "rec[8u * word + (7u - p % 8u)]"),
    "chunk_major_offsets": ("for (unsigned d = 0; d < RADIX; ++d)\n                for (uint32_t c = 0; c < T; ++c) {",
                            "for (uint32_t c = 0; c < T; ++c)\n                for (unsigned d = 0; d < RADIX; ++d) {"),
    "dropped_top_digits": ("const uint32_t passes = 8u * kw;", "const uint32_t passes = 8u * kw - 2u;"),
    "passes_not_chained": ("const uint8_t *src = (p == 0) ? j->in : j->buf[p % 2u == 1u ? 0 : 1];",
                           "const uint8_t *src = j->in;"),
}


def _pins_pass(sort_fn) -> bool:
    """The pin suite in miniature, run against an arbitrary sort function."""
    try:
        for n in range(0, 5):
            for combo in itertools.product(KEY_ALPHABET_1W, repeat=n):
                recs = _recs_from_keys(list(combo), 2, 1)
                if not np.array_equal(sort_fn(recs, 8, 1), brute_force_sort(recs, 8)):
                    return False
        for n in range(0, 4):
            for combo in itertools.product(KEY_ALPHABET_2W, repeat=n):
                recs = _recs_from_keys(list(combo), 3, 2)
                if not np.array_equal(sort_fn(recs, 16, 1), brute_force_sort(recs, 16)):
                    return False
        for threads in (1, 3):
            recs = datagen.random_records(2000, 16, 8, 21, alphabet=3)
            if not np.array_equal(sort_fn(recs, 8, threads), lexsort_sort(recs, 8)):
                return False
    except Exception:
        return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(tmp_path, name):
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")
    src = open(here).read()
    old, new = MUTANTS[name]
    assert old in src, f"mutant {name} no longer applies"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    lib.oracle_sort.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_uint32]

    def sort_fn(recs, kb, threads):
        out = np.empty_like(recs)
        rc = lib.oracle_sort(recs.ctypes.data, out.ctypes.data, recs.shape[0], recs.shape[1] * 8, kb, threads)
        if rc:
            raise ValueError(rc)
        return out

    assert not _pins_pass(sort_fn), f"pins failed to catch mutant {name}"


def test_pins_accept_true_oracle(oracle_mod):
    assert _pins_pass(lambda r, kb, t: oracle_mod.sort(r, kb, threads=t))
