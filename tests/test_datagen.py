"""The seeded workload generators follow the stated input recipe (CPU):
payload layouts, component mixtures, value ranges, distinct-value counts,
array-size law, prefix stability of the uniform workloads, determinism of
the mixtures.  Tolerances are several standard deviations of the sampling
error."""
from __future__ import annotations

import math

import numpy as np
import pytest

import datagen

N = 1 << 20


def test_uniform16_payload_and_uniform_top_byte():
    r = datagen.uniform16(N)
    assert r.shape == (N, 2) and r.dtype == np.uint64
    assert np.array_equal(r[:, 1], np.arange(N, dtype=np.uint64))
    top = np.bincount((r[:, 0] >> np.uint64(56)).astype(np.int64), minlength=256)
    expect = N / 256
    chi2 = float(((top - expect) ** 2 / expect).sum())
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)  # chi-square with 255 degrees of freedom, far tail


def test_uniform_inputs_are_prefixes_of_larger_ones():
    big = datagen.uniform16(3 << 24)  # spans several generator chunks
    small = datagen.uniform16(1 << 20)
    assert np.array_equal(big[: 1 << 20], small)
    assert np.array_equal(datagen.uniform8(1 << 20)[:1000], datagen.uniform8(1000))


def test_mixtures_are_seeded_same_law_draws():
    # not prefixes (each chunk's components are drawn in batches sized by the
    # fill), but deterministic for a given n and seed
    a = datagen.skewed16(1 << 18)
    assert np.array_equal(a, datagen.skewed16(1 << 18))
    assert not np.array_equal(a, datagen.skewed16(1 << 18, seed=datagen.SEEDS["skewed16"] + 1))


def test_skewed16_mixture():
    r = datagen.skewed16(N)
    k = r[:, 0]
    assert np.array_equal(r[:, 1], np.arange(N, dtype=np.uint64))
    exp_part = (k < np.uint64(1 << 43)).mean()                       # exponential component (mean 1e12)
    top16 = k >> np.uint64(48)
    norm_part = ((top16 == 0x7FFF) | (top16 == 0x8000)).mean()       # 2^63 + N(0, 2^40)
    sd = math.sqrt(0.25 / N)
    assert abs(exp_part - 0.30) < 6 * sd + 1e-4
    assert abs(norm_part - 0.20) < 6 * sd + 1e-4
    # Zipf(1.1) component: its rank-1 key holds about 0.5 / zeta(1.1) of the records
    vals, counts = np.unique(k, return_counts=True)
    zeta = sum(i ** -1.1 for i in range(1, 200000)) + (200000 ** -0.1) / 0.1   # tail by the integral
    share = counts.max() / N
    assert abs(share - 0.5 / zeta) < 0.006
    assert vals.size < N * 0.75                                      # heavy duplication overall


def test_widekey32_layout():
    n = 1 << 18
    r = datagen.widekey32(n)
    assert r.shape == (n, 4)
    idx = np.arange(n, dtype=np.uint64)
    assert np.array_equal(r[:, 2], idx)
    assert np.array_equal(r[:, 3], datagen.mix64(idx, datagen.SEEDS["widekey32"]))
    distinct = np.unique(r[:, 0]).size
    assert distinct <= datagen.DISTINCT5
    # Zipf(1.0) over 2^20 values: the top value holds about 1 / H(2^20) of the records
    h = float(np.sum(1.0 / np.arange(1, datagen.DISTINCT5 + 1)))
    top_share = np.unique(r[:, 0], return_counts=True)[1].max() / n
    assert abs(top_share - 1.0 / h) < 0.01
    assert np.unique(r[:, 1]).size > n * 0.999                       # word 1 uniform: almost no repeats


def test_batched_sizes_law():
    u = datagen.batched_upper()
    sizes = datagen.batched_sizes()
    assert sizes.size == datagen.BATCHED_N_ARRAYS
    assert sizes.min() >= datagen.BATCHED_MIN and sizes.max() <= u
    assert 40_000 < u < 45_000
    # log-uniform on [16, U]: its mean times the array count is 2^30
    mean = (u - datagen.BATCHED_MIN) / math.log(u / datagen.BATCHED_MIN)
    assert abs(mean * sizes.size / (1 << 30) - 1.0) < 1e-6
    total = int(sizes.sum())
    assert abs(total / (1 << 30) - 1.0) < 0.01


def test_batched16_odd_arrays_share_their_top_half():
    sizes = datagen.batched_sizes()[:64]
    recs, offsets = datagen.batched16(sizes=sizes)
    assert offsets[0] == 0 and offsets[-1] == recs.shape[0]
    assert np.array_equal(np.diff(offsets.astype(np.int64)), sizes)
    for a in range(64):
        top = recs[int(offsets[a]):int(offsets[a + 1]), 0] >> np.uint64(32)
        if a % 2:
            assert np.unique(top).size == 1
        else:
            assert np.unique(top).size > 1


@pytest.mark.parametrize("name", ["uniform8", "uniform16", "skewed16", "widekey32"])
def test_shapes_match_the_bench_table(name):
    n = 4096
    r = datagen.WORKLOADS[name](n)
    assert r.shape == (n, datagen.REC_BYTES[name] // 8)
    assert datagen.KEY_BYTES[name] <= datagen.REC_BYTES[name]


def test_batched_wide_sizes_law():
    """The second batched reading: log-uniform sizes on [16, 2^20] drawn until
    their sum first reaches 2^30 (the last array crosses it)."""
    sizes = datagen.batched_sizes_wide()
    assert sizes.min() >= datagen.BATCHED_MIN and sizes.max() <= datagen.BATCHED_WIDE_MAX
    total = int(sizes.sum())
    assert total >= 1 << 30 and total - int(sizes[-1]) < 1 << 30
    # mean of log-uniform [16, 2^20] is (2^20 - 16) / ln(2^16): about 94,547 -> about 11,360 arrays
    mean = (datagen.BATCHED_WIDE_MAX - datagen.BATCHED_MIN) / math.log(datagen.BATCHED_WIDE_MAX / datagen.BATCHED_MIN)
    assert abs(sizes.size * mean / (1 << 30) - 1.0) < 0.05
    assert (sizes > 40_960).mean() > 0.25     # about 29% of the arrays lie above the mid-size class
    recs, offs = datagen.batched16w(sizes=sizes[:40])
    assert offs[-1] == recs.shape[0] and np.array_equal(np.diff(offs.astype(np.int64)), sizes[:40])
