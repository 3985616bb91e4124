"""The autotuner: every candidate it times must sort correctly, and sorts with
the settings it keeps (plain and batched) still equal the oracle bit for bit.
Each distribution tile shape is also checked on its own."""
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


@pytest.mark.parametrize("variant", [1, 5, 8, 9, 10, 11])
def test_each_distribution_shape_matches_oracle(oracle_mod, variant):
    recs = datagen.random_records(3_000_001, 16, 8, 77)
    old = os.environ.get("RADULS_SCATTER_VARIANT")
    os.environ["RADULS_SCATTER_VARIANT"] = str(variant)
    try:
        got = gpu_sort(recs, 8)
    finally:
        if old is None:
            del os.environ["RADULS_SCATTER_VARIANT"]
        else:
            os.environ["RADULS_SCATTER_VARIANT"] = old
    np.testing.assert_array_equal(got, oracle_mod.sort(recs, 8, threads=8))


def test_tuned_settings_keep_parity(oracle_mod):
    import torch
    p = lib()
    try:
        n = 1 << 22
        a = scratch(n, 2)
        b = scratch(n, 2)
        t = p.raduls_autotune(a, b, n, 16, 8)
        assert t["candidates"] >= 2 and t["best_ms"] > 0
        assert t["block_cap"] in (2048, 2560, 4096, 5120, 8192) and t["scatter_variant"] in (1, 5, 8, 9, 10, 11)
        assert 8 <= t["digit_bits"] <= 10 and 0 < t["leaf"] <= t["block_cap"] and t["bin_sort"] in (0, 1)
        for size in (1 << 21, 3_000_001):
            recs = datagen.random_records(size, 16, 8, size)
            np.testing.assert_array_equal(gpu_sort(recs, 8), oracle_mod.sort(recs, 8, threads=8))
        # batched: tune with an offset table, then a batched call on new data
        sizes = datagen.batched_sizes(3000)
        recs, offs = datagen.batched16(sizes=sizes)
        d_off = torch.from_numpy(offs.astype(np.uint64).view(np.int64)).cuda()
        m = recs.shape[0]
        a2, b2 = scratch(m, 2), scratch(m, 2)
        tb = p.raduls_autotune(a2, b2, m, 16, 8, d_off, offs.size - 1)
        assert tb["candidates"] >= 2
        d = to_dev(recs)
        p.raduls_sort_batched(d, b2, d_off, offs.size - 1, 16, 8)
        assert p.raduls_stream_status() == 0
        np.testing.assert_array_equal(from_dev(d, m, 2), oracle_mod.sort_segments(recs, 8, offs, threads=8))
    finally:
        p.raduls_autotune_reset()
