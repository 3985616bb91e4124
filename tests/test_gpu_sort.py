"""GPU parity of the sorter against the CPU oracle: bit-exact, element by element.

Each step kernel (histogram, one distribution pass) and the full sort are
compared with the oracle on the same seeded inputs, at sizes that span many
tiles with a ragged tail, for every record shape class, plus edge cases.
"""
from __future__ import annotations

import numpy as np
import pytest

import datagen
from gpu_util import from_dev, gpu_sort, lib, scratch, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8), (16, 8), (24, 8), (32, 16), (16, 16), (40, 32), (64, 8), (24, 24), (256, 16)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


@pytest.mark.parametrize("rec_bytes,key_bytes", [(8, 8), (16, 8), (32, 16), (40, 32)])
def test_histogram_matches_oracle(oracle_mod, rec_bytes, key_bytes):
    import torch
    p = lib()
    recs = datagen.random_records(3 * 65536 + 1234, rec_bytes, key_bytes, 5, alphabet=7)
    d = to_dev(recs)
    for digit in sorted({0, 3, 7, 8 * key_bytes // 8 - 1, 8 * key_bytes // 8 - 5}):
        h = torch.zeros(256, dtype=torch.int64, device="cuda")
        p.raduls_histogram(d, recs.shape[0], rec_bytes, key_bytes, digit, h)
        got = h.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(got, oracle_mod.histogram(recs, key_bytes, digit))


@pytest.mark.parametrize("rec_bytes,key_bytes", [(8, 8), (16, 8), (24, 8), (32, 16), (40, 32), (256, 16)])
@pytest.mark.parametrize("alphabet", [3, None])
def test_distribution_pass_matches_oracle(oracle_mod, rec_bytes, key_bytes, alphabet):
    p = lib()
    n = 2 * 65536 + 5 * 8192 + 333      # several chunks (look-back), tiles within them, ragged tail
    recs = datagen.random_records(n, rec_bytes, key_bytes, 17 + rec_bytes, alphabet=alphabet)
    d = to_dev(recs)
    out = scratch(n, rec_bytes // 8)
    for digit in sorted({0, 8 * key_bytes // 8 - 1, 9 % (8 * key_bytes // 8)}):
        p.raduls_distribution_pass(d, out, n, rec_bytes, key_bytes, digit)
        assert p.raduls_stream_status() == 0
        np.testing.assert_array_equal(from_dev(out, n, rec_bytes // 8),
                                      oracle_mod.counting_pass(recs, key_bytes, digit))


@pytest.mark.parametrize("rec_bytes,key_bytes", SHAPES)
def test_sort_sizes_and_shapes(oracle_mod, rec_bytes, key_bytes):
    sizes = [0, 1, 2, 3, 31, 32, 33, 255, 256, 257, 1000, 4095, 4096, 4097, 8191, 8193, 40000, 300001]
    for n in sizes:
        for alphabet in (None, 2):
            recs = datagen.random_records(n, rec_bytes, key_bytes, n * 7 + rec_bytes + key_bytes, alphabet=alphabet)
            got = gpu_sort(recs, key_bytes)
            np.testing.assert_array_equal(got, oracle_mod.sort(recs, key_bytes, threads=4),
                                          err_msg=f"n={n} shape={rec_bytes},{key_bytes} alphabet={alphabet}")


def _edge_inputs(n, rec_bytes, key_bytes, seed):
    rng = np.random.default_rng(seed)
    rw, kw = rec_bytes // 8, key_bytes // 8
    base = datagen.random_records(n, rec_bytes, key_bytes, seed)
    out = {}
    eq = base.copy()
    eq[:, :kw] = base[0, :kw]
    out["all_equal"] = eq
    srt = base[np.lexsort([base[:, j] for j in range(kw - 1, -1, -1)])].copy()
    if rw > kw:
        srt[:, kw] = np.arange(n, dtype=np.uint64)
    out["sorted"] = srt
    rev = srt[::-1].copy()
    if rw > kw:
        rev[:, kw] = np.arange(n, dtype=np.uint64)
    out["reverse"] = rev
    one = base.copy()
    one[:, :kw] = 0
    one[:, kw - 1] = rng.integers(0, 256, size=n).astype(np.uint64) << np.uint64(24)
    out["one_varying_byte"] = one
    top = base.copy()
    top[:, 0] = (top[:, 0] & np.uint64(0xFFFFFF)) | np.uint64(0xABCDEF0123000000)
    out["top_bytes_constant"] = top
    hi = base.copy()
    hi[:, :kw] = rng.integers(0, 3, size=(n, kw)).astype(np.uint64) * np.uint64(0x0101010101010101)
    out["few_distinct"] = hi
    ext = base.copy()
    ext[:, :kw] = np.where(rng.random((n, kw)) < 0.5, np.uint64(0), np.uint64(2**64 - 1))
    out["extremes"] = ext
    return out


@pytest.mark.parametrize("rec_bytes,key_bytes", [(8, 8), (16, 8), (32, 16), (24, 24)])
@pytest.mark.parametrize("n", [5000, 70001])
def test_sort_edge_cases(oracle_mod, rec_bytes, key_bytes, n):
    for name, recs in _edge_inputs(n, rec_bytes, key_bytes, n + rec_bytes).items():
        got = gpu_sort(recs, key_bytes)
        np.testing.assert_array_equal(got, oracle_mod.sort(recs, key_bytes, threads=4), err_msg=name)


def test_workload_uniform8_full(oracle_mod):
    recs = datagen.uniform8()          # 2^20 x 8 B, the full small workload
    np.testing.assert_array_equal(gpu_sort(recs, 8), oracle_mod.sort(recs, 8, threads=8))


@pytest.mark.parametrize("name,n", [("uniform16", 1 << 22), ("skewed16", 1 << 22), ("widekey32", 1 << 21)])
def test_workload_prefixes(oracle_mod, name, n):
    recs = datagen.WORKLOADS[name](n)
    kb = datagen.KEY_BYTES[name]
    np.testing.assert_array_equal(gpu_sort(recs, kb), oracle_mod.sort(recs, kb, threads=8))


def test_stats_report_passes(oracle_mod):
    recs = datagen.uniform16(1 << 21)
    p = lib()
    d = to_dev(recs)
    t = scratch(recs.shape[0], 2)
    st = p.raduls_sort_ex(d, t, recs.shape[0], 16, 8, mode="plain", stats=True)
    assert st["grid_passes"] >= 1 and st["scatter_bytes"] > 0
    assert st["block_items"] + st["bucket_items"] > 0
    np.testing.assert_array_equal(from_dev(d, recs.shape[0], 2), oracle_mod.sort(recs, 8, threads=8))


def test_timeout_is_reported_and_context_survives(oracle_mod):
    """A histogram chunk withholds its look-back counts: its successor's bounded
    wait runs out, the pass reports RADULS_ERR_TIMEOUT, skips its writes, and
    the next call on the same context works."""
    p = lib()
    n = 4 * 65536 + 100
    recs = datagen.random_records(n, 16, 8, 99)
    d = to_dev(recs)
    out = scratch(n, 2)
    p.raduls_set_wait_limit_ns(200_000_000)
    try:
        p.raduls_debug_inject(1, 2)
        p.raduls_distribution_pass(d, out, n, 16, 8, 7)
        assert p.raduls_stream_status() == 6
        assert p.raduls_stream_status() == 0          # status is cleared once read
    finally:
        p.raduls_debug_inject(0, 0)
        p.raduls_set_wait_limit_ns(2_000_000_000)
    p.raduls_distribution_pass(d, out, n, 16, 8, 7)
    assert p.raduls_stream_status() == 0
    np.testing.assert_array_equal(from_dev(out, n, 2), oracle_mod.counting_pass(recs, 8, 7))
